// divide.cu -- the divide step of Alg. 1 on the GPU.
//
// Sample-based (Alg. 2): draw eta points (the eta smallest SplitMix64 keys,
// found by an 8-pass radix select), triangulate them with the engine, turn
// the sample DT into a weighted graph (Table 1 weights), partition it into k
// balanced blocks (Hilbert runs refined by size-constrained label
// propagation; stands in for KaHIP), and label every input point with the
// block of its nearest sample point by a greedy walk on the sample's
// Delaunay graph with exact distance comparisons.
// kd (Sec. 2.3): recursive median splits with cyclic dimension.
// Both end with a stable counting sort of the points by label.
#include <cmath>

#include "bbox.cuh"
#include "divide.cuh"
#include "pipeline.cuh"
#include "sort.cuh"

namespace gdt {

// ---------------------------------------------------------------- sampling
__device__ __forceinline__ unsigned long long sample_key(unsigned long long s, long long i) {
  return splitmix64(s ^ (unsigned long long)i);
}

struct SelState {
  unsigned long long prefix, mask;
  long long rank;     // rank (0-based) of the wanted key among those matching prefix
};

__global__ void k_sel_hist(int64_t n, unsigned long long s, const SelState* st, int shift, int* hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long pre = st->prefix, msk = st->mask;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long k = sample_key(s, i);
    if ((k & msk) == pre) atomicAdd(&h[(k >> shift) & 255], 1);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_sel_pick(SelState* st, int* hist, int shift) {
  long long r = st->rank, cum = 0;
  int b = 0;
  for (; b < 256; b++) {
    if (cum + hist[b] > r) break;
    cum += hist[b];
  }
  if (b > 255) b = 255;
  st->prefix |= (unsigned long long)b << shift;
  st->mask |= 255ull << shift;
  st->rank = r - cum;
  for (int i = 0; i < 256; i++) hist[i] = 0;
}

__global__ void k_sel_flag(int64_t n, unsigned long long s, const SelState* st, int* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = sample_key(s, i) <= st->prefix ? 1 : 0;
}

__global__ void k_compact_idx(const int* flag, const int* pos, int64_t n, int* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[pos[i]] = (int)i;
}

int64_t sample_size(int64_t n, double frac, int D) {
  double e = frac <= 0 ? std::ceil(std::sqrt((double)n)) : std::ceil(frac * (double)n);
  int64_t eta = (int64_t)e;
  if (eta < D + 2) eta = D + 2;
  if (eta > n) eta = n;
  return eta;
}

// Alg. 2 (sampling): the eta smallest keys splitmix64(splitmix64(seed) ^ i);
// writes their indices, ascending, to ids.
int select_sample(dt_ctx* c, int64_t n, int64_t eta, uint64_t seed, int* ids) {
  cudaStream_t s = c->stream;
  SelState* st = (SelState*)pool_get(c, "sel.st", sizeof(SelState));
  int* hist = (int*)pool_get(c, "sel.hist", 4 * 256);
  int* flag = (int*)pool_get(c, "sel.flag", 4 * n);
  int* pos = (int*)pool_get(c, "sel.pos", 4 * n);
  if (!st || !hist || !flag || !pos) return set_err(c, DT_E_NOMEM, "sample selection");
  SelState h0 = {0ull, 0ull, (long long)(eta - 1)};
  CUDA_OK(cudaMemcpyAsync(st, &h0, sizeof(h0), cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemsetAsync(hist, 0, 4 * 256, s));
  unsigned long long sm = splitmix64(seed);
  unsigned g = (unsigned)std::min<int64_t>(ceil_div<int64_t>(n, 256), 152 * 8);
  for (int shift = 56; shift >= 0; shift -= 8) {
    k_sel_hist<<<g, 256, (++c->launches, 0), s>>>(n, sm, st, shift, hist);
    k_sel_pick<<<1, 1, (++c->launches, 0), s>>>(st, hist, shift);
  }
  unsigned gn = (unsigned)ceil_div<int64_t>(n, 256);
  k_sel_flag<<<gn, 256, (++c->launches, 0), s>>>(n, sm, st, flag);
  int rc = exclusive_scan_i32(c, flag, pos, n, nullptr);
  if (rc) return rc;
  k_compact_idx<<<gn, 256, (++c->launches, 0), s>>>(flag, pos, n, ids);
  return 0;
}

template <int D>
__global__ void k_gather_pts(const typename PT<D>::T* P, const int* ids, int64_t m, typename PT<D>::T* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = P[ids[i]];
}

int gather_points(dt_ctx* c, int dim, const void* P, const int* ids, int64_t m, void* out) {
  unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(m, 1), 256);
  if (dim == 2) k_gather_pts<2><<<g, 256, (++c->launches, 0), c->stream>>>((const double2*)P, ids, m, (double2*)out);
  else k_gather_pts<3><<<g, 256, (++c->launches, 0), c->stream>>>((const double4_32a*)P, ids, m, (double4_32a*)out);
  return 0;
}

// ---------------------------------------------------------------- graph
// Edges (u < v, sample-local indices) of the live finite simplices.
template <int D>
__global__ void k_emit_edges(const int4* tv, int lo, int hi, int2* edges, int* nedges, int* ucount) {
  int s = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= hi) return;
  int4 v = tv[s];
  int a[4] = {v.x, v.y, v.z, v.w};
  for (int i = 0; i <= D; i++) if (a[i] < 0) return;
  constexpr int NE = D == 2 ? 3 : 6;
  int base = atomicAdd(nedges, NE);
  int k = 0;
  for (int i = 0; i <= D; i++)
    for (int j = i + 1; j <= D; j++) {
      int u = min(a[i], a[j]), w = max(a[i], a[j]);
      edges[base + k++] = make_int2(u, w);
      atomicAdd(&ucount[u], 1);
    }
}

__global__ void k_bucket_edges(const int2* edges, int64_t m, const int* ustart, int* ufill, int* vout) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int2 e = edges[i];
  vout[ustart[e.x] + atomicAdd(&ufill[e.x], 1)] = e.y;
}

// Sort each bucket and drop duplicates; ucount[u] becomes the unique count.
__global__ void k_unique_buckets(int* vout, const int* ustart, int* ucount, int64_t eta) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= eta) return;
  int s = ustart[u], m = ucount[u];
  for (int i = 1; i < m; i++) {
    int x = vout[s + i], j = i - 1;
    while (j >= 0 && vout[s + j] > x) { vout[s + j + 1] = vout[s + j]; j--; }
    vout[s + j + 1] = x;
  }
  int k = 0;
  for (int i = 0; i < m; i++)
    if (i == 0 || vout[s + i] != vout[s + i - 1]) vout[s + k++] = vout[s + i];
  ucount[u] = k;
}

__global__ void k_write_unique(const int* vout, const int* ustart, const int* ucount, const int* upos, int64_t eta,
                               int2* E) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= eta) return;
  for (int i = 0; i < ucount[u]; i++) E[upos[u] + i] = make_int2((int)u, vout[ustart[u] + i]);
}

// bounding box of the sample (single block)
template <int D>
__global__ void k_bbox(const typename PT<D>::T* P, int64_t n, double* box) {
  __shared__ double lo[3][256], hi[3][256];
  double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    for (int c = 0; c < D; c++) { double x = comp(P[i], c); l[c] = fmin(l[c], x); h[c] = fmax(h[c], x); }
  for (int c = 0; c < 3; c++) { lo[c][threadIdx.x] = l[c]; hi[c][threadIdx.x] = h[c]; }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int c = 0; c < 3; c++) {
        lo[c][threadIdx.x] = fmin(lo[c][threadIdx.x], lo[c][threadIdx.x + st]);
        hi[c][threadIdx.x] = fmax(hi[c][threadIdx.x], hi[c][threadIdx.x + st]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) { box[c] = lo[c][0]; box[3 + c] = hi[c][0]; }
}

// Table 1 weights on d = |v - w| / d*, d* the sample bounding-box diagonal;
// w = max(1, rint(1000 * omega)).  Plain IEEE operations (no contraction).
template <int D>
__global__ void k_edge_weights(const typename PT<D>::T* P, const int2* E, int64_t m, const double* box, int kind,
                               long long* w) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  double ds = 0;
  for (int c = 0; c < D; c++) {
    double e = __dsub_rn(box[3 + c], box[c]);
    ds = __dadd_rn(ds, __dmul_rn(e, e));
  }
  double dstar = __dsqrt_rn(ds);
  int2 e = E[i];
  double sq = 0;
  for (int c = 0; c < D; c++) {
    double x = __dsub_rn(comp(P[e.x], c), comp(P[e.y], c));
    sq = c == 0 ? __dmul_rn(x, x) : __dadd_rn(sq, __dmul_rn(x, x));
  }
  double d = __ddiv_rn(__dsqrt_rn(sq), dstar);
  double om;
  if (kind == DT_WEIGHT_LOG) om = -log(d);
  else if (kind == DT_WEIGHT_CONSTANT) om = 1.0 / 1000.0;
  else if (kind == DT_WEIGHT_INVERSE) om = fmin(__ddiv_rn(1.0, d), 1e6);
  else om = __dsub_rn(1.0, d);
  double r = rint(__dmul_rn(1000.0, om));
  w[i] = r < 1.0 ? 1 : (long long)r;
}

// CSR (both directions) from unique edges.
__global__ void k_degree(const int2* E, int64_t m, int* deg) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  atomicAdd(&deg[E[i].x], 1);
  atomicAdd(&deg[E[i].y], 1);
}
__global__ void k_fill_csr(const int2* E, const long long* w, int64_t m, const int* rowptr, int* fill, int* col,
                           long long* cw) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int2 e = E[i];
  int a = rowptr[e.x] + atomicAdd(&fill[e.x], 1);
  col[a] = e.y; cw[a] = w[i];
  int b = rowptr[e.y] + atomicAdd(&fill[e.y], 1);
  col[b] = e.x; cw[b] = w[i];
}

int graph_bbox(dt_ctx* c, int dim, const void* PS, int64_t eta, double* box) {
  if (dim == 2) k_bbox<2><<<1, 256, (++c->launches, 0), c->stream>>>((const double2*)PS, eta, box);
  else k_bbox<3><<<1, 256, (++c->launches, 0), c->stream>>>((const double4_32a*)PS, eta, box);
  return 0;
}

int build_csr(dt_ctx* c, SampleGraph& G) {
  cudaStream_t s = c->stream;
  int64_t eta = G.eta;
  G.rowptr = (int*)pool_get(c, "g.rowptr", 4 * (eta + 1));
  int* deg = (int*)pool_get(c, "g.deg", 4 * (eta + 1));
  int* fill = (int*)pool_get(c, "g.fill", 4 * (eta + 1));
  G.col = (int*)pool_get(c, "g.col", 4 * std::max<int64_t>(2 * G.m, 1));
  G.cw = (long long*)pool_get(c, "g.cw", 8 * std::max<int64_t>(2 * G.m, 1));
  if (!G.rowptr || !deg || !fill || !G.col || !G.cw) return set_err(c, DT_E_NOMEM, "csr");
  CUDA_OK(cudaMemsetAsync(deg, 0, 4 * (eta + 1), s));
  CUDA_OK(cudaMemsetAsync(fill, 0, 4 * (eta + 1), s));
  unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(G.m, 1), 256);
  if (G.m) k_degree<<<g, 256, (++c->launches, 0), s>>>(G.E, G.m, deg);
  int rc = exclusive_scan_i32(c, deg, G.rowptr, eta + 1, nullptr);
  if (rc) return rc;
  if (G.m) k_fill_csr<<<g, 256, (++c->launches, 0), s>>>(G.E, G.w, G.m, G.rowptr, fill, G.col, G.cw);
  return 0;
}

// Alg. 2 (sample triangulation and graph): G = (P_S, edges of DT(P_S), omega).
int sample_graph(dt_ctx* c, const EngineRun& run, const void* PS, int dim, int kind, SampleGraph& G) {
  cudaStream_t s = c->stream;
  int64_t eta = run.npts;
  G.eta = eta;
  int lo = (int)run.h_toff[0], hi = run.h_tcount[0];
  int64_t maxe = (int64_t)(hi - lo) * (dim == 2 ? 3 : 6) + 1;
  int2* raw = (int2*)pool_get(c, "g.raw", 8 * maxe);
  int* cnt = (int*)pool_get(c, "g.cnt", 16);
  int* ucount = (int*)pool_get(c, "g.ucount", 4 * (eta + 1));
  int* ustart = (int*)pool_get(c, "g.ustart", 4 * (eta + 1));
  int* ufill = (int*)pool_get(c, "g.ufill", 4 * (eta + 1));
  int* vout = (int*)pool_get(c, "g.vout", 4 * maxe);
  int* upos = (int*)pool_get(c, "g.upos", 4 * (eta + 1));
  G.box = (double*)pool_get(c, "g.box", 8 * 6);
  if (!raw || !cnt || !ucount || !ustart || !ufill || !vout || !upos || !G.box)
    return set_err(c, DT_E_NOMEM, "sample graph");
  CUDA_OK(cudaMemsetAsync(cnt, 0, 16, s));
  CUDA_OK(cudaMemsetAsync(ucount, 0, 4 * (eta + 1), s));
  CUDA_OK(cudaMemsetAsync(ufill, 0, 4 * (eta + 1), s));
  unsigned g = (unsigned)ceil_div(std::max(hi - lo, 1), 256);
  if (dim == 2) k_emit_edges<2><<<g, 256, (++c->launches, 0), s>>>((const int4*)run.tv, lo, hi, raw, cnt, ucount);
  else k_emit_edges<3><<<g, 256, (++c->launches, 0), s>>>((const int4*)run.tv, lo, hi, raw, cnt, ucount);
  int nraw = 0;
  CUDA_OK(cudaMemcpyAsync(&nraw, cnt, 4, cudaMemcpyDeviceToHost, s));
  int rc = exclusive_scan_i32(c, ucount, ustart, eta + 1, nullptr);
  if (rc) return rc;
  CUDA_OK(cudaStreamSynchronize(s));
  unsigned ge = (unsigned)ceil_div<int64_t>(std::max(nraw, 1), 256);
  k_bucket_edges<<<ge, 256, (++c->launches, 0), s>>>(raw, nraw, ustart, ufill, vout);
  unsigned gu = (unsigned)ceil_div<int64_t>(eta, 128);
  k_unique_buckets<<<gu, 128, (++c->launches, 0), s>>>(vout, ustart, ucount, eta);
  int m = 0;
  rc = exclusive_scan_i32(c, ucount, upos, eta + 1, &m);
  if (rc) return rc;
  G.m = m;
  G.E = (int2*)pool_get(c, "g.E", 8 * std::max(m, 1));
  G.w = (long long*)pool_get(c, "g.w", 8 * std::max(m, 1));
  if (!G.E || !G.w) return set_err(c, DT_E_NOMEM, "graph edges");
  k_write_unique<<<gu, 128, (++c->launches, 0), s>>>(vout, ustart, ucount, upos, eta, G.E);
  if (dim == 2) k_bbox<2><<<1, 256, (++c->launches, 0), s>>>((const double2*)PS, eta, G.box);
  else k_bbox<3><<<1, 256, (++c->launches, 0), s>>>((const double4_32a*)PS, eta, G.box);
  unsigned gm = (unsigned)ceil_div<int64_t>(std::max(m, 1), 256);
  if (m) {
    if (dim == 2) k_edge_weights<2><<<gm, 256, (++c->launches, 0), s>>>((const double2*)PS, G.E, m, G.box, kind, G.w);
    else k_edge_weights<3><<<gm, 256, (++c->launches, 0), s>>>((const double4_32a*)PS, G.E, m, G.box, kind, G.w);
  }
  return build_csr(c, G);
}

// ---------------------------------------------------------------- partition
// Skilling's transpose construction of the Hilbert index.
__device__ __forceinline__ uint32_t hilbert_key(uint32_t* X, int n, int bits) {
  uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    uint32_t P = Q - 1;
    for (int i = 0; i < n; i++) {
      if (X[i] & Q) X[0] ^= P;
      else { uint32_t t = (X[0] ^ X[i]) & P; X[0] ^= t; X[i] ^= t; }
    }
  }
  for (int i = 1; i < n; i++) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1) if (X[n - 1] & Q) t ^= Q - 1;
  for (int i = 0; i < n; i++) X[i] ^= t;
  uint32_t key = 0;
  for (int b = bits - 1; b >= 0; b--)
    for (int i = 0; i < n; i++) key = (key << 1) | ((X[i] >> b) & 1u);
  return key;
}

template <int D>
__global__ void k_hilbert(const typename PT<D>::T* P, int64_t n, const double* box, int bits, uint32_t* keys,
                          int* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t X[3] = {0, 0, 0};
  for (int c = 0; c < D; c++) {
    double lo = box[c], hi = box[3 + c];
    if (hi > lo) {
      double w = __dmul_rn(__ddiv_rn(__dsub_rn(comp(P[i], c), lo), __dsub_rn(hi, lo)), (double)(1u << bits));
      double f = floor(w);
      double mx = (double)((1u << bits) - 1);
      X[c] = (uint32_t)(f < mx ? f : mx);
    }
  }
  keys[i] = hilbert_key(X, D, bits);
  idx[i] = (int)i;
}

__global__ void k_initial_blocks(const int* order, int64_t eta, int k, int* block) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < eta) block[order[r]] = (int)((r * k) / eta);
}

// One label-propagation proposal per vertex of this round's parity class.
__global__ void k_lp_propose(const int* rowptr, const int* col, const long long* cw, const int* block, int64_t eta,
                             int parity, int* target) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= eta) return;
  int t = -1;
  if ((v & 1) == parity) {
    int a = rowptr[v], b = rowptr[v + 1];
    int own = block[v];
    long long ownw = 0, bestw = -1;
    int best = -1;
    for (int j = a; j < b; j++) {
      int bj = block[col[j]];
      bool seen = false;
      for (int l = a; l < j; l++) if (block[col[l]] == bj) { seen = true; break; }
      if (seen) continue;
      long long sum = 0;
      for (int l = j; l < b; l++) if (block[col[l]] == bj) sum += cw[l];
      if (bj == own) { ownw = sum; continue; }
      if (sum > bestw || (sum == bestw && bj < best)) { bestw = sum; best = bj; }
    }
    if (best >= 0 && bestw > ownw) t = best;
  }
  target[v] = t;
}

__global__ void k_lp_source(const int* target, const int* block, int64_t eta, int* source) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < eta) source[v] = target[v] >= 0 ? block[v] : -1;
}

__global__ void k_lp_apply(const int* target, const int* rankT, const int* rankS, const int* sizes, int64_t eta,
                           int lmin, int lmax, int* block) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= eta) return;
  int t = target[v];
  if (t < 0) return;
  int a = block[v];
  if (rankT[v] < lmax - sizes[t] && rankS[v] < sizes[a] - lmin) block[v] = t;
}

void partition_bounds(int64_t eta, int k, double eps, int* lmin, int* lmax) {
  int64_t ideal = (eta + k - 1) / k;
  *lmax = (int)std::floor((1.0 + eps) * (double)ideal);
  int64_t l = (int64_t)std::floor((1.0 - eps) * (double)eta / (double)k);
  *lmin = (int)std::max<int64_t>(1, l);
}

// Size-constrained k-way partition (see the oracle's partition() for the
// exact rule); block[] receives eta labels.
int partition_graph(dt_ctx* c, const void* PS, int dim, SampleGraph& G, int k, double eps, int rounds, int init,
                    int* block) {
  cudaStream_t s = c->stream;
  int64_t eta = G.eta;
  if (k <= 1) { CUDA_OK(cudaMemsetAsync(block, 0, 4 * eta, s)); return 0; }
  if (k > 256) return set_err(c, DT_E_ARG, "the sample partitioner supports k <= 256");
  uint32_t* keys = (uint32_t*)pool_get(c, "p.keys", 4 * eta);
  int* idx = (int*)pool_get(c, "p.idx", 4 * eta);
  int* target = (int*)pool_get(c, "p.target", 4 * eta);
  int* source = (int*)pool_get(c, "p.source", 4 * eta);
  int* rankT = (int*)pool_get(c, "p.rankT", 4 * eta);
  int* rankS = (int*)pool_get(c, "p.rankS", 4 * eta);
  int* rankB = (int*)pool_get(c, "p.rankB", 4 * eta);
  int* sizes = (int*)pool_get(c, "p.sizes", 4 * 256);
  if (!keys || !idx || !target || !source || !rankT || !rankS || !rankB || !sizes)
    return set_err(c, DT_E_NOMEM, "partition buffers");
  unsigned g = (unsigned)ceil_div<int64_t>(eta, 256);
  int rc;
  if (init == DT_INIT_KD || init == DT_INIT_AUTO) {
    // the comparator's median cuts, applied to the sample
    rc = kd_divide(c, dim, PS, eta, k, block, "pkd");
    if (rc) return rc;
  } else {
    int bits = dim == 2 ? 16 : 10;
    if (dim == 2) k_hilbert<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)PS, eta, G.box, bits, keys, idx);
    else k_hilbert<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)PS, eta, G.box, bits, keys, idx);
    rc = radix_sort_pairs<uint32_t, int>(c, keys, idx, eta, bits * dim, "p.sort");
    if (rc) return rc;
    k_initial_blocks<<<g, 256, (++c->launches, 0), s>>>(idx, eta, k, block);
  }
  if (c->cfg.partitioner == DT_PART_MULTILEVEL) return partition_multilevel(c, G, k, eps, rounds, block);
  int lmin, lmax;
  partition_bounds(eta, k, eps, &lmin, &lmax);
  for (int r = 0; r < rounds; r++) {
    rc = group_rank(c, block, eta, rankB, sizes, k);
    if (rc) return rc;
    k_lp_propose<<<g, 256, (++c->launches, 0), s>>>(G.rowptr, G.col, G.cw, block, eta, r & 1, target);
    k_lp_source<<<g, 256, (++c->launches, 0), s>>>(target, block, eta, source);
    rc = group_rank(c, target, eta, rankT, nullptr, k);
    if (rc) return rc;
    rc = group_rank(c, source, eta, rankS, nullptr, k);
    if (rc) return rc;
    k_lp_apply<<<g, 256, (++c->launches, 0), s>>>(target, rankT, rankS, sizes, eta, lmin, lmax, block);
  }
  return 0;
}

__global__ void k_cut_weight(const int2* E, const long long* w, int64_t m, const int* block,
                             unsigned long long* cut) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m && block[E[i].x] != block[E[i].y]) atomicAdd(cut, (unsigned long long)w[i]);
}

int cut_weight(dt_ctx* c, const SampleGraph& G, const int* block, long long* out) {
  unsigned long long* d = (unsigned long long*)pool_get(c, "p.cut", 8);
  if (!d) return set_err(c, DT_E_NOMEM, "cut");
  CUDA_OK(cudaMemsetAsync(d, 0, 8, c->stream));
  if (G.m)
    k_cut_weight<<<(unsigned)ceil_div<int64_t>(G.m, 256), 256, (++c->launches, 0), c->stream>>>(G.E, G.w, G.m, block, d);
  unsigned long long h = 0;
  CUDA_OK(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  *out = (long long)h;
  return 0;
}

// ---------------------------------------------------------------- labels
__global__ void k_fill_int(int* a, int64_t n, int v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

struct StartGrid {
  double lo[3], inv[3];
  int dims[3];
};

template <int D>
__device__ __forceinline__ int64_t grid_cell(const typename PT<D>::T& p, const StartGrid& sg) {
  int64_t id = 0;
  for (int c = D - 1; c >= 0; c--) {
    double f = (comp(p, c) - sg.lo[c]) * sg.inv[c];
    int x = f < 0 ? 0 : (f >= sg.dims[c] ? sg.dims[c] - 1 : (int)f);
    id = id * sg.dims[c] + x;
  }
  return id;
}

template <int D>
__global__ void k_seed_cells(const typename PT<D>::T* S, int64_t m, StartGrid sg, int* cellv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) atomicMin(&cellv[grid_cell<D>(S[i], sg)], (int)i);
}

// one dilation pass: an empty cell takes the smallest seed among face neighbours
template <int D>
__global__ void k_dilate(const int* in, int* out, StartGrid sg, int64_t ncell) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int v = in[id];
  if (v == 0x7fffffff) {
    int64_t rem = id, stride = 1;
    for (int c = 0; c < D; c++) {
      int x = (int)(rem % sg.dims[c]);
      rem /= sg.dims[c];
      if (x > 0) v = min(v, in[id - stride]);
      if (x + 1 < sg.dims[c]) v = min(v, in[id + stride]);
      stride *= sg.dims[c];
    }
  }
  out[id] = v;
}

// FP32 copies of the sample points relative to the origin o (the centre of the
// points' bounding box): X = fl32(fl64(x - o)).
template <int D>
__global__ void k_sample_x32(const typename PT<D>::T* S, int64_t m, StartGrid sg, double3 o, float4* XS) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m) return;
  const typename PT<D>::T q = S[j];
  XS[j] = make_float4((float)(cx(q) - o.x), (float)(cy(q) - o.y), D == 3 ? (float)(cz(q) - o.z) : 0.0f, 0.0f);
}

// First stage of sign(|p - a|^2 - |p - b|^2) in FP32 with a rigorous bound.
// Every copy X = fl32(fl64(x - o)) is within (u32 + 2 u64) R of x - o (R: the
// largest |x_c - o_c|), so a difference A = fl32(Xa - Xp) is within
// e(A) = eta + u32 |A| (1 + 2 u32) of a - p, eta = 2 (u32 + 2 u64) R.  Then
// |A^2 - (a - p)^2| <= e (2 |A| + e), the sums of three squares are exact to
// gamma_3 = 3 u32 / (1 - 3 u32) of themselves and the final difference to u32
// of itself; the bound is evaluated in FP32 and enlarged by 0.1 % to cover its
// own roundings.  Returns -1 / +1 when decided, 0 when the FP64 test must run.
template <int D>
__device__ __forceinline__ int closer_f32(const float4& xp, const float4& xa, const float4& xb, float eta) {
  const float u = 5.9604645e-8f;                      // 2^-24
  const float ax = xa.x - xp.x, ay = xa.y - xp.y, az = D == 3 ? xa.z - xp.z : 0.0f;
  const float bx = xb.x - xp.x, by = xb.y - xp.y, bz = D == 3 ? xb.z - xp.z : 0.0f;
  const float sa = fmaf(az, az, fmaf(ay, ay, ax * ax));
  const float sb = fmaf(bz, bz, fmaf(by, by, bx * bx));
  const float d = sa - sb;
  auto term = [&](float t) {
    const float at = fabsf(t), e = fmaf(u * (1.0f + 2.0f * u), at, eta);
    return e * (2.0f * at + e);
  };
  const float g3 = 3.0f * u / (1.0f - 3.0f * u);
  const float err = 1.001f * (g3 * (1.0f + g3) * (sa + sb) + term(ax) + term(ay) + term(az) + term(bx) + term(by) +
                              term(bz)) + 2.0f * u * fabsf(d);
  if (!(err < 1e30f) || !(sa + sb > 1e-30f)) return 0;   // outside the range the bound covers
  if (d > err) return 1;
  if (d < -err) return -1;
  return 0;
}

// Greedy walk on the sample Delaunay graph to the exactly nearest sample
// point (ties: smaller global index); label = its block.  Distances are
// compared in FP32 first (closer_f32), in FP64 and exactly (closer) when that
// cannot decide.
template <int D>
__global__ void k_label_walk(const typename PT<D>::T* P, int64_t n, const typename PT<D>::T* S, const int* srank,
                             const int* rowptr, const int* col, const int* block, const int* cellv, StartGrid sg,
                             int64_t m, int* label, int* nearest, DevStatus* st, const float4* XS, double3 o,
                             float eta) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename PT<D>::T p = P[i];
  const float4 xp = make_float4((float)(cx(p) - o.x), (float)(cy(p) - o.y), D == 3 ? (float)(cz(p) - o.z) : 0.0f, 0.0f);
  int v = cellv[grid_cell<D>(p, sg)];
  if (v < 0 || v >= m) v = 0;
  for (int64_t step = 0; step <= m; step++) {
    int a = rowptr[v], b = rowptr[v + 1];
    int nv = -1;
    const float4 xv = XS[v];
    for (int j = a; j < b; j++) {
      int w = col[j];
      int cmp = closer_f32<D>(xp, XS[w], xv, eta);
      if (cmp == 0) cmp = closer(p, S[w], S[v], D);
      if (cmp < 0 || (cmp == 0 && srank[w] < srank[v])) { nv = w; break; }
    }
    if (nv < 0) break;
    v = nv;
    if (step == m) set_error(st, DT_E_TIMEOUT, 20);
  }
  if (label) label[i] = block[v];
  if (nearest) nearest[i] = v;
}

// label[i] = block[nearest[i]]: the labels once the partition is known (the walk to the
// nearest sample point does not depend on the blocks and can run beside the partitioner).
__global__ void k_map_labels(const int* nearest, const int* block, int64_t n, int* label) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) label[i] = block[nearest[i]];
}

int map_labels(dt_ctx* c, const int* nearest, const int* block, int64_t n, int* label) {
  if (n > 0)
    k_map_labels<<<(unsigned)ceil_div<int64_t>(n, 256), 256, (++c->launches, 0), c->stream>>>(nearest, block, n, label);
  return 0;
}

int label_points(dt_ctx* c, int dim, const void* P, int64_t n, const void* S, const int* srank, const SampleGraph& G,
                 const int* block, int* label, int* nearest) {
  cudaStream_t s = c->stream;
  int64_t m = G.eta;
  // start grid over the bounding box of all points, about m/4 cells
  double* box = (double*)pool_get(c, "lw.box", 48);
  unsigned long long* ub = (unsigned long long*)pool_get(c, "lw.ubox", 48);
  if (!box || !ub) return set_err(c, DT_E_NOMEM, "label box");
  k_box_init<<<1, 32, (++c->launches, 0), s>>>(ub, 1);
  if (dim == 2) k_box_reduce<2><<<box_grid(n), 256, (++c->launches, 0), s>>>((const double2*)P, nullptr, n, ub);
  else k_box_reduce<3><<<box_grid(n), 256, (++c->launches, 0), s>>>((const double4_32a*)P, nullptr, n, ub);
  k_box_to_double<<<1, 32, (++c->launches, 0), s>>>(ub, 1, dim, box);
  double hb[6];
  CUDA_OK(cudaMemcpyAsync(hb, box, 48, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  StartGrid sg;
  double vol = 1.0;
  int nd = 0;
  for (int cc = 0; cc < dim; cc++) if (hb[3 + cc] > hb[cc]) { vol *= hb[3 + cc] - hb[cc]; nd++; }
  double target = std::max<double>(1.0, (double)m / 4.0);
  double side = nd ? std::pow(vol / target, 1.0 / nd) : 1.0;
  int64_t ncell = 1;
  for (int cc = 0; cc < 3; cc++) {
    sg.lo[cc] = cc < dim ? hb[cc] : 0;
    double ext = cc < dim ? hb[3 + cc] - hb[cc] : 0;
    int d = (cc < dim && ext > 0 && side > 0) ? (int)std::min(1024.0, std::max(1.0, std::ceil(ext / side))) : 1;
    sg.dims[cc] = d;
    sg.inv[cc] = (ext > 0) ? d / ext : 0.0;
    ncell *= d;
  }
  int* cv0 = (int*)pool_get(c, "lw.cv0", 4 * ncell);
  int* cv1 = (int*)pool_get(c, "lw.cv1", 4 * ncell);
  if (!cv0 || !cv1) return set_err(c, DT_E_NOMEM, "label grid");
  unsigned gm = (unsigned)ceil_div<int64_t>(m, 256);
  k_fill_int<<<(unsigned)ceil_div<int64_t>(ncell, 256), 256, (++c->launches, 0), s>>>(cv0, ncell, 0x7fffffff);
  if (dim == 2) k_seed_cells<2><<<gm, 256, (++c->launches, 0), s>>>((const double2*)S, m, sg, cv0);
  else k_seed_cells<3><<<gm, 256, (++c->launches, 0), s>>>((const double4_32a*)S, m, sg, cv0);
  unsigned gc = (unsigned)ceil_div<int64_t>(ncell, 256);
  for (int pass = 0; pass < 6; pass++) {
    if (dim == 2) k_dilate<2><<<gc, 256, (++c->launches, 0), s>>>(cv0, cv1, sg, ncell);
    else k_dilate<3><<<gc, 256, (++c->launches, 0), s>>>(cv0, cv1, sg, ncell);
    std::swap(cv0, cv1);
  }
  // FP32 stage: origin at the box centre, eta = 2 (u32 + 2 u64) R rounded up
  double oc[3] = {0, 0, 0}, R = 0.0;
  for (int cc = 0; cc < dim; cc++) {
    oc[cc] = 0.5 * hb[cc] + 0.5 * hb[3 + cc];
    R = std::max(R, std::max(hb[3 + cc] - oc[cc], oc[cc] - hb[cc]));
  }
  const double3 o = make_double3(oc[0], oc[1], oc[2]);
  const double etad = 2.02 * (std::ldexp(1.0, -24) + std::ldexp(1.0, -52)) * R * (1.0 + 1e-9);
  float eta = (float)etad;
  if (!((double)eta >= etad)) eta = std::nextafter(eta, INFINITY);
  float4* XS = (float4*)pool_get(c, "lw.xs", 16 * (size_t)std::max<int64_t>(m, 1));
  if (!XS) return set_err(c, DT_E_NOMEM, "label walk copies");
  if (dim == 2) k_sample_x32<2><<<gm, 256, (++c->launches, 0), s>>>((const double2*)S, m, sg, o, XS);
  else k_sample_x32<3><<<gm, 256, (++c->launches, 0), s>>>((const double4_32a*)S, m, sg, o, XS);
  unsigned gn = (unsigned)ceil_div<int64_t>(n, 128);
  if (dim == 2)
    k_label_walk<2><<<gn, 128, (++c->launches, 0), s>>>((const double2*)P, n, (const double2*)S, srank, G.rowptr, G.col, block, cv0, sg,
                                       m, label, nearest, c->status, XS, o, eta);
  else
    k_label_walk<3><<<gn, 128, (++c->launches, 0), s>>>((const double4_32a*)P, n, (const double4_32a*)S, srank, G.rowptr, G.col, block, cv0, sg,
                                       m, label, nearest, c->status, XS, o, eta);
  return 0;
}


// ---------------------------------------------------------------- kd divide
__device__ __forceinline__ unsigned long long orderable(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);   // -0.0 -> +0.0
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <int D>
__global__ void k_kd_keys(const typename PT<D>::T* P, int64_t n, int dimc, unsigned long long* keys, int* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) { keys[i] = orderable(comp(P[i], dimc)); idx[i] = (int)i; }
}

__global__ void k_kd_nodekeys(const int* idx, const int* label, int64_t n, uint32_t* nkeys) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) nkeys[j] = (uint32_t)label[idx[j]];
}

// node tables indexed by node id (= first leaf): start, left size, left leaves, leaves
__global__ void k_kd_assign(const int* idx, int64_t n, const int* nstart, const int* nml, const int* nkl,
                            const int* nkk, int* label) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int p = idx[j];
  int node = label[p];
  if (nkk[node] <= 1) return;
  int pos = (int)(j - nstart[node]);
  label[p] = pos < nml[node] ? node : node + nkl[node];
}

int kd_divide(dt_ctx* c, int dim, const void* P, int64_t n, int k, int* label, const char* tag) {
  cudaStream_t s = c->stream;
  const std::string t(tag);
  unsigned long long* keys = (unsigned long long*)pool_get(c, t + ".keys", 8 * n);
  int* idx = (int*)pool_get(c, t + ".idx", 4 * n);
  uint32_t* nkeys = (uint32_t*)pool_get(c, t + ".nkeys", 4 * n);
  int* tabs = (int*)pool_get(c, t + ".tabs", 4 * 4 * (size_t)k);
  if (!keys || !idx || !nkeys || !tabs) return set_err(c, DT_E_NOMEM, "kd buffers");
  CUDA_OK(cudaMemsetAsync(label, 0, 4 * n, s));
  struct Node { int first, kk; int64_t size; };
  std::vector<Node> nodes = {{0, k, n}};
  int nbits = 1;
  while ((1 << nbits) < k) nbits++;
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  for (int depth = 0;; depth++) {
    bool any = false;
    for (auto& nd : nodes) any |= nd.kk > 1;
    if (!any) break;
    std::vector<int> hs(4 * (size_t)k, 0);
    int64_t start = 0;
    std::vector<Node> next;
    for (auto& nd : nodes) {
      int kl = nd.kk / 2;
      int64_t ml = nd.kk > 1 ? (nd.size * kl) / nd.kk : nd.size;
      hs[nd.first] = (int)start;
      hs[k + nd.first] = (int)ml;
      hs[2 * k + nd.first] = kl;
      hs[3 * k + nd.first] = nd.kk;
      start += nd.size;
      if (nd.kk > 1) {
        next.push_back({nd.first, kl, ml});
        next.push_back({nd.first + kl, nd.kk - kl, nd.size - ml});
      } else {
        next.push_back(nd);
      }
    }
    CUDA_OK(cudaMemcpyAsync(tabs, hs.data(), 4 * 4 * (size_t)k, cudaMemcpyHostToDevice, s));
    int cdim = depth % dim;
    if (dim == 2) k_kd_keys<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)P, n, cdim, keys, idx);
    else k_kd_keys<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)P, n, cdim, keys, idx);
    int rc = radix_sort_pairs<unsigned long long, int>(c, keys, idx, n, 64, t + ".s1");
    if (rc) return rc;
    k_kd_nodekeys<<<g, 256, (++c->launches, 0), s>>>(idx, label, n, nkeys);
    rc = radix_sort_pairs<uint32_t, int>(c, nkeys, idx, n, nbits, t + ".s2");
    if (rc) return rc;
    k_kd_assign<<<g, 256, (++c->launches, 0), s>>>(idx, n, tabs, tabs + k, tabs + 2 * k, tabs + 3 * k, label);
    nodes = next;
    CUDA_OK(cudaStreamSynchronize(s));   // host tables are reused next level
  }
  return 0;
}

// ---------------------------------------------------------------- scatter
template <int D>
__global__ void k_scatter(const typename PT<D>::T* P, const int* label, const int* rank, const int* poff, int64_t n,
                          typename PT<D>::T* Ps, int* gid, int* pinst, int* where) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l = label[i];
  int pos = poff[l] + rank[i];
  Ps[pos] = P[i];
  gid[pos] = (int)i;
  pinst[pos] = l;
  if (where) where[i] = pos;
}

// Stable counting sort of the points by label; poff (host) receives k+1 offsets.
int scatter_by_label(dt_ctx* c, int dim, const void* P, const int* label, int64_t n, int k, void* Ps, int* gid,
                     int* pinst, std::vector<int64_t>& poff, std::vector<int64_t>& sizes_out) {
  cudaStream_t s = c->stream;
  int* rank = (int*)pool_get(c, "sc.rank", 4 * n);
  int* sizes = (int*)pool_get(c, "sc.sizes", 4 * (k + 1));
  int* dpoff = (int*)pool_get(c, "sc.poff", 4 * (k + 1));
  if (!rank || !sizes || !dpoff) return set_err(c, DT_E_NOMEM, "scatter");
  int rc = group_rank(c, label, n, rank, sizes, k);
  if (rc) return rc;
  std::vector<int> hs(k);
  CUDA_OK(cudaMemcpyAsync(hs.data(), sizes, 4 * k, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  poff.assign(k + 1, 0);
  sizes_out.assign(k, 0);
  std::vector<int> hp(k + 1, 0);
  for (int i = 0; i < k; i++) { poff[i + 1] = poff[i] + hs[i]; hp[i + 1] = (int)poff[i + 1]; sizes_out[i] = hs[i]; }
  if (poff[k] != n) return set_err(c, DT_E_INTERNAL, "labels out of range");
  CUDA_OK(cudaMemcpyAsync(dpoff, hp.data(), 4 * (k + 1), cudaMemcpyHostToDevice, s));
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  if (dim == 2) k_scatter<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)P, label, rank, dpoff, n, (double2*)Ps, gid, pinst, nullptr);
  else k_scatter<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)P, label, rank, dpoff, n, (double4_32a*)Ps, gid, pinst, nullptr);
  return 0;
}

}  // namespace gdt
