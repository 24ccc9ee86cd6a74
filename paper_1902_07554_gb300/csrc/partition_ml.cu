// partition_ml.cu -- multilevel refinement of the sample partition (the
// graph-partitioning step of Alg. 2; KaHIP, which the paper uses, is not
// available).
//
// Starting from the initial blocks, heavy-edge matchings inside the blocks
// coarsen the sample graph level by level (a coarse vertex is a matched pair,
// its weight the pair's total); the coarse graphs inherit the blocks, so every
// level has the same block weights.  Then, from the coarsest level down,
// rounds of size-constrained label propagation with vertex weights refine the
// blocks, which are projected to the next finer level.  A move on a coarse
// level moves a whole cluster of sample points at once.  Every step is
// deterministic (synchronous sweeps, ties broken by index) and follows the
// oracle's ml_partition rule for rule.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "divide.cuh"
#include "sort.cuh"

namespace gdt {

namespace {

constexpr int ML_SWEEPS = 4;       // handshake sweeps per matching
constexpr int ML_MAX_LEVELS = 12;  // levels including the sample graph itself
constexpr int ML_NONE = 256;       // group key of "no candidate" (blocks are < 256)

struct MLGraph {
  int64_t n = 0, nnz = 0;
  int* rowptr = nullptr;   // n + 1
  int* col = nullptr;      // nnz
  long long* cw = nullptr; // nnz edge weights
  int* vw = nullptr;       // n vertex weights
  int* block = nullptr;    // n
  int* cmap = nullptr;     // n: coarse vertex of the next level (levels that were coarsened)
};

__global__ void k_ml_fill(int* a, int64_t n, int v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// Handshake preference: the unmatched neighbour in the same block whose pair
// weight stays within cmax, with the heaviest edge (ties: smaller index).
__global__ void k_ml_pref(MLGraph g, const int* mate, int cmax, int* pref) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= g.n) return;
  int best = -1;
  long long bw = -1;
  if (mate[v] < 0) {
    const int bv = g.block[v], wv = g.vw[v];
    for (int j = g.rowptr[v]; j < g.rowptr[v + 1]; j++) {
      const int u = g.col[j];
      if (mate[u] >= 0 || g.block[u] != bv || g.vw[u] + wv > cmax) continue;
      const long long w = g.cw[j];
      if (w > bw || (w == bw && u < best)) { best = u; bw = w; }
    }
  }
  pref[v] = best;
}

__global__ void k_ml_mutual(int64_t n, const int* pref, int* mate) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int p = pref[v];
  if (mate[v] < 0 && p >= 0 && pref[p] == (int)v) mate[v] = p;
}

// A pair is represented by its smaller vertex, an unmatched vertex by itself.
__global__ void k_ml_isrep(int64_t n, const int* mate, int* isrep) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) isrep[v] = (mate[v] < 0 || (int)v < mate[v]) ? 1 : 0;
}

__global__ void k_ml_cmap(MLGraph g, const int* mate, const int* cid, int* cvw, int* cblock) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= g.n) return;
  const int m = mate[v];
  const int rep = (m >= 0 && m < (int)v) ? m : (int)v;
  g.cmap[v] = cid[rep];
  if (rep == (int)v) {
    cvw[cid[v]] = g.vw[v] + (m >= 0 ? g.vw[m] : 0);
    cblock[cid[v]] = g.block[v];
  }
}

// Key of every directed fine edge: (coarse row) * nc + (coarse column), or the
// sentinel nc * nc for an edge inside a pair.
__global__ void k_ml_edge_keys(MLGraph g, unsigned long long nc, unsigned long long* keys, int* vals) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= g.n) return;
  const unsigned long long a = (unsigned long long)g.cmap[v];
  for (int j = g.rowptr[v]; j < g.rowptr[v + 1]; j++) {
    const unsigned long long b = (unsigned long long)g.cmap[g.col[j]];
    keys[j] = a != b ? a * nc + b : nc * nc;
    vals[j] = j;
  }
}

__global__ void k_ml_uflag(int64_t m, const unsigned long long* keys, unsigned long long sentinel, int* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) flag[i] = (keys[i] != sentinel && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
}

// The coarse CSR: one entry per distinct (row, column), weights summed
// (integer sums: the order of the additions does not matter).
__global__ void k_ml_cedges(int64_t m, const unsigned long long* keys, const int* vals, const long long* fcw,
                            const int* flag, const int* uid, unsigned long long nc, int* ccol, long long* ccw,
                            int* crowcnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m || keys[i] == nc * nc) return;
  const int e = uid[i] + flag[i] - 1;
  atomicAdd((unsigned long long*)&ccw[e], (unsigned long long)fcw[vals[i]]);
  if (flag[i]) {
    ccol[e] = (int)(keys[i] % nc);
    atomicAdd(&crowcnt[keys[i] / nc], 1);
  }
}

__global__ void k_ml_block_weights(MLGraph g, long long* W) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < g.n) atomicAdd((unsigned long long*)&W[g.block[v]], (unsigned long long)g.vw[v]);
}

// Label-propagation proposal of vertex v (this round's parity class): the
// neighbouring block with the largest total edge weight (ties: smaller
// block), if it beats v's own block; -1 otherwise.
__global__ void k_ml_propose(MLGraph g, int parity, int* target, int* tkey, int* skey, int* idx) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= g.n) return;
  int t = -1;
  if ((v & 1) == parity) {
    const int a = g.rowptr[v], b = g.rowptr[v + 1];
    const int own = g.block[v];
    long long ownw = 0, bestw = -1;
    int best = -1;
    for (int j = a; j < b; j++) {
      const int bj = g.block[g.col[j]];
      bool seen = false;
      for (int l = a; l < j; l++)
        if (g.block[g.col[l]] == bj) { seen = true; break; }
      if (seen) continue;
      long long sum = 0;
      for (int l = j; l < b; l++)
        if (g.block[g.col[l]] == bj) sum += g.cw[l];
      if (bj == own) { ownw = sum; continue; }
      if (sum > bestw || (sum == bestw && bj < best)) { bestw = sum; best = bj; }
    }
    if (best >= 0 && bestw > ownw) t = best;
  }
  target[v] = t;
  tkey[v] = t >= 0 ? t : ML_NONE;
  skey[v] = t >= 0 ? g.block[v] : ML_NONE;
  idx[v] = (int)v;
}

// Acceptance within one group (one CTA per block b): the candidates of b,
// sorted by vertex, are accepted while the running total of their weights
// (every earlier candidate counted, accepted or not) stays within room[b].
__global__ void __launch_bounds__(256) k_ml_accept(const uint32_t* keys, const int* vals, int64_t n,
                                                   const int* vw, const long long* W, long long lbound, int in_side,
                                                   unsigned char* ok) {
  __shared__ long long s_scan[256];
  __shared__ int s_lo, s_hi;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) {
    // [s_lo, s_hi): the positions whose key is b (keys sorted ascending)
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if ((int)keys[mid] < b) lo = mid + 1; else hi = mid; }
    int64_t lo2 = lo, hi2 = n;
    while (lo2 < hi2) { int64_t mid = (lo2 + hi2) >> 1; if ((int)keys[mid] <= b) lo2 = mid + 1; else hi2 = mid; }
    s_lo = (int)lo;
    s_hi = (int)lo2;
  }
  __syncthreads();
  // room: lmax - W_b on the target side, W_b - lmin on the source side
  const long long room = in_side ? lbound - W[b] : W[b] - lbound;
  long long base = 0;
  for (int p0 = s_lo; p0 < s_hi; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    const long long w = p < s_hi ? (long long)vw[vals[p]] : 0;
    s_scan[threadIdx.x] = w;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const long long x = threadIdx.x >= (unsigned)off ? s_scan[threadIdx.x - off] : 0;
      __syncthreads();
      s_scan[threadIdx.x] += x;
      __syncthreads();
    }
    if (p < s_hi) ok[vals[p]] = (base + s_scan[threadIdx.x] <= room) ? 1 : 0;
    const long long tot = s_scan[blockDim.x - 1];
    __syncthreads();
    base += tot;
  }
}

__global__ void k_ml_apply(MLGraph g, const int* target, const unsigned char* ok_in, const unsigned char* ok_out) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < g.n && target[v] >= 0 && ok_in[v] && ok_out[v]) g.block[v] = target[v];
}

__global__ void k_ml_project(int64_t n, const int* cmap, const int* cblock, int* block) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) block[v] = cblock[cmap[v]];
}

inline unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, ceil_div<int64_t>(n, 256)); }

int bits_for(unsigned long long x) {
  int b = 1;
  while (b < 64 && (x >> b) != 0) b++;
  return b;
}

// Heavy-edge matching of level g (ML_SWEEPS handshake sweeps).
int ml_match(dt_ctx* c, const MLGraph& g, int cmax, int* mate, int* pref) {
  cudaStream_t s = c->stream;
  const unsigned gr = grid_of(g.n);
  k_ml_fill<<<gr, 256, (++c->launches, 0), s>>>(mate, g.n, -1);
  for (int sw = 0; sw < ML_SWEEPS; sw++) {
    k_ml_pref<<<gr, 256, (++c->launches, 0), s>>>(g, mate, cmax, pref);
    k_ml_mutual<<<gr, 256, (++c->launches, 0), s>>>(g.n, pref, mate);
  }
  return 0;
}

// The coarse graph of level g's matching; fills g.cmap and the coarse level
// (its buffers from the pool under `tag`); *nc_out = its vertex count.
int ml_contract(dt_ctx* c, MLGraph& g, const int* mate, const std::string& tag, MLGraph& cg) {
  cudaStream_t s = c->stream;
  const unsigned gr = grid_of(g.n);
  int* isrep = (int*)pool_get(c, tag + ".isrep", 4 * (size_t)g.n);
  int* cid = (int*)pool_get(c, tag + ".cid", 4 * (size_t)g.n);
  if (!isrep || !cid) return set_err(c, DT_E_NOMEM, "multilevel contraction");
  k_ml_isrep<<<gr, 256, (++c->launches, 0), s>>>(g.n, mate, isrep);
  int nc = 0;
  int rc = exclusive_scan_i32(c, isrep, cid, g.n, &nc);
  if (rc) return rc;
  cg.n = nc;
  cg.vw = (int*)pool_get(c, tag + ".cvw", 4 * (size_t)std::max(nc, 1));
  cg.block = (int*)pool_get(c, tag + ".cblock", 4 * (size_t)std::max(nc, 1));
  cg.rowptr = (int*)pool_get(c, tag + ".crow", 4 * (size_t)(nc + 1));
  if (!cg.vw || !cg.block || !cg.rowptr) return set_err(c, DT_E_NOMEM, "multilevel coarse graph");
  k_ml_cmap<<<gr, 256, (++c->launches, 0), s>>>(g, mate, cid, cg.vw, cg.block);
  // coarse edges: sort the directed fine edges by (coarse row, coarse column)
  const int64_t m = g.nnz;
  const unsigned long long ncu = (unsigned long long)nc;
  unsigned long long* keys = (unsigned long long*)pool_get(c, tag + ".ekeys", 8 * (size_t)std::max<int64_t>(m, 1));
  int* vals = (int*)pool_get(c, tag + ".evals", 4 * (size_t)std::max<int64_t>(m, 1));
  int* flag = (int*)pool_get(c, tag + ".eflag", 4 * (size_t)std::max<int64_t>(m, 1));
  int* uid = (int*)pool_get(c, tag + ".euid", 4 * (size_t)std::max<int64_t>(m, 1));
  int* crowcnt = (int*)pool_get(c, tag + ".crowcnt", 4 * (size_t)(nc + 1));
  if (!keys || !vals || !flag || !uid || !crowcnt) return set_err(c, DT_E_NOMEM, "multilevel coarse edges");
  int nnzc = 0;
  if (m > 0) {
    k_ml_edge_keys<<<gr, 256, (++c->launches, 0), s>>>(g, ncu, keys, vals);
    rc = radix_sort_pairs<unsigned long long, int>(c, keys, vals, m, bits_for(ncu * ncu), tag + ".esort");
    if (rc) return rc;
    k_ml_uflag<<<grid_of(m), 256, (++c->launches, 0), s>>>(m, keys, ncu * ncu, flag);
    rc = exclusive_scan_i32(c, flag, uid, m, &nnzc);
    if (rc) return rc;
  }
  cg.nnz = nnzc;
  cg.col = (int*)pool_get(c, tag + ".ccol", 4 * (size_t)std::max(nnzc, 1));
  cg.cw = (long long*)pool_get(c, tag + ".ccw", 8 * (size_t)std::max(nnzc, 1));
  if (!cg.col || !cg.cw) return set_err(c, DT_E_NOMEM, "multilevel coarse edges");
  CUDA_OK(cudaMemsetAsync(cg.cw, 0, 8 * (size_t)std::max(nnzc, 1), s));
  CUDA_OK(cudaMemsetAsync(crowcnt, 0, 4 * (size_t)(nc + 1), s));
  if (m > 0)
    k_ml_cedges<<<grid_of(m), 256, (++c->launches, 0), s>>>(m, keys, vals, g.cw, flag, uid, ncu, cg.col, cg.cw,
                                                           crowcnt);
  rc = exclusive_scan_i32(c, crowcnt, cg.rowptr, nc + 1, nullptr);
  if (rc) return rc;
  return 0;
}

// `rounds` rounds of label propagation with vertex weights on level g.
int ml_lp(dt_ctx* c, MLGraph& g, int k, int lmin, int lmax, int rounds, const std::string& tag) {
  cudaStream_t s = c->stream;
  const int64_t n = g.n;
  const unsigned gr = grid_of(n);
  int* target = (int*)pool_get(c, tag + ".target", 4 * (size_t)n);
  uint32_t* tkey = (uint32_t*)pool_get(c, tag + ".tkey", 4 * (size_t)n);
  uint32_t* skey = (uint32_t*)pool_get(c, tag + ".skey", 4 * (size_t)n);
  int* tidx = (int*)pool_get(c, tag + ".tidx", 4 * (size_t)n);
  int* sidx = (int*)pool_get(c, tag + ".sidx", 4 * (size_t)n);
  unsigned char* ok_in = (unsigned char*)pool_get(c, tag + ".okin", (size_t)n);
  unsigned char* ok_out = (unsigned char*)pool_get(c, tag + ".okout", (size_t)n);
  long long* W = (long long*)pool_get(c, tag + ".W", 8 * 256);
  if (!target || !tkey || !skey || !tidx || !sidx || !ok_in || !ok_out || !W)
    return set_err(c, DT_E_NOMEM, "multilevel refinement");
  for (int r = 0; r < rounds; r++) {
    CUDA_OK(cudaMemsetAsync(W, 0, 8 * 256, s));
    k_ml_block_weights<<<gr, 256, (++c->launches, 0), s>>>(g, W);
    k_ml_propose<<<gr, 256, (++c->launches, 0), s>>>(g, r & 1, target, (int*)tkey, (int*)skey, tidx);
    CUDA_OK(cudaMemcpyAsync(sidx, tidx, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    // stable sorts by target and by source block keep the vertex order inside each group
    int rc = radix_sort_pairs<uint32_t, int>(c, tkey, tidx, n, 9, tag + ".st");
    if (rc) return rc;
    rc = radix_sort_pairs<uint32_t, int>(c, skey, sidx, n, 9, tag + ".ss");
    if (rc) return rc;
    CUDA_OK(cudaMemsetAsync(ok_in, 0, (size_t)n, s));
    CUDA_OK(cudaMemsetAsync(ok_out, 0, (size_t)n, s));
    k_ml_accept<<<k, 256, (++c->launches, 0), s>>>(tkey, tidx, n, g.vw, W, lmax, 1, ok_in);
    k_ml_accept<<<k, 256, (++c->launches, 0), s>>>(skey, sidx, n, g.vw, W, lmin, 0, ok_out);
    k_ml_apply<<<gr, 256, (++c->launches, 0), s>>>(g, target, ok_in, ok_out);
  }
  return 0;
}

}  // namespace

// Multilevel refinement of `block` (eta labels, in place) on the sample
// graph G; see the file comment.  k <= 256.
int partition_multilevel(dt_ctx* c, const SampleGraph& G, int k, double eps, int rounds, int* block) {
  cudaStream_t s = c->stream;
  const int64_t eta = G.eta;
  int lmin, lmax;
  partition_bounds(eta, k, eps, &lmin, &lmax);
  const int cmax = std::max(2, lmax / 4);
  std::vector<MLGraph> lv;
  MLGraph g0;
  g0.n = eta;
  g0.nnz = 2 * G.m;
  g0.rowptr = G.rowptr;
  g0.col = G.col;
  g0.cw = G.cw;
  g0.vw = (int*)pool_get(c, "ml.vw0", 4 * (size_t)std::max<int64_t>(eta, 1));
  g0.block = block;
  if (!g0.vw) return set_err(c, DT_E_NOMEM, "multilevel partition");
  k_ml_fill<<<grid_of(eta), 256, (++c->launches, 0), s>>>(g0.vw, eta, 1);
  lv.push_back(g0);
  while ((int)lv.size() < ML_MAX_LEVELS) {
    MLGraph& g = lv.back();
    const std::string tag = "ml.L" + std::to_string(lv.size());
    int* mate = (int*)pool_get(c, tag + ".mate", 4 * (size_t)std::max<int64_t>(g.n, 1));
    int* pref = (int*)pool_get(c, tag + ".pref", 4 * (size_t)std::max<int64_t>(g.n, 1));
    g.cmap = (int*)pool_get(c, tag + ".cmap", 4 * (size_t)std::max<int64_t>(g.n, 1));
    if (!mate || !pref || !g.cmap) return set_err(c, DT_E_NOMEM, "multilevel matching");
    int rc = ml_match(c, g, cmax, mate, pref);
    if (rc) return rc;
    MLGraph cg;
    rc = ml_contract(c, g, mate, tag, cg);
    if (rc) return rc;
    // a level that keeps more than 95 % of its vertices ends the coarsening
    if ((double)cg.n > 0.95 * (double)g.n) break;
    lv.push_back(cg);
  }
  // rounds on the sample graph, half as many (at least one) on every coarse level
  for (int l = (int)lv.size() - 1; l >= 0; l--) {
    int rc = ml_lp(c, lv[l], k, lmin, lmax, l == 0 ? rounds : std::max(1, rounds / 2), "ml.lp" + std::to_string(l));
    if (rc) return rc;
    if (l > 0)
      k_ml_project<<<grid_of(lv[l - 1].n), 256, (++c->launches, 0), s>>>(lv[l - 1].n, lv[l - 1].cmap, lv[l].block,
                                                                        lv[l - 1].block);
  }
  return 0;
}

}  // namespace gdt
