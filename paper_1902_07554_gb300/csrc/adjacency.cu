// adjacency.cu -- the neighbourhood update that ends the merge of Alg. 1,
// and a certificate that a triangulation is DT(P).
//
// Neighbourhood update (Alg. 1, merging): every output simplex keeps the
// links it had in the triangulation it came from (a partial T_i or T_B) as
// long as the neighbour is itself in the output.  A facet whose neighbour
// was stripped (a border simplex), was not kept (a T_B simplex inside one
// partition that replaced nothing), or was a ghost (the hull of T_i or of
// T_B) is "open": it goes into a lock-free hash of facet keys (sorted
// global-index d-tuples), and the two open entries with equal keys are
// linked.  An open facet without partner is on the hull of P.  Two output
// simplices that share a facet but do not link directly are both open on
// it: if one of them linked to a neighbour in its source, that neighbour
// would be a third output simplex on the facet.
//
// Certificate (the Delaunay lemma, Sec. 2.1): a set of d-simplices on P is
// DT(P) when every simplex is non-flat, every facet lies in at most two
// simplices, the two simplices on an interior facet lie on opposite sides
// of it and each one's apex is outside the other's (perturbed)
// circumsphere, the boundary is locally convex at every hull ridge, every
// point is a vertex, and the Euler characteristic is 1 (one component).
#include "adjacency.cuh"
#include "predicates.cuh"

namespace gdt {

constexpr int kPivotLimit = 4096;

__device__ __forceinline__ unsigned long long facet_hash(const int* f, int d) {
  unsigned long long h = 0x2545F4914F6CDD1Dull;
  for (int i = 0; i < d; i++) h = splitmix64(h ^ (unsigned)f[i]);
  return h;
}

// The facet of row (v >> 2) opposite its vertex (v & 3), ascending.
template <int D>
__device__ __forceinline__ void facet_of(const int32_t* rows, int v, int* f) {
  const int32_t* r = rows + (int64_t)(v >> 2) * (D + 1);
  int j = v & 3, k = 0;
#pragma unroll
  for (int i = 0; i <= D; i++)
    if (i != j) f[k++] = r[i];
}

__device__ __forceinline__ void warp_append(bool take, int value, int* list, int* count) {
  unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  int lane = threadIdx.x & 31, leader = __ffs(mask) - 1, base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) list[base + __popc(mask & ((1u << lane) - 1))] = value;
}

__global__ void k_slot_row(const int* origin, int64_t m, int* slot_row) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < m) slot_row[origin[r]] = (int)r;
}

// Links that survive the merge; the other facets are appended to `open`.
template <int D>
__global__ void k_link_direct(const int32_t* rows, int64_t m, LinkSources S, const int* slot_row, int32_t* nbr,
                              int* open, int* nopen) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = r < m;
  int o = live ? S.origin[r] : 0;
  const bool second = o >= S.base1;
  const int slot = second ? (int)(o - S.base1) : o;
  const int4* tv = second ? S.tv1 : S.tv0;
  const int4* tn = second ? S.tn1 : S.tn0;
  const int* gid = second ? S.gid1 : S.gid0;
  const int64_t base = second ? S.base1 : 0;
  int4 v = make_int4(0, 0, 0, 0), nb = make_int4(-1, -1, -1, -1);
  if (live) { v = tv[slot]; nb = tn[slot]; }
  const int vv[4] = {v.x, v.y, v.z, v.w}, pp[4] = {nb.x, nb.y, nb.z, nb.w};
  const int32_t* row = rows + (live ? r : 0) * (D + 1);
#pragma unroll
  for (int i = 0; i <= D; i++) {
    bool is_open = false;
    int j = 0;
    if (live) {
      const int g = gid[vv[i]];
#pragma unroll
      for (int q = 0; q <= D; q++)
        if (row[q] == g) j = q;
      int link = -1;
      if (pp[i] >= 0) link = slot_row[base + (pp[i] >> 2)];   // ghosts and dropped simplices: -1
      nbr[r * (D + 1) + j] = link;
      is_open = link < 0;
    }
    warp_append(is_open, (int)((live ? r : 0) << 2) | j, open, nopen);
  }
}

// Every facet of every row is open (rows without provenance).
template <int D>
__global__ void k_all_open(int64_t m, int* open) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
#pragma unroll
  for (int j = 0; j <= D; j++) open[r * (D + 1) + j] = (int)(r << 2) | j;
}

template <int D>
__global__ void k_open_insert(const int32_t* rows, const int* open, int64_t nopen, int* table, unsigned mask,
                              int* fail) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nopen) return;
  const int v = open[i];
  int f[D];
  facet_of<D>(rows, v, f);
  unsigned slot = (unsigned)facet_hash(f, D) & mask;
  for (unsigned probe = 0; probe <= mask; probe++) {
    if (atomicCAS(&table[slot], -1, v) == -1) return;
    slot = (slot + 1) & mask;
  }
  atomicExch(fail, 1);
}

// Partner of each open facet: the other entry with the same key.
template <int D>
__global__ void k_open_match(const int32_t* rows, const int* open, int64_t nopen, const int* table, unsigned mask,
                             int32_t* nbr, unsigned long long* cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nopen) return;
  const int v = open[i];
  int f[D], g[D];
  facet_of<D>(rows, v, f);
  unsigned slot = (unsigned)facet_hash(f, D) & mask;
  int partner = -1, more = 0;
  for (unsigned probe = 0; probe <= mask; probe++) {
    const int w = table[slot];
    if (w < 0) break;
    if (w != v) {
      facet_of<D>(rows, w, g);
      bool eq = true;
#pragma unroll
      for (int q = 0; q < D; q++) eq &= f[q] == g[q];
      if (eq) {
        if (partner < 0) partner = w; else more = 1;
      }
    }
    slot = (slot + 1) & mask;
  }
  nbr[(int64_t)(v >> 2) * (D + 1) + (v & 3)] = partner < 0 ? -1 : partner >> 2;
  if (more) atomicAdd(&cnt[0], 1ull);
  if (partner < 0) atomicAdd(&cnt[2], 1ull);
}

// cnt: [0] facets with more than one partner, [1] table full, [2] facets without partner.
static int match_open(dt_ctx* c, int dim, const int32_t* rows, const int* open, int64_t nopen, int32_t* nbr,
                      int64_t* non_manifold, int64_t* unmatched) {
  cudaStream_t s = c->stream;
  unsigned tsize = 64;
  while (tsize < 2 * nopen + 2) tsize <<= 1;
  int* table = (int*)pool_get(c, "adj.table", 4 * (size_t)tsize);
  unsigned long long* cnt = (unsigned long long*)pool_get(c, "adj.cnt", 24);
  if (!table || !cnt) return set_err(c, DT_E_NOMEM, "facet hash");
  CUDA_OK(cudaMemsetAsync(table, 0xff, 4 * (size_t)tsize, s));
  CUDA_OK(cudaMemsetAsync(cnt, 0, 24, s));
  if (nopen) {
    unsigned g = (unsigned)ceil_div<int64_t>(nopen, 256);
    int* fail = (int*)(cnt + 1);
    if (dim == 2) {
      k_open_insert<2><<<g, 256, (++c->launches, 0), s>>>(rows, open, nopen, table, tsize - 1, fail);
      k_open_match<2><<<g, 256, (++c->launches, 0), s>>>(rows, open, nopen, table, tsize - 1, nbr, cnt);
    } else {
      k_open_insert<3><<<g, 256, (++c->launches, 0), s>>>(rows, open, nopen, table, tsize - 1, fail);
      k_open_match<3><<<g, 256, (++c->launches, 0), s>>>(rows, open, nopen, table, tsize - 1, nbr, cnt);
    }
  }
  unsigned long long h[3];
  CUDA_OK(cudaMemcpyAsync(h, cnt, 24, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (h[1]) return set_err(c, DT_E_OVERFLOW, "facet hash table full");
  *non_manifold = (int64_t)h[0];
  if (unmatched) *unmatched = (int64_t)h[2];
  return 0;
}

int neighbor_update(dt_ctx* c, int dim, const int32_t* rows, int64_t m, const LinkSources& src, int32_t** nbr_out) {
  cudaStream_t s = c->stream;
  if (m >= (int64_t)1 << 29) return set_err(c, DT_E_OVERFLOW, "too many simplices for packed facet ids");
  const int64_t nf = (int64_t)(dim + 1) * std::max<int64_t>(m, 1);
  int32_t* nbr = (int32_t*)pool_get(c, "adj.nbr", 4 * nf);
  int* open = (int*)pool_get(c, "adj.open", 4 * nf);
  int* slot_row = (int*)pool_get(c, "adj.slot_row", 4 * (size_t)std::max<int64_t>(src.total, 1));
  int* nopen_d = (int*)pool_get(c, "adj.nopen", 16);
  if (!nbr || !open || !slot_row || !nopen_d) return set_err(c, DT_E_NOMEM, "neighbour buffers");
  *nbr_out = nbr;
  if (m == 0) return 0;
  CUDA_OK(cudaMemsetAsync(slot_row, 0xff, 4 * (size_t)src.total, s));
  CUDA_OK(cudaMemsetAsync(nopen_d, 0, 4, s));
  unsigned g = (unsigned)ceil_div<int64_t>(m, 256);
  k_slot_row<<<g, 256, (++c->launches, 0), s>>>(src.origin, m, slot_row);
  if (dim == 2) k_link_direct<2><<<g, 256, (++c->launches, 0), s>>>(rows, m, src, slot_row, nbr, open, nopen_d);
  else k_link_direct<3><<<g, 256, (++c->launches, 0), s>>>(rows, m, src, slot_row, nbr, open, nopen_d);
  int nopen = 0;
  CUDA_OK(cudaMemcpyAsync(&nopen, nopen_d, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  int64_t extra = 0, hull = 0;
  int rc = match_open(c, dim, rows, open, nopen, nbr, &extra, &hull);
  if (rc) return rc;
  c->stats.hull_facets = hull;
  if (extra) return set_err(c, DT_E_INTERNAL, "a facet of the merged triangulation lies in more than two simplices");
  return 0;
}

int match_all_facets(dt_ctx* c, int dim, const int32_t* rows, int64_t m, int32_t** nbr_out, int64_t* non_manifold) {
  if (m >= (int64_t)1 << 29) return set_err(c, DT_E_OVERFLOW, "too many simplices for packed facet ids");
  const int64_t nf = (int64_t)(dim + 1) * std::max<int64_t>(m, 1);
  int32_t* nbr = (int32_t*)pool_get(c, "adj.nbr", 4 * nf);
  int* open = (int*)pool_get(c, "adj.open", 4 * nf);
  if (!nbr || !open) return set_err(c, DT_E_NOMEM, "neighbour buffers");
  *nbr_out = nbr;
  *non_manifold = 0;
  if (m == 0) return 0;
  unsigned g = (unsigned)ceil_div<int64_t>(m, 256);
  if (dim == 2) k_all_open<2><<<g, 256, (++c->launches, 0), c->stream>>>(m, open);
  else k_all_open<3><<<g, 256, (++c->launches, 0), c->stream>>>(m, open);
  return match_open(c, dim, rows, open, (dim + 1) * m, nbr, non_manifold, nullptr);
}

// ---------------------------------------------------------------- certificate
enum { V_INTERIOR, V_HULL, V_FLAT, V_FOLDED, V_NONDEL, V_NONCONVEX, V_PIVOT, V_ASYM, V_UNUSED, V_EDGES, V_FAIL, V_N };

template <int D>
__global__ void k_prepare_rows(const int32_t* in, int64_t m, int64_t n, int32_t* out, unsigned long long* bad) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  int v[D + 1];
  bool ok = true;
#pragma unroll
  for (int i = 0; i <= D; i++) {
    v[i] = in[r * (D + 1) + i];
    ok &= v[i] >= 0 && v[i] < n;
  }
  for (int a = 1; a <= D; a++)
    for (int b = a; b > 0 && v[b] < v[b - 1]; b--) { int t = v[b]; v[b] = v[b - 1]; v[b - 1] = t; }
  for (int a = 1; a <= D; a++) ok &= v[a] != v[a - 1];
  if (!ok) {   // a placeholder of negative ids: skipped by the checks, shares no facet with any row
    atomicAdd(bad, 1ull);
    for (int i = 0; i <= D; i++) v[i] = -1 - (int)((r & 0x1fffffff) * 4 + i);
  }
#pragma unroll
  for (int i = 0; i <= D; i++) out[r * (D + 1) + i] = v[i];
}

// Walks around the hull ridge e = facet minus `other` from row r (apex p
// opposite the hull facet) to the next hull facet; returns its vertex off
// the ridge, or -1 when the walk fails or hits the step limit.
template <int D>
__device__ int hull_pivot(const int32_t* rows, const int32_t* nbr, int64_t m, int r, int p, int other,
                          const int* e, unsigned long long* cnt) {
  int cur = r, ain = other, aout = p;
  for (int step = 0; step < kPivotLimit; step++) {
    const int32_t* rc = rows + (int64_t)cur * (D + 1);
    int pin = -1;
#pragma unroll
    for (int q = 0; q <= D; q++)
      if (rc[q] == ain) pin = q;
    if (pin < 0) { atomicAdd(&cnt[V_ASYM], 1ull); return -1; }
    const int t = nbr[(int64_t)cur * (D + 1) + pin];
    if (t < 0) return aout;
    if (t >= m) { atomicAdd(&cnt[V_ASYM], 1ull); return -1; }
    const int32_t* rt = rows + (int64_t)t * (D + 1);
    int z = -1, nz = 0;
#pragma unroll
    for (int q = 0; q <= D; q++) {
      const int u = rt[q];
      bool on = u == aout;
#pragma unroll
      for (int k = 0; k < D - 1; k++) on |= u == e[k];
      if (!on) { z = u; nz++; }
    }
    if (nz != 1) { atomicAdd(&cnt[V_ASYM], 1ull); return -1; }
    cur = t;
    ain = aout;
    aout = z;
  }
  atomicAdd(&cnt[V_PIVOT], 1ull);
  return -1;
}

template <int D, typename PT>
__global__ void __launch_bounds__(128) k_validate(const PT* P, const int* ident, const int32_t* rows,
                                                  const int32_t* nbr, int64_t m, unsigned long long* cnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int32_t* row = rows + r * (D + 1);
  if (row[0] < 0) return;   // rejected by prepare_rows
  int v[4] = {row[0], row[1], row[2], D == 3 ? row[3] : 0};
  const int o = orient_p(P, v);
  if (o == 0) { atomicAdd(&cnt[V_FLAT], 1ull); return; }
  int w[4] = {v[0], v[1], v[2], v[3]};
  if (o < 0) { w[0] = v[1]; w[1] = v[0]; }           // positively oriented copy
  unsigned long long interior = 0, hull = 0;
  for (int j = 0; j <= D; j++) {
    const int wi = (o < 0 && j < 2) ? 1 - j : j;      // position of v[j] in w
    const int t = nbr[r * (D + 1) + j];
    if (t < 0) {
      hull++;
      // local convexity at each ridge of this hull facet
      int f[D], k = 0;
      for (int q = 0; q <= D; q++)
        if (q != j) f[k++] = v[q];
      for (int a = 0; a < D; a++) {
        int e[3], ke = 0;
        for (int q = 0; q < D; q++)
          if (q != a) e[ke++] = f[q];
        const int far = hull_pivot<D>(rows, nbr, m, (int)r, v[j], f[a], e, cnt);
        if (far < 0 || far == v[j]) continue;
        int y[4] = {w[0], w[1], w[2], w[3]};
        y[wi] = far;
        if (orient_p(P, y) < 0) atomicAdd(&cnt[V_NONCONVEX], 1ull);
      }
      continue;
    }
    interior++;
    if (t >= m) { atomicAdd(&cnt[V_ASYM], 1ull); continue; }
    const int32_t* rt = rows + (int64_t)t * (D + 1);
    int x = -1, xpos = -1, shared = 0;
    for (int i = 0; i <= D; i++) {
      const int u = rt[i];
      bool in = false;
      for (int q = 0; q <= D; q++)
        if (q != j && v[q] == u) in = true;
      if (in) shared++; else { x = u; xpos = i; }
    }
    if (shared != D || x < 0 || nbr[(int64_t)t * (D + 1) + xpos] != (int)r) {
      atomicAdd(&cnt[V_ASYM], 1ull);
      continue;
    }
    if (r < t) {
      int z[4] = {w[0], w[1], w[2], w[3]};
      z[wi] = x;
      if (orient_p(P, z) >= 0) atomicAdd(&cnt[V_FOLDED], 1ull);
      else if (insphere_sos(P, ident, w, x, D) > 0) atomicAdd(&cnt[V_NONDEL], 1ull);
    }
  }
  if (interior) atomicAdd(&cnt[V_INTERIOR], interior);
  if (hull) atomicAdd(&cnt[V_HULL], hull);
}

__global__ void k_mark_used(const int32_t* rows, int64_t nidx, int64_t n, unsigned char* used) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nidx) return;
  const int v = rows[i];
  if (v >= 0 && v < n) used[v] = 1;
}

__global__ void k_count_unused(const unsigned char* used, int64_t n, unsigned long long* cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool un = i < n && !used[i];
  unsigned mask = __ballot_sync(0xffffffffu, un);
  if ((threadIdx.x & 31) == 0 && mask) atomicAdd(cnt, (unsigned long long)__popc(mask));
}

// Distinct edges of 3D rows (a hash set of vertex pairs).
__global__ void k_edges3(const int32_t* rows, int64_t m, unsigned long long* table, unsigned long long mask,
                         unsigned long long* cnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int32_t* row = rows + r * 4;
  if (row[0] < 0) return;
  unsigned long long added = 0;
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      const unsigned long long key = ((unsigned long long)(unsigned)row[a] << 32) | (unsigned)row[b];
      unsigned long long slot = splitmix64(key) & mask;
      bool done = false;
      for (unsigned long long probe = 0; probe <= mask && !done; probe++) {
        const unsigned long long old = atomicCAS(&table[slot], ~0ull, key);
        if (old == ~0ull) { added++; done = true; }
        else if (old == key) done = true;
        else slot = (slot + 1) & mask;
      }
      if (!done) atomicAdd(&cnt[V_FAIL], 1ull);
    }
  if (added) atomicAdd(&cnt[V_EDGES], added);
}

__global__ void k_iota_ident(int* a, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int)i;
}

int prepare_rows(dt_ctx* c, int dim, const int32_t* in, int64_t m, int64_t n, int32_t* out, int64_t* bad) {
  cudaStream_t s = c->stream;
  unsigned long long* b = (unsigned long long*)pool_get(c, "val.bad", 8);
  if (!b) return set_err(c, DT_E_NOMEM, "validation buffers");
  CUDA_OK(cudaMemsetAsync(b, 0, 8, s));
  if (m) {
    unsigned g = (unsigned)ceil_div<int64_t>(m, 256);
    if (dim == 2) k_prepare_rows<2><<<g, 256, (++c->launches, 0), s>>>(in, m, n, out, b);
    else k_prepare_rows<3><<<g, 256, (++c->launches, 0), s>>>(in, m, n, out, b);
  }
  unsigned long long h = 0;
  CUDA_OK(cudaMemcpyAsync(&h, b, 8, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  *bad = (int64_t)h;
  return 0;
}

// The exact fallback's range-error counter of this translation unit (never reset).
static __global__ void k_adj_range(int* out) { *out = g_range_error; }

static int read_range(dt_ctx* c, int* out) {
  int* d = (int*)pool_get(c, "val.range", 16);
  if (!d) return set_err(c, DT_E_NOMEM, "range counter");
  k_adj_range<<<1, 1, (++c->launches, 0), c->stream>>>(d);
  CUDA_OK(cudaMemcpyAsync(out, d, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  return 0;
}

int validate_rows(dt_ctx* c, int dim, const void* P, int64_t n, const int32_t* rows, int64_t m, const int32_t* nbr,
                  int64_t non_manifold, dt_validation* out) {
  cudaStream_t s = c->stream;
  int range0 = 0, range1 = 0;
  int rc = read_range(c, &range0);
  if (rc) return rc;
  unsigned long long* cnt = (unsigned long long*)pool_get(c, "val.cnt", 8 * V_N);
  int* ident = (int*)pool_get(c, "val.ident", 4 * (size_t)std::max<int64_t>(n, 1));
  unsigned char* used = (unsigned char*)pool_get(c, "val.used", (size_t)std::max<int64_t>(n, 1));
  if (!cnt || !ident || !used) return set_err(c, DT_E_NOMEM, "validation buffers");
  CUDA_OK(cudaMemsetAsync(cnt, 0, 8 * V_N, s));
  CUDA_OK(cudaMemsetAsync(used, 0, (size_t)n, s));
  k_iota_ident<<<(unsigned)ceil_div<int64_t>(std::max<int64_t>(n, 1), 256), 256, (++c->launches, 0), s>>>(ident, n);
  if (m) {
    unsigned g = (unsigned)ceil_div<int64_t>(m, 128);
    if (dim == 2)
      k_validate<2><<<g, 128, (++c->launches, 0), s>>>((const double2*)P, ident, rows, nbr, m, cnt);
    else
      k_validate<3><<<g, 128, (++c->launches, 0), s>>>((const double4_32a*)P, ident, rows, nbr, m, cnt);
    const int64_t nidx = (dim + 1) * m;
    k_mark_used<<<(unsigned)ceil_div<int64_t>(nidx, 256), 256, (++c->launches, 0), s>>>(rows, nidx, n, used);
  }
  k_count_unused<<<(unsigned)ceil_div<int64_t>(std::max<int64_t>(n, 1), 256), 256, (++c->launches, 0), s>>>(
      used, n, cnt + V_UNUSED);
  if (dim == 3 && m) {
    unsigned long long tsize = 64;
    while (tsize < 4 * (unsigned long long)m + 2) tsize <<= 1;   // about 1.15 m edges
    unsigned long long* table = (unsigned long long*)pool_get(c, "val.edges", 8 * tsize);
    if (!table) return set_err(c, DT_E_NOMEM, "edge table");
    CUDA_OK(cudaMemsetAsync(table, 0xff, 8 * tsize, s));
    k_edges3<<<(unsigned)ceil_div<int64_t>(m, 256), 256, (++c->launches, 0), s>>>(rows, m, table, tsize - 1, cnt);
  }
  unsigned long long h[V_N];
  CUDA_OK(cudaMemcpyAsync(h, cnt, 8 * V_N, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (h[V_FAIL]) return set_err(c, DT_E_OVERFLOW, "edge table full");
  rc = read_range(c, &range1);
  if (rc) return rc;
  if (range1 != range0) return set_err(c, DT_E_RANGE, "coordinate range too wide for the exact fallback");
  dt_validation v;
  memset(&v, 0, sizeof(v));
  v.simplices = m;
  v.interior_facets = (int64_t)h[V_INTERIOR] / 2;
  v.hull_facets = (int64_t)h[V_HULL];
  v.flat = (int64_t)h[V_FLAT];
  v.non_manifold = non_manifold;
  v.asymmetric = (int64_t)h[V_ASYM];
  v.folded = (int64_t)h[V_FOLDED];
  v.non_delaunay = (int64_t)h[V_NONDEL];
  v.non_convex = (int64_t)h[V_NONCONVEX];
  v.unused_points = (int64_t)h[V_UNUSED];
  v.pivot_limit = (int64_t)h[V_PIVOT];
  const int64_t V = n - v.unused_points;
  const int64_t F = ((dim + 1) * m + v.hull_facets) / 2;   // facets (each interior one counted twice above)
  if (dim == 2) {
    v.edges = F;
    v.euler = V - F + m;
  } else {
    v.edges = (int64_t)h[V_EDGES];
    v.euler = V - v.edges + F - m;
  }
  v.violations = v.bad_index + v.flat + v.non_manifold + v.asymmetric + v.folded + v.non_delaunay + v.non_convex +
                 v.unused_points + v.pivot_limit + (v.euler != 1 ? 1 : 0);
  *out = v;
  return 0;
}

}  // namespace gdt
