// recursive.cu -- recursive bisection (Sec. 3.1, "Recursive Bisection &
// Direct k-way Partitioning"): the divide is applied log2 k times with
// k' = 2 -- every node draws a fresh sample of its own points, triangulates
// and bisects it and assigns its points (Alg. 2), or splits at the median of
// the cyclic dimension (the kd comparator, whose labels already are a
// recursive bisection) -- and the k leaves are merged pairwise, level by
// level: k - 1 merges and k - 1 border triangulations.
//
// Every merge level is batched over its nodes: one border-detection launch
// over all parts (each part tested against the points of its sibling only),
// one insertion-engine run over all the level's border vertex sets (one
// instance per node), one hash merge.  Above the leaves a part's
// triangulation is a set of rows; it becomes an arena again for the next
// border test: its finite simplices plus one ghost simplex per hull facet
// (facets found through the facet hash, oriented by the exact orientation of
// their simplex).
#include <cmath>

#include "adjacency.cuh"
#include "border.cuh"
#include "divide.cuh"
#include "merge.cuh"
#include "pipeline.cuh"
#include "predicates.cuh"

namespace gdt {

// Child label of a node's points: the first leaf of the side they fall on.
__global__ void k_rb_child_label(const int* side, int64_t m, int first, int half, int* lab) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) lab[i] = first + (side[i] ? half : 0);
}

// Part of each point at a merge level: its leaf with the low `shift` bits dropped.
__global__ void k_rb_part(const int* leaf, int64_t n, int shift, int* part) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) part[i] = leaf[i] >> shift;
}

// out[gid[i]] = val[i]
__global__ void k_rb_by_gid(const int* val, const int* gid, int64_t n, int* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[gid[i]] = val[i];
}

// Border vertex j (a partition-sorted point) belongs to merge node part / 2.
__global__ void k_rb_inst(const int* part, const int* idx, int64_t m, int* inst, int* count) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int v = part[idx[j]] >> 1;
  inst[j] = v;
  atomicAdd(&count[v], 1);
}

// Per part: finite simplices and arena slots (finite + one ghost per hull facet).
template <int D>
__global__ void k_rb_count(const int32_t* rows, const int32_t* nbr, int64_t m, const int* where, const int* part,
                           int* nfin, int* nslot) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int p = part[where[rows[r * (D + 1)]]];
  int h = 0;
  for (int j = 0; j <= D; j++) h += nbr[r * (D + 1) + j] < 0;
  atomicAdd(&nfin[p], 1);
  atomicAdd(&nslot[p], 1 + h);
}

// Writes each row (partition-sorted indices) and its ghosts into its part's
// arena.  The ghost on the hull facet opposite vertex j is the row with the
// infinite vertex in slot j, oriented so that its orientation with a point x
// in slot j is positive exactly when x lies beyond the facet: the row's own
// orientation sigma (exact) has the sign of that determinant at x = v_j,
// which is on the inner side, so a positive sigma swaps two finite entries.
template <int D>
__global__ void k_rb_fill(const typename PT<D>::T* P, const int32_t* rows, const int32_t* nbr, int64_t m,
                          const int* where, const int* part, const int* toff, int* fill, int4* tv) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  int v[4] = {0, 0, 0, 0};
  int h = 0;
  for (int j = 0; j <= D; j++) {
    v[j] = where[rows[r * (D + 1) + j]];
    h += nbr[r * (D + 1) + j] < 0;
  }
  const int p = part[v[0]];
  int slot = toff[p] + atomicAdd(&fill[p], 1 + h);
  tv[slot++] = make_int4(v[0], v[1], v[2], v[3]);
  if (!h) return;
  const int sigma = orient_p(P, v);
  for (int j = 0; j <= D; j++) {
    if (nbr[r * (D + 1) + j] >= 0) continue;
    int g[4] = {v[0], v[1], v[2], v[3]};
    g[j] = INF_V;
    if (sigma > 0) {
      const int a = j == 0 ? 1 : 0, b = j <= 1 ? 2 : 1;
      const int t = g[a]; g[a] = g[b]; g[b] = t;
    }
    tv[slot++] = make_int4(g[0], g[1], g[2], g[3]);
  }
}

// Rows (canonical, global indices) of the parts at one level -> an arena whose
// instances are the parts; a part without finite simplices gets status 1 (its
// points are then border vertices, as for a partition too flat to triangulate).
static int rows_to_arena(dt_ctx* c, int dim, const void* Ps, const int32_t* rows, const int32_t* nbr, int64_t m,
                         const int* where, const int* part, int np, int64_t n, EngineRun& fa) {
  cudaStream_t s = c->stream;
  int* nfin = (int*)pool_get(c, "rb.nfin", 4 * (size_t)np);
  int* nslot = (int*)pool_get(c, "rb.nslot", 4 * (size_t)np);
  int* fill = (int*)pool_get(c, "rb.fill", 4 * (size_t)np);
  int* toff = (int*)pool_get(c, "rb.toff", 4 * (size_t)np);
  int* tcount = (int*)pool_get(c, "rb.tcount", 4 * (size_t)np);
  int* status = (int*)pool_get(c, "rb.status", 4 * (size_t)np);
  if (!nfin || !nslot || !fill || !toff || !tcount || !status) return set_err(c, DT_E_NOMEM, "part arenas");
  CUDA_OK(cudaMemsetAsync(nfin, 0, 4 * (size_t)np, s));
  CUDA_OK(cudaMemsetAsync(nslot, 0, 4 * (size_t)np, s));
  CUDA_OK(cudaMemsetAsync(fill, 0, 4 * (size_t)np, s));
  unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(m, 1), 256);
  if (m) {
    if (dim == 2) k_rb_count<2><<<g, 256, (++c->launches, 0), s>>>(rows, nbr, m, where, part, nfin, nslot);
    else k_rb_count<3><<<g, 256, (++c->launches, 0), s>>>(rows, nbr, m, where, part, nfin, nslot);
  }
  std::vector<int> hf(np), hs(np);
  CUDA_OK(cudaMemcpyAsync(hf.data(), nfin, 4 * (size_t)np, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaMemcpyAsync(hs.data(), nslot, 4 * (size_t)np, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  fa = EngineRun();
  fa.dim = dim;
  fa.ninst = np;
  fa.npts = n;
  fa.h_toff.resize(np);
  fa.h_tcount.resize(np);
  fa.h_status.resize(np);
  int64_t total = 0;
  for (int i = 0; i < np; i++) {
    fa.h_toff[i] = total;
    total += hs[i];
    fa.h_tcount[i] = (int)total;
    fa.h_status[i] = hf[i] ? 0 : 1;
  }
  if (total >= ((int64_t)1 << 31)) return set_err(c, DT_E_OVERFLOW, "part arena too large");
  fa.total_slots = total;
  int4* tv = (int4*)pool_get(c, "rb.tv", 16 * (size_t)std::max<int64_t>(total, 1));
  if (!tv) return set_err(c, DT_E_NOMEM, "part arena");
  std::vector<int> ht(np);
  for (int i = 0; i < np; i++) ht[i] = (int)fa.h_toff[i];
  CUDA_OK(cudaMemcpyAsync(toff, ht.data(), 4 * (size_t)np, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(tcount, fa.h_tcount.data(), 4 * (size_t)np, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(status, fa.h_status.data(), 4 * (size_t)np, cudaMemcpyHostToDevice, s));
  if (m) {
    if (dim == 2)
      k_rb_fill<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)Ps, rows, nbr, m, where, part, toff, fill, tv);
    else
      k_rb_fill<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)Ps, rows, nbr, m, where, part, toff, fill,
                                                      tv);
  }
  CUDA_OK(cudaStreamSynchronize(s));   // host vectors above go out of scope
  fa.tv = tv;
  fa.toff = toff;
  fa.tcount = tcount;
  fa.inst_status = status;
  return 0;
}

int run_recursive(dt_ctx* c, const void* P, int64_t n, int dim, int k, double frac) {
  cudaStream_t s = c->stream;
  const dt_config& cfg = c->cfg;
  if (k & (k - 1)) return set_err(c, DT_E_ARG, "recursive bisection needs k a power of two");
  if (k > 64) return set_err(c, DT_E_ARG, "recursive bisection supports k <= 64");
  int L = 0;
  while ((1 << L) < k) L++;
  const size_t psz = dim == 2 ? 16 : 32;
  auto at = [&](const void* base, int64_t off) { return (const void*)((const char*)base + off * psz); };
  for (int i = 0; i < 7; i++) c->stats.ms_phase[i] = 0;
  auto tick = [&]() { cudaEventRecord(c->ev[12], s); };
  auto tock = [&](int ph) {
    cudaEventRecord(c->ev[13], s);
    cudaEventSynchronize(c->ev[13]);
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[12], c->ev[13]);
    c->stats.ms_phase[ph] += ms;
  };
  c->labels = (int32_t*)pool_get(c, "pl.labels", 4 * n);
  if (!c->labels) return set_err(c, DT_E_NOMEM, "labels");
  c->sample = nullptr;
  c->sample_block = nullptr;
  c->eta = 0;
  int rc;
  unsigned gn = (unsigned)ceil_div<int64_t>(n, 256);
  // ---------------- divide: log2 k bisections
  const void* Ps;
  int *gid, *leaf;
  std::vector<int64_t> poff, sizes;
  int64_t eta_total = 0;
  tick();
  if (cfg.divide == DT_DIVIDE_SAMPLE) {
    void* Pa = pool_get(c, "rb.Pa", psz * n);
    void* Pb = pool_get(c, "rb.Pb", psz * n);
    int* ga = (int*)pool_get(c, "rb.ga", 4 * n);
    int* gb = (int*)pool_get(c, "rb.gb", 4 * n);
    int* la = (int*)pool_get(c, "rb.la", 4 * n);
    int* lb = (int*)pool_get(c, "rb.lb", 4 * n);
    int* side = (int*)pool_get(c, "rb.side", 4 * n);
    int* pos = (int*)pool_get(c, "rb.pos", 4 * n);
    if (!Pa || !Pb || !ga || !gb || !la || !lb || !side || !pos) return set_err(c, DT_E_NOMEM, "bisection buffers");
    CUDA_OK(cudaMemcpyAsync(Pa, P, psz * n, cudaMemcpyDeviceToDevice, s));
    k_iota<<<gn, 256, (++c->launches, 0), s>>>(ga, n, 0);
    CUDA_OK(cudaMemsetAsync(la, 0, 4 * n, s));
    poff.assign(k + 1, n);
    poff[0] = 0;
    for (int depth = 0; depth < L; depth++) {
      const int kk = k >> depth, half = kk / 2;
      for (int first = 0; first < k; first += kk) {
        // the node's points: bucket `first` of the last scatter, ascending global index
        const int64_t off = poff[first], m = poff[first + kk] - poff[first];
        const int64_t eta = sample_size(m, frac, dim);
        if (m < 2 * (dim + 2) || eta < dim + 2) return run_direct(c, P, n, dim);
        int* ids = (int*)pool_get(c, "rb.sid", 4 * eta);
        int* zeros = (int*)pool_get(c, "rb.sz", 4 * eta);
        void* PS = pool_get(c, "rb.PS", psz * eta);
        int* block = (int*)pool_get(c, "rb.blk", 4 * eta);
        if (!ids || !zeros || !PS || !block) return set_err(c, DT_E_NOMEM, "node sample");
        rc = select_sample(c, m, eta, cfg.seed + (uint64_t)depth, ids);
        if (rc) return rc;
        gather_points(c, dim, at(Pa, off), ids, eta, PS);
        CUDA_OK(cudaMemsetAsync(zeros, 0, 4 * eta, s));
        rc = engine_run(c, c->run_sample, dim, PS, ids, zeros, eta, {0, eta}, "sample");
        if (rc) return rc;
        if (c->run_sample.h_status[0] != 0) return run_direct(c, P, n, dim);   // flat node sample
        SampleGraph G;
        rc = sample_graph(c, c->run_sample, PS, dim, cfg.weight, G);
        if (rc) return rc;
        rc = partition_graph(c, PS, dim, G, 2, cfg.epsilon, cfg.lp_rounds, cfg.partition_init, block);
        if (rc) return rc;
        rc = label_points(c, dim, at(Pa, off), m, PS, ids, G, block, side + off, nullptr);
        if (rc) return rc;
        k_rb_child_label<<<(unsigned)ceil_div<int64_t>(m, 256), 256, (++c->launches, 0), s>>>(side + off, m, first,
                                                                                              half, la + off);
        eta_total += eta;
      }
      // stable scatter: every child's points contiguous, in ascending global index
      rc = scatter_by_label(c, dim, Pa, la, n, k, Pb, pos, lb, poff, sizes);
      if (rc) return rc;
      k_gather_i32<<<gn, 256, (++c->launches, 0), s>>>(ga, pos, n, gb);
      std::swap(Pa, Pb);
      std::swap(ga, gb);
      std::swap(la, lb);
    }
    Ps = Pa;
    gid = ga;
    leaf = la;
    k_rb_by_gid<<<gn, 256, (++c->launches, 0), s>>>(leaf, gid, n, c->labels);
  } else {
    rc = kd_divide(c, dim, P, n, k, c->labels);
    if (rc) return rc;
    void* Psk = pool_get(c, "dc.Ps", psz * n);
    gid = (int*)pool_get(c, "dc.gid", 4 * n);
    leaf = (int*)pool_get(c, "dc.pinst", 4 * n);
    if (!Psk || !gid || !leaf) return set_err(c, DT_E_NOMEM, "scatter buffers");
    rc = scatter_by_label(c, dim, P, c->labels, n, k, Psk, gid, leaf, poff, sizes);
    if (rc) return rc;
    Ps = Psk;
  }
  {
    double mu = (double)n / k, ss = 0, mx = -1e300;
    int64_t smax = 0, smin = n;
    for (int i = 0; i < k; i++) {
      ss += (sizes[i] - mu) * (sizes[i] - mu);
      mx = std::max(mx, sizes[i] / mu - 1.0);
      smax = std::max(smax, sizes[i]);
      smin = std::min(smin, sizes[i]);
    }
    c->stats.imbalance = mx;
    c->stats.cv = k > 1 ? std::sqrt(ss / (k - 1)) / mu : 0.0;
    c->stats.partition_size_max = smax;
    c->stats.partition_size_min = smin;
  }
  tock(0);
  // ---------------- leaves: the k partial triangulations in one engine run
  tick();
  rc = engine_run(c, c->run_parts, dim, Ps, gid, leaf, n, poff, "parts");
  if (rc) return rc;
  c->stats.rounds_max = c->run_parts.rounds;
  tock(2);
  // ---------------- log2 k merge levels
  int* where = (int*)pool_get(c, "rb.where", 4 * n);
  int* part = (int*)pool_get(c, "rb.part", 4 * n);
  int* labg = (int*)pool_get(c, "rb.labg", 4 * n);
  int* idxB = (int*)pool_get(c, "rb.idxB", 4 * n);
  unsigned char* fg = (unsigned char*)pool_get(c, "dc.fg", n);
  if (!where || !part || !labg || !idxB || !fg) return set_err(c, DT_E_NOMEM, "merge buffers");
  k_iota<<<gn, 256, (++c->launches, 0), s>>>(idxB, n, 0);
  k_rb_by_gid<<<gn, 256, (++c->launches, 0), s>>>(idxB, gid, n, where);   // where[gid] = sorted position
  CUDA_OK(cudaMemsetAsync(fg, 0, n, s));
  EngineRun fa;
  const EngineRun* arena = &c->run_parts;
  int64_t nVB_total = 0, nB_total = 0, nTB_total = 0;
  for (int h = 1; h <= L; h++) {
    const int np = k >> (h - 1), nm = np / 2;
    k_rb_part<<<gn, 256, (++c->launches, 0), s>>>(leaf, n, h - 1, part);
    std::vector<unsigned long long> om(np);
    for (int i = 0; i < np; i++) om[i] = 1ull << (i ^ 1);   // each part against its sibling
    tick();
    unsigned char *bflag, *vflag;
    int64_t nB = 0, nVB = 0;
    rc = border_detect(c, dim, *arena, Ps, part, np, cfg.grid_cell, cfg.primitive, &bflag, &vflag, &nB, &om);
    if (rc) return rc;
    rc = compact_flags(c, vflag, n, idxB, &nVB, "rb.cvb");
    if (rc) return rc;
    k_flag_by_gid<<<gn, 256, (++c->launches, 0), s>>>(vflag, gid, n, fg);
    tock(3);
    // border triangulations, one instance per merge node
    tick();
    const int64_t mB = std::max<int64_t>(nVB, 1);
    void* PB = pool_get(c, "dc.PB", psz * mB);
    int* gidB = (int*)pool_get(c, "dc.gidB", 4 * mB);
    int* instB = (int*)pool_get(c, "dc.zB", 4 * mB);
    int* cntB = (int*)pool_get(c, "rb.cntB", 4 * (size_t)nm);
    if (!PB || !gidB || !instB || !cntB) return set_err(c, DT_E_NOMEM, "border points");
    CUDA_OK(cudaMemsetAsync(cntB, 0, 4 * (size_t)nm, s));
    if (nVB) {
      unsigned gb = (unsigned)ceil_div<int64_t>(nVB, 256);
      gather_points(c, dim, Ps, idxB, nVB, PB);
      k_gather_i32<<<gb, 256, (++c->launches, 0), s>>>(gid, idxB, nVB, gidB);
      k_rb_inst<<<gb, 256, (++c->launches, 0), s>>>(part, idxB, nVB, instB, cntB);
    }
    std::vector<int> hc(nm);
    CUDA_OK(cudaMemcpyAsync(hc.data(), cntB, 4 * (size_t)nm, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    std::vector<int64_t> poffB(nm + 1, 0);
    for (int i = 0; i < nm; i++) poffB[i + 1] = poffB[i] + hc[i];
    rc = engine_run(c, c->run_border, dim, PB, gidB, instB, nVB, poffB, "border");
    if (rc) return rc;
    for (int i = 0; i < nm; i++)   // a flat or tiny border set has no full-dimensional simplices
      if (c->run_border.h_status[i] != 0) {
        c->run_border.h_tcount[i] = (int)c->run_border.h_toff[i];
        CUDA_OK(cudaMemcpyAsync(c->run_border.tcount + i, c->run_border.toff + i, 4, cudaMemcpyDeviceToDevice, s));
      }
    c->stats.rounds_max = std::max(c->stats.rounds_max, c->run_border.rounds);
    tock(4);
    // merge of every node's two children
    tick();
    k_rb_by_gid<<<gn, 256, (++c->launches, 0), s>>>(part, gid, n, labg);
    int4* rows;
    int64_t nrows;
    MergeStats ms;
    rc = merge(c, dim, *arena, gid, bflag, c->run_border, gidB, labg, &rows, &nrows, &ms, nullptr);
    if (rc) return rc;
    nVB_total += nVB;
    nB_total += ms.n_border_simplices;
    nTB_total += ms.n_tb;
    if (h < L) {
      int32_t *packed, *nbr;
      int64_t m, non_manifold = 0;
      rc = canonicalize_rows(c, dim, rows, nrows, n, &packed, &m, "rb.canon");
      if (rc) return rc;
      rc = match_all_facets(c, dim, packed, m, &nbr, &non_manifold);
      if (rc) return rc;
      if (non_manifold) return set_err(c, DT_E_INTERNAL, "a merged part has a facet in more than two simplices");
      k_rb_part<<<gn, 256, (++c->launches, 0), s>>>(leaf, n, h, part);
      rc = rows_to_arena(c, dim, Ps, packed, nbr, m, where, part, nm, n, fa);
      if (rc) return rc;
      arena = &fa;
      tock(5);
    } else {
      tock(5);
      tick();
      rc = canonicalize_rows(c, dim, rows, nrows, n, &c->out, &c->nout, "final");
      if (rc) return rc;
      tock(6);
    }
  }
  c->links = LinkSources();
  c->links_ok = false;
  // border vertices of all levels in global indices, ascending
  c->border_vtx = (int32_t*)pool_get(c, "dc.bv", 4 * n);
  if (!c->border_vtx) return set_err(c, DT_E_NOMEM, "border vertex list");
  int64_t nbv = 0;
  rc = compact_flags(c, fg, n, c->border_vtx, &nbv, "dc.cbv");
  if (rc) return rc;
  c->n_border = nbv;
  rc = check_status(c, "recursive bisection");
  if (rc) return rc;
  c->eta = eta_total;
  c->stats.eta = eta_total;
  c->stats.k = k;
  c->stats.cut_weight = 0;
  c->stats.border_vertices = nVB_total;
  c->stats.border_simplices = nB_total;
  c->stats.border_dt_simplices = nTB_total;
  c->stats.o_dt = (double)(n + eta_total + nVB_total) / (double)n;
  c->rows_only = true;
  return 0;
}

}  // namespace gdt
