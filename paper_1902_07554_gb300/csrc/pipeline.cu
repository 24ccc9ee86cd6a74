// pipeline.cu -- Alg. 1 driver: divide (Alg. 2 or kd), partial DTs,
// border detection, border DT, merge, canonical output.
#include <cmath>

#include "adjacency.cuh"
#include "border.cuh"
#include "divide.cuh"
#include "merge.cuh"
#include "pipeline.cuh"
#include "sort.cuh"

namespace gdt {



// Base case of Alg. 1 (n < N, or k = 1): one triangulation of all points.
int run_direct(dt_ctx* c, const void* P, int64_t n, int dim) {
  cudaStream_t s = c->stream;
  int* gid = (int*)pool_get(c, "pl.gid", 4 * n);
  int* pinst = (int*)pool_get(c, "pl.pinst", 4 * n);
  if (!gid || !pinst) return set_err(c, DT_E_NOMEM, "pipeline buffers");
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  k_iota<<<g, 256, (++c->launches, 0), s>>>(gid, n, 0);
  CUDA_OK(cudaMemsetAsync(pinst, 0, 4 * n, s));
  std::vector<int64_t> poff = {0, n};
  int rc = engine_run(c, c->run_parts, dim, P, gid, pinst, n, poff, "parts");
  if (rc) return rc;
  if (c->run_parts.h_status[0] == 1) return set_err(c, DT_E_DEGENERATE, "all points are collinear/coplanar");
  if (c->run_parts.h_status[0] != 0) return set_err(c, DT_E_ARG, "too few points");
  c->stats.rounds_max = c->run_parts.rounds;
  int4* rows; int64_t nrows;
  int *src, *osrc;
  rc = collect_finite(c, c->run_parts, gid, nullptr, 0, &rows, &nrows, "final", &src, 0);
  if (rc) return rc;
  rc = canonicalize_rows(c, dim, rows, nrows, n, &c->out, &c->nout, "final", src, &osrc);
  if (rc) return rc;
  c->links = LinkSources();
  c->links.tv0 = (const int4*)c->run_parts.tv;
  c->links.tn0 = (const int4*)c->run_parts.tn;
  c->links.gid0 = gid;
  c->links.base1 = c->run_parts.total_slots;
  c->links.total = c->run_parts.total_slots;
  c->links.origin = osrc;
  c->links_ok = true;
  c->stats.k = 1;
  c->labels = (int32_t*)pool_get(c, "pl.labels", 4 * n);
  if (!c->labels) return set_err(c, DT_E_NOMEM, "labels");
  CUDA_OK(cudaMemsetAsync(c->labels, 0, 4 * n, s));
  c->sample = nullptr;
  c->sample_block = nullptr;
  c->eta = 0;
  c->border_vtx = nullptr;
  c->n_border = 0;
  return check_status(c, "direct triangulation");
}

__global__ void k_flag_compact(const unsigned char* flag, const int* pos, int64_t n, int* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[pos[i]] = (int)i;
}
__global__ void k_u8_to_i32(const unsigned char* a, int64_t n, int* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
__global__ void k_gather_i32(const int* src, const int* idx, int64_t m, int* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = src[idx[i]];
}
__global__ void k_flag_by_gid(const unsigned char* vflag, const int* gid, int64_t n, unsigned char* fg) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && vflag[i]) fg[gid[i]] = 1;
}

// Indices i with flag[i] set, ascending; *m receives the count.
int compact_flags(dt_ctx* c, const unsigned char* flag, int64_t n, int* out, int64_t* m, const char* tag) {
  int* f32 = (int*)pool_get(c, std::string(tag) + ".f", 4 * std::max<int64_t>(n, 1));
  int* pos = (int*)pool_get(c, std::string(tag) + ".p", 4 * std::max<int64_t>(n, 1));
  if (!f32 || !pos) return set_err(c, DT_E_NOMEM, "compaction");
  unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(n, 1), 256);
  k_u8_to_i32<<<g, 256, (++c->launches, 0), c->stream>>>(flag, n, f32);
  int total = 0;
  int rc = exclusive_scan_i32(c, f32, pos, n, &total);
  if (rc) return rc;
  k_flag_compact<<<g, 256, (++c->launches, 0), c->stream>>>(flag, pos, n, out);
  *m = total;
  return 0;
}

static float ev_ms(dt_ctx* c, int a, int b) {
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]);
  return ms;
}

// Alg. 1 with k partitions.
static int run_dc(dt_ctx* c, const void* P, int64_t n, int dim, int k, double frac) {
  cudaStream_t s = c->stream;
  const dt_config& cfg = c->cfg;
  int rc;
  c->labels = (int32_t*)pool_get(c, "pl.labels", 4 * n);
  if (!c->labels) return set_err(c, DT_E_NOMEM, "labels");
  cudaEventRecord(c->ev[2], s);
  // ---------------- (a) divide
  c->sample = nullptr;
  c->sample_block = nullptr;
  c->eta = 0;
  if (cfg.divide == DT_DIVIDE_SAMPLE) {
    if (k > 256) return set_err(c, DT_E_ARG, "the sample divide supports k <= 256");
    int64_t eta = sample_size(n, frac, dim);
    int* ids = (int*)pool_get(c, "dc.sample", 4 * eta);
    int* zeros = (int*)pool_get(c, "dc.szero", 4 * eta);
    void* PS = pool_get(c, "dc.PS", (dim == 2 ? 16 : 32) * (size_t)eta);
    int* block = (int*)pool_get(c, "dc.block", 4 * eta);
    if (!ids || !zeros || !PS || !block) return set_err(c, DT_E_NOMEM, "sample buffers");
    rc = select_sample(c, n, eta, cfg.seed, ids);
    if (rc) return rc;
    gather_points(c, dim, P, ids, eta, PS);
    CUDA_OK(cudaMemsetAsync(zeros, 0, 4 * eta, s));
    rc = engine_run(c, c->run_sample, dim, PS, ids, zeros, eta, {0, eta}, "sample");
    if (rc) return rc;
    if (c->run_sample.h_status[0] != 0) return run_direct(c, P, n, dim);   // flat sample
    SampleGraph G;
    rc = sample_graph(c, c->run_sample, PS, dim, cfg.weight, G);
    if (rc) return rc;
    cudaEventRecord(c->ev[3], s);
    // Alg. 2's assignment walk needs the sample DT but not the blocks: it runs on a
    // second stream beside the partitioner, and the labels are mapped once both are done
    int* nearest = (int*)pool_get(c, "dc.nearest", 4 * (size_t)n);
    if (!nearest) return set_err(c, DT_E_NOMEM, "nearest sample points");
    if (!c->aux_stream && cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->aux_stream = nullptr;
    }
    for (cudaEvent_t& e : c->aux_ev)
      if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); e = nullptr; }
    const bool aux = c->aux_stream && c->aux_ev[0] && c->aux_ev[1];
    if (aux) {
      CUDA_OK(cudaEventRecord(c->aux_ev[0], s));
      CUDA_OK(cudaStreamWaitEvent(c->aux_stream, c->aux_ev[0], 0));
      c->stream = c->aux_stream;
    }
    rc = label_points(c, dim, P, n, PS, ids, G, nullptr, nullptr, nearest);
    if (aux) {
      cudaEventRecord(c->aux_ev[1], c->aux_stream);
      c->stream = s;
    }
    if (rc) return rc;
    rc = partition_graph(c, PS, dim, G, k, cfg.epsilon, cfg.lp_rounds, cfg.partition_init, block);
    if (rc) return rc;
    long long cut = 0;
    rc = cut_weight(c, G, block, &cut);
    if (rc) return rc;
    c->stats.cut_weight = cut;
    if (aux) CUDA_OK(cudaStreamWaitEvent(s, c->aux_ev[1], 0));
    map_labels(c, nearest, block, n, c->labels);
    c->sample = ids;
    c->sample_block = block;
    c->eta = eta;
    c->stats.eta = eta;
  } else {
    cudaEventRecord(c->ev[3], s);
    rc = kd_divide(c, dim, P, n, k, c->labels);
    if (rc) return rc;
  }
  // stable counting sort by label
  void* Ps = pool_get(c, "dc.Ps", (dim == 2 ? 16 : 32) * (size_t)n);
  int* gid_sorted = (int*)pool_get(c, "dc.gid", 4 * n);
  int* pinst = (int*)pool_get(c, "dc.pinst", 4 * n);
  if (!Ps || !gid_sorted || !pinst) return set_err(c, DT_E_NOMEM, "scatter buffers");
  std::vector<int64_t> poff, sizes;
  rc = scatter_by_label(c, dim, P, c->labels, n, k, Ps, gid_sorted, pinst, poff, sizes);
  if (rc) return rc;
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
  cudaEventRecord(c->ev[4], s);
  // ---------------- (b) partial triangulations
  rc = engine_run(c, c->run_parts, dim, Ps, gid_sorted, pinst, n, poff, "parts");
  if (rc) return rc;
  c->stats.rounds_max = c->run_parts.rounds;
  cudaEventRecord(c->ev[5], s);
  // ---------------- (c) border simplices and vertices(B)
  unsigned char *bflag, *vflag;
  int64_t nB = 0;
  rc = border_detect(c, dim, c->run_parts, Ps, pinst, k, cfg.grid_cell, cfg.primitive, &bflag, &vflag, &nB);
  if (rc) return rc;
  int* idxB = (int*)pool_get(c, "dc.idxB", 4 * n);
  if (!idxB) return set_err(c, DT_E_NOMEM, "border list");
  int64_t nVB = 0;
  rc = compact_flags(c, vflag, n, idxB, &nVB, "dc.cvb");
  if (rc) return rc;
  cudaEventRecord(c->ev[6], s);
  // ---------------- (d) border triangulation T_B = DT(vertices(B))
  void* PB = pool_get(c, "dc.PB", (dim == 2 ? 16 : 32) * (size_t)std::max<int64_t>(nVB, 1));
  int* gidB = (int*)pool_get(c, "dc.gidB", 4 * std::max<int64_t>(nVB, 1));
  int* zB = (int*)pool_get(c, "dc.zB", 4 * std::max<int64_t>(nVB, 1));
  if (!PB || !gidB || !zB) return set_err(c, DT_E_NOMEM, "border points");
  if (nVB) {
    gather_points(c, dim, Ps, idxB, nVB, PB);
    k_gather_i32<<<(unsigned)ceil_div<int64_t>(nVB, 256), 256, (++c->launches, 0), s>>>(gid_sorted, idxB, nVB, gidB);
    CUDA_OK(cudaMemsetAsync(zB, 0, 4 * nVB, s));
  }
  rc = engine_run(c, c->run_border, dim, PB, gidB, zB, nVB, {0, nVB}, "border");
  if (rc) return rc;
  // a flat or tiny border vertex set has no full-dimensional simplices
  if (c->run_border.h_status[0] != 0) c->run_border.h_tcount[0] = (int)c->run_border.h_toff[0];
  c->stats.rounds_max = std::max(c->stats.rounds_max, c->run_border.rounds);
  cudaEventRecord(c->ev[7], s);
  // ---------------- (e) merge
  if (c->run_border.h_status[0] != 0)
    CUDA_OK(cudaMemcpyAsync(c->run_border.tcount, c->run_border.toff, 4, cudaMemcpyDeviceToDevice, s));
  int4* rows;
  int64_t nrows;
  MergeStats ms;
  int *src, *osrc;
  rc = merge(c, dim, c->run_parts, gid_sorted, bflag, c->run_border, gidB, c->labels, &rows, &nrows, &ms, &src);
  if (rc) return rc;
  cudaEventRecord(c->ev[8], s);
  rc = canonicalize_rows(c, dim, rows, nrows, n, &c->out, &c->nout, "final", src, &osrc);
  if (rc) return rc;
  c->links = LinkSources();
  c->links.tv0 = (const int4*)c->run_parts.tv;
  c->links.tn0 = (const int4*)c->run_parts.tn;
  c->links.gid0 = gid_sorted;
  c->links.base1 = c->run_parts.total_slots;
  c->links.tv1 = (const int4*)c->run_border.tv;
  c->links.tn1 = (const int4*)c->run_border.tn;
  c->links.gid1 = gidB;
  c->links.total = c->run_parts.total_slots + c->run_border.total_slots;
  c->links.origin = osrc;
  c->links_ok = true;
  cudaEventRecord(c->ev[9], s);
  // border vertex list in global indices, ascending
  unsigned char* fg = (unsigned char*)pool_get(c, "dc.fg", n);
  c->border_vtx = (int32_t*)pool_get(c, "dc.bv", 4 * std::max<int64_t>(nVB, 1));
  if (!fg || !c->border_vtx) return set_err(c, DT_E_NOMEM, "border vertex list");
  CUDA_OK(cudaMemsetAsync(fg, 0, n, s));
  k_flag_by_gid<<<(unsigned)ceil_div<int64_t>(n, 256), 256, (++c->launches, 0), s>>>(vflag, gid_sorted, n, fg);
  int64_t nbv = 0;
  rc = compact_flags(c, fg, n, c->border_vtx, &nbv, "dc.cbv");
  if (rc) return rc;
  c->n_border = nbv;
  rc = check_status(c, "divide and conquer");
  if (rc) return rc;
  c->stats.k = k;
  c->stats.border_vertices = nVB;
  c->stats.border_simplices = ms.n_border_simplices;
  c->stats.border_dt_simplices = ms.n_tb;
  c->stats.o_dt = (double)(n + c->eta + nVB) / (double)n;
  c->stats.ms_phase[0] = ev_ms(c, 2, 3);
  c->stats.ms_phase[1] = ev_ms(c, 3, 4);
  c->stats.ms_phase[2] = ev_ms(c, 4, 5);
  c->stats.ms_phase[3] = ev_ms(c, 5, 6);
  c->stats.ms_phase[4] = ev_ms(c, 6, 7);
  c->stats.ms_phase[5] = ev_ms(c, 7, 8);
  c->stats.ms_phase[6] = ev_ms(c, 8, 9);
  return 0;
}

// ---------------------------------------------------------------- batches
__global__ void k_inst_of_point(const long long* off, int count, int64_t n, int* inst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  inst[i] = lo;
}

// Canonical rows (global indices) -> instance-local indices, per-instance counts.
template <int D>
__global__ void k_rows_to_local(int32_t* rows, int64_t nrows, const long long* off, int count, int* icount) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int32_t* row = rows + r * (D + 1);
  int v0 = row[0];
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= v0) lo = mid; else hi = mid - 1;
  }
  int base = (int)off[lo];
  for (int j = 0; j <= D; j++) row[j] -= base;
  atomicAdd(&icount[lo], 1);
}

// Many independent problems in one engine run: instance i is points
// [offsets[i], offsets[i+1]); each is triangulated directly.
int run_batch(dt_ctx* c, const double* points, const int64_t* offsets, int count, int dim) {
  cudaStream_t s = c->stream;
  c->links_ok = false;
  c->rows_only = false;
  c->nbr_ok = false;
  int64_t n = offsets[count];
  std::vector<int64_t> poff(offsets, offsets + count + 1);
  std::vector<long long> hoff(offsets, offsets + count + 1);
  long long* doff = (long long*)pool_get(c, "bt.off", 8 * (size_t)(count + 1));
  int* pinst = (int*)pool_get(c, "bt.pinst", 4 * std::max<int64_t>(n, 1));
  int* gid = (int*)pool_get(c, "bt.gid", 4 * std::max<int64_t>(n, 1));
  int* icount = (int*)pool_get(c, "bt.icount", 4 * (size_t)(count + 1));
  int* ipos = (int*)pool_get(c, "bt.ipos", 4 * (size_t)(count + 1));
  if (!doff || !pinst || !gid || !icount || !ipos) return set_err(c, DT_E_NOMEM, "batch buffers");
  CUDA_OK(cudaMemcpyAsync(doff, hoff.data(), 8 * (size_t)(count + 1), cudaMemcpyHostToDevice, s));
  unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(n, 1), 256);
  k_inst_of_point<<<g, 256, (++c->launches, 0), s>>>(doff, count, n, pinst);
  void* P = nullptr;
  int rc = stage_points(c, points, n, dim, &P, "in", pinst);
  if (rc) return rc;
  k_iota<<<g, 256, (++c->launches, 0), s>>>(gid, n, 0);
  cudaEventRecord(c->ev[4], s);
  rc = engine_run(c, c->run_parts, dim, P, gid, pinst, n, poff, "parts");
  if (rc) return rc;
  cudaEventRecord(c->ev[5], s);
  c->stats.rounds_max = c->run_parts.rounds;
  int4* rows;
  int64_t nrows;
  rc = collect_finite(c, c->run_parts, gid, nullptr, 0, &rows, &nrows, "final");
  if (rc) return rc;
  rc = canonicalize_rows(c, dim, rows, nrows, std::max<int64_t>(n, 1), &c->out, &c->nout, "final");
  if (rc) return rc;
  CUDA_OK(cudaMemsetAsync(icount, 0, 4 * (size_t)(count + 1), s));
  if (nrows) {
    unsigned gr = (unsigned)ceil_div<int64_t>(nrows, 256);
    if (dim == 2) k_rows_to_local<2><<<gr, 256, (++c->launches, 0), s>>>(c->out, nrows, doff, count, icount);
    else k_rows_to_local<3><<<gr, 256, (++c->launches, 0), s>>>(c->out, nrows, doff, count, icount);
  }
  int total = 0;
  rc = exclusive_scan_i32(c, icount, ipos, count + 1, &total);
  if (rc) return rc;
  std::vector<int> hp(count + 1);
  CUDA_OK(cudaMemcpyAsync(hp.data(), ipos, 4 * (size_t)(count + 1), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  c->batch_offsets.assign(hp.begin(), hp.end());
  c->batch_status.assign(count, 0);
  for (int i = 0; i < count; i++)
    c->batch_status[i] = c->run_parts.h_status[i] == 0 ? 0 : (c->run_parts.h_status[i] == 1 ? DT_E_DEGENERATE : DT_E_ARG);
  c->batch_count = count;
  c->stats.ms_phase[2] = ev_ms(c, 4, 5);
  c->labels = nullptr;
  c->sample = nullptr;
  c->sample_block = nullptr;
  c->border_vtx = nullptr;
  c->eta = 0;
  c->n_border = 0;
  return check_status(c, "batch");
}

// Neighbourhood update of the last result (once per result).
int ensure_neighbors(dt_ctx* c) {
  if (c->nbr_ok) return 0;
  int rc;
  if (c->links_ok) {
    rc = neighbor_update(c, c->dim, c->out, c->nout, c->links, &c->nbr);
  } else if (c->rows_only) {   // a single triangulation without link sources: every facet through the hash
    int64_t nm = 0;
    rc = match_all_facets(c, c->dim, c->out, c->nout, &c->nbr, &nm);
    if (!rc && nm) rc = set_err(c, DT_E_INTERNAL, "a facet in more than two simplices");
  } else {
    return set_err(c, DT_E_ARG, "no single triangulation result to link");
  }
  if (rc) return rc;
  c->nbr_ok = true;
  return 0;
}

int run_pipeline(dt_ctx* c, const double* points, int64_t n, int dim, int k, double frac) {
  void* P = nullptr;
  c->links_ok = false;
  c->rows_only = false;
  c->nbr_ok = false;
  int rc = stage_points(c, points, n, dim, &P, "in");
  if (rc) return rc;
  if (k == 1 || n / k < c->cfg.base_threshold) rc = run_direct(c, P, n, dim);
  else if (c->cfg.recursive) rc = run_recursive(c, P, n, dim, k, frac);
  else rc = run_dc(c, P, n, dim, k, frac);
  if (rc) return rc;
  if (!c->cfg.neighbors && !c->cfg.validate) return 0;
  cudaEventRecord(c->ev[10], c->stream);
  rc = ensure_neighbors(c);
  if (rc) return rc;
  if (c->cfg.validate) {
    dt_validation v;
    rc = validate_rows(c, dim, P, n, c->out, c->nout, c->nbr, 0, &v);
    if (rc) return rc;
    if (v.violations) {
      char msg[256];
      snprintf(msg, sizeof msg,
               "certificate failed: flat %lld, non-manifold %lld, asymmetric %lld, folded %lld, non-Delaunay %lld, "
               "non-convex %lld, unused %lld, pivot %lld, euler %lld",
               (long long)v.flat, (long long)v.non_manifold, (long long)v.asymmetric, (long long)v.folded,
               (long long)v.non_delaunay, (long long)v.non_convex, (long long)v.unused_points,
               (long long)v.pivot_limit, (long long)v.euler);
      return set_err(c, DT_E_INTERNAL, msg);
    }
    c->stats.validated = 1;
  }
  cudaEventRecord(c->ev[11], c->stream);
  CUDA_OK(cudaEventSynchronize(c->ev[11]));
  c->stats.ms_phase[7] = ev_ms(c, 10, 11);
  return 0;
}

}  // namespace gdt

namespace gdt {
__global__ void k_i64_to_i32b(const long long* in, int* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)in[i];
}
}  // namespace gdt

using namespace gdt;

// Alg. 2 (assignment of the points) on caller inputs (see include/dt.h).
extern "C" int dt_label_points(dt_ctx* c, const double* P, int64_t n, int dim, const double* S,
                               const int64_t* srank, const int32_t* block, int64_t m, int32_t* out) {
  if (!c) return DT_E_ARG;
  if (!P || !S || !srank || !block || !out || (dim != 2 && dim != 3) || n < 1 || m < dim + 1)
    return set_err(c, DT_E_ARG, "bad label arguments");
  cudaSetDevice(c->device);
  cudaStream_t s = c->stream;
  void *dP, *dS;
  int rc = stage_points(c, P, n, dim, &dP, "lp.P");
  if (rc) return rc;
  rc = stage_points(c, S, m, dim, &dS, "lp.S");
  if (rc) return rc;
  const long long* r64 = (const long long*)stage_in(c, srank, 8 * m, "lp.r64", &rc);
  if (rc) return rc;
  const int* dblock = (const int*)stage_in(c, block, 4 * m, "lp.block", &rc);
  if (rc) return rc;
  int* r32 = (int*)pool_get(c, "lp.r32", 4 * m);
  int* zeros = (int*)pool_get(c, "lp.z", 4 * m);
  int* lab = (int*)pool_get(c, "lp.out", 4 * n);
  if (!r32 || !zeros || !lab) return set_err(c, DT_E_NOMEM, "label buffers");
  k_i64_to_i32b<<<(unsigned)ceil_div<int64_t>(m, 256), 256, (++c->launches, 0), s>>>(r64, r32, m);
  CUDA_OK(cudaMemsetAsync(zeros, 0, 4 * m, s));
  EngineRun run;
  rc = engine_run(c, run, dim, dS, r32, zeros, m, {0, m}, "lp.dt");
  if (rc) return rc;
  if (run.h_status[0] != 0) return set_err(c, DT_E_DEGENERATE, "sample points are flat");
  SampleGraph G;
  rc = sample_graph(c, run, dS, dim, DT_WEIGHT_CONSTANT, G);
  if (rc) return rc;
  rc = label_points(c, dim, dP, n, dS, r32, G, dblock, lab, nullptr);
  if (rc) return rc;
  rc = check_status(c, "label points");
  if (rc) return rc;
  return copy_out(c, out, lab, 4 * n);
}

// The k-way partitioner on a caller graph (see include/dt.h).
extern "C" int dt_partition_graph(dt_ctx* c, const double* S, int64_t eta, int dim, const int32_t* E,
                                  const int64_t* w, int64_t m, int k, double eps, int rounds, int32_t* out) {
  if (!c) return DT_E_ARG;
  if (!S || !out || (dim != 2 && dim != 3) || eta < 1 || m < 0 || (m > 0 && (!E || !w)) || k < 1 || k > 256 ||
      eps < 0 || rounds < 0)
    return set_err(c, DT_E_ARG, "bad partition arguments");
  cudaSetDevice(c->device);
  cudaStream_t s = c->stream;
  void* dS;
  int rc = stage_points(c, S, eta, dim, &dS, "pg.S");
  if (rc) return rc;
  SampleGraph G;
  G.eta = eta;
  G.m = m;
  G.E = (int2*)stage_in(c, E ? (const void*)E : (const void*)S, 8 * std::max<int64_t>(m, 1), "pg.E", &rc);
  if (rc) return rc;
  G.w = (long long*)stage_in(c, w ? (const void*)w : (const void*)S, 8 * std::max<int64_t>(m, 1), "pg.w", &rc);
  if (rc) return rc;
  G.box = (double*)pool_get(c, "pg.box", 48);
  int* block = (int*)pool_get(c, "pg.block", 4 * eta);
  if (!G.box || !block) return set_err(c, DT_E_NOMEM, "partition buffers");
  rc = graph_bbox(c, dim, dS, eta, G.box);
  if (rc) return rc;
  rc = build_csr(c, G);
  if (rc) return rc;
  rc = partition_graph(c, dS, dim, G, k, eps, rounds, c->cfg.partition_init, block);
  if (rc) return rc;
  rc = check_status(c, "partition graph");
  if (rc) return rc;
  return copy_out(c, out, block, 4 * eta);
}
