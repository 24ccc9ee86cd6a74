// capi.cu -- the C ABI (include/dt.h): context, argument checks, input
// staging, and the orchestration of Alg. 1 (see pipeline.cu for the
// divide-and-conquer steps).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "ctx.cuh"
#include "adjacency.cuh"
#include "jobs.h"
#include "pipeline.cuh"

using namespace gdt;

namespace gdt {
const char* last_cuda_fail();

int pred_counters_engine(dt_ctx* c, unsigned long long* calls, int* range, bool reset);
}  // namespace gdt

extern "C" int dt_config_default(dt_config* cfg) {
  if (!cfg) return DT_E_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->divide = DT_DIVIDE_SAMPLE;
  cfg->primitive = DT_PRIM_GRID;
  cfg->weight = DT_WEIGHT_LOG;
  cfg->lp_rounds = 16;
  cfg->epsilon = 0.05;
  cfg->grid_cell = 1.0;
  cfg->seed = 1;
  cfg->base_threshold = 2048;
  cfg->validate = 0;
  cfg->cavity_cap = 0;
  return DT_OK;
}

static bool cfg_valid(const dt_config* c) {
  return c->divide >= 0 && c->divide <= 1 && c->primitive >= 0 && c->primitive <= 2 && c->weight >= 0 &&
         c->weight <= 3 && c->lp_rounds >= 0 && c->lp_rounds <= 1000 && c->epsilon >= 0 && c->epsilon <= 10 &&
         c->grid_cell > 0 && c->grid_cell <= 64 && c->base_threshold >= 0 && c->cavity_cap >= 0 &&
         c->cavity_cap <= 4096 && c->first_batch >= 0 &&
         (c->brio_growth == 0 || (c->brio_growth > 100 && c->brio_growth <= 10000)) && c->small_rounds >= -1 &&
         c->brio_drain >= 0 && c->brio_drain <= 64 && c->partition_init >= 0 && c->partition_init <= 2 &&
         (c->recursive == 0 || c->recursive == 1) && c->active_ratio >= 0 && c->active_ratio <= 10000 &&
         c->nominate_rings >= 0 && c->nominate_rings <= 2 && (c->partitioner == DT_PART_LP ||
         c->partitioner == DT_PART_MULTILEVEL) && c->round_limit >= 0 && c->walk_limit >= 0 &&
         c->arena_factor >= 0 && c->arena_factor <= 1024 && c->cavity_blocks >= 0 && c->cavity_blocks <= 64 &&
         (c->cavity_occupancy == 0 || c->cavity_occupancy == 8 || c->cavity_occupancy == 12 ||
          c->cavity_occupancy == 16) &&
         (c->cavity_group == 0 || c->cavity_group == 16 || c->cavity_group == 32);
}

extern "C" int dt_create(dt_ctx** out, int device, void* cuda_stream, const dt_config* cfg) {
  if (!out) return DT_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DT_E_ARG;
  }
  if (cfg && !cfg_valid(cfg)) return DT_E_ARG;
  dt_ctx* c = new dt_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return DT_E_CUDA; }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return DT_E_CUDA; }
    c->own_stream = true;
  }
  if (cfg) c->cfg = *cfg; else dt_config_default(&c->cfg);
  {
    int m = 0;
    if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && m > 0) c->sms = m;
    else cudaGetLastError();
  }
  if (cudaMalloc(&c->status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->status_host, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->counters_host, 64 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    dt_destroy(c);
    return DT_E_NOMEM;
  }
  for (int i = 0; i < 16; i++) cudaEventCreate(&c->ev[i]);
  for (int i = 0; i < 16; i++) cudaEventCreate(&c->pev[i]);
  memset(&c->stats, 0, sizeof(c->stats));
  *out = c;
  return DT_OK;
}

extern "C" int dt_set_config(dt_ctx* c, const dt_config* cfg) {
  if (!c) return DT_E_ARG;
  if (cfg && !cfg_valid(cfg)) return set_err(c, DT_E_ARG, "invalid configuration");
  if (cfg) c->cfg = *cfg; else dt_config_default(&c->cfg);
  return DT_OK;
}

extern "C" void dt_destroy(dt_ctx* c) {
  if (!c) return;
  delete c->jobs;            // lets a running job finish, drops queued ones, joins the worker
  c->jobs = nullptr;
  if (c->job_ctx) dt_destroy(c->job_ctx);
  c->job_ctx = nullptr;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  dt_stream_cleanup(c);
  pool_free_all(c);
  if (c->status) cudaFree(c->status);
  if (c->status_host) cudaFreeHost(c->status_host);
  if (c->counters_host) cudaFreeHost(c->counters_host);
  for (int i = 0; i < 16; i++) if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (int i = 0; i < 16; i++) if (c->pev[i]) cudaEventDestroy(c->pev[i]);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (auto& rg : c->round_graphs) {
    if (rg.gx) cudaGraphExecDestroy(rg.gx);
    if (rg.g) cudaGraphDestroy(rg.g);
  }
  c->round_graphs.clear();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  for (cudaEvent_t e : c->aux_ev) if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

extern "C" const char* dt_last_error(dt_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

namespace gdt {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from a host-or-device pointer into a pool buffer.
void* stage_in(dt_ctx* c, const void* src, size_t bytes, const std::string& name, int* rc) {
  void* d = pool_get(c, name, bytes);
  if (!d) { *rc = set_err(c, DT_E_NOMEM, "staging " + name); return nullptr; }
  cudaError_t e = cudaMemcpyAsync(d, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) { *rc = set_err(c, gdt_cuda_fail(e, "stage_in", __FILE__, __LINE__), "staging"); return nullptr; }
  *rc = 0;
  return d;
}

int copy_out(dt_ctx* c, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return 0;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                                       : cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "copy_out", __FILE__, __LINE__), "copy out");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "copy_out", __FILE__, __LINE__), "copy out");
  return 0;
}

// Row-major (n x D) doubles -> the engine's point layout (double2 / double4_32a),
// with a finiteness check.
template <int D>
__global__ void k_pack_points(const double* in, int64_t n, typename PT<D>::T* out, int* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = in[i * D], y = in[i * D + 1], z = D == 3 ? in[i * D + 2] : 0.0;
  if (!isfinite(x) || !isfinite(y) || !isfinite(z) || fabs(x) > 1e300 || fabs(y) > 1e300 || fabs(z) > 1e300)
    atomicExch(bad, 1);
  if constexpr (D == 2) out[i] = make_double2(x, y);
  else out[i] = make_double4_32a(x, y, z, 0.0);
}

__global__ void k_iota(int* a, int64_t n, int start) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int)(start + i);
}

// Exact-duplicate detection with an open-addressing table of point indices
// keyed by the coordinate bits (-0.0 folded onto +0.0).
template <int D>
__global__ void k_dup_check(const typename PT<D>::T* P, int64_t n, int* table, unsigned mask, int* dup,
                            const int* inst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = cx(P[i]) + 0.0, y = cy(P[i]) + 0.0, z = cz(P[i]) + 0.0;
  int my = inst ? inst[i] : 0;
  uint64_t h = splitmix64((uint64_t)__double_as_longlong(x) ^ splitmix64((uint64_t)__double_as_longlong(y) ^
                          splitmix64((uint64_t)__double_as_longlong(z) ^ (uint64_t)my)));
  unsigned slot = (unsigned)h & mask;
  for (unsigned probe = 0; probe <= mask; probe++) {
    int prev = atomicCAS(&table[slot], -1, (int)i);
    if (prev == -1) return;
    if (cx(P[prev]) == x && cy(P[prev]) == y && cz(P[prev]) == z && (!inst || inst[prev] == my)) {
      atomicExch(dup, 1);
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicExch(dup, 2);
}

int stage_points(dt_ctx* c, const double* points, int64_t n, int dim, void** P_out, const char* tag,
                 const int* inst) {
  int rc = 0;
  std::string t(tag);
  const double* src = (const double*)stage_in(c, points, sizeof(double) * n * dim, t + ".raw", &rc);
  if (rc) return rc;
  size_t psz = dim == 2 ? sizeof(double2) : sizeof(double4_32a);
  void* P = pool_get(c, t + ".pts", psz * n);
  int* flags = (int*)pool_get(c, t + ".flags", 16);
  unsigned tsize = 1;
  while (tsize < 2 * n) tsize <<= 1;
  int* table = (int*)pool_get(c, "in.dup", 4 * (size_t)tsize);
  if (!P || !flags || !table) return set_err(c, DT_E_NOMEM, "input staging");
  CUDA_OK(cudaMemsetAsync(flags, 0, 16, c->stream));
  CUDA_OK(cudaMemsetAsync(table, 0xff, 4 * (size_t)tsize, c->stream));
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  if (dim == 2) {
    k_pack_points<2><<<g, 256, (++c->launches, 0), c->stream>>>(src, n, (double2*)P, flags);
    k_dup_check<2><<<g, 256, (++c->launches, 0), c->stream>>>((const double2*)P, n, table, tsize - 1, flags + 1, inst);
  } else {
    k_pack_points<3><<<g, 256, (++c->launches, 0), c->stream>>>(src, n, (double4_32a*)P, flags);
    k_dup_check<3><<<g, 256, (++c->launches, 0), c->stream>>>((const double4_32a*)P, n, table, tsize - 1, flags + 1, inst);
  }
  int h[2];
  CUDA_OK(cudaMemcpyAsync(h, flags, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  if (h[0]) return set_err(c, DT_E_ARG, "non-finite coordinate (or |x| > 1e300)");
  if (h[1] == 1) return set_err(c, DT_E_DUPLICATE, "two input points coincide");
  if (h[1]) return set_err(c, DT_E_INTERNAL, "duplicate table full");
  *P_out = P;
  return 0;
}

}  // namespace gdt

extern "C" int dt_triangulate(dt_ctx* c, const double* points, int64_t n, int dim, int k, double sample_frac) {
  if (!c) return DT_E_ARG;
  c->err.clear();
  if (!points || (dim != 2 && dim != 3)) return set_err(c, DT_E_ARG, "points must be non-null and dim 2 or 3");
  if (n < dim + 1) return set_err(c, DT_E_ARG, "need at least dim+1 points");
  if (n >= (int64_t(1) << 28)) return set_err(c, DT_E_ARG, "n must be below 2^28");
  if (k < 1 || k > 4096) return set_err(c, DT_E_ARG, "k must be in [1, 4096]");
  if (!(sample_frac >= 0.0 && sample_frac <= 1.0)) return set_err(c, DT_E_ARG, "sample_frac must be in [0, 1]");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  c->dim = dim;
  c->n = n;
  c->nout = 0;
  c->out = nullptr;
  memset(&c->stats, 0, sizeof(c->stats));
  c->stats.n = n;
  c->stats.dim = dim;
  c->stats.k = 1;
  c->kprof.clear();
  c->batch_count = 0;
  long long l0 = c->launches;
  cudaEventRecord(c->ev[0], c->stream);
  int rc = run_pipeline(c, points, n, dim, k, sample_frac);
  if (rc) return rc;
  cudaEventRecord(c->ev[1], c->stream);
  cudaError_t e = cudaEventSynchronize(c->ev[1]);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "sync", __FILE__, __LINE__), "final sync");
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
  c->stats.ms_total = ms;
  unsigned long long calls; int range;
  rc = pred_counters_engine(c, &calls, &range, true);
  if (rc) return rc;
  c->stats.exact_calls = (int32_t)std::min<unsigned long long>(calls, 0x7fffffffull);
  c->stats.simplices = c->nout;
  c->stats.launches = c->launches - l0;
  return DT_OK;
}

extern "C" int dt_get_kernel_profile(dt_ctx* c, dt_kernel_profile* out, int max, int* count) {
  if (!c || !count) return DT_E_ARG;
  *count = (int)c->kprof.size();
  if (!out) return DT_OK;
  for (int i = 0; i < max && i < (int)c->kprof.size(); i++) {
    memset(&out[i], 0, sizeof(out[i]));
    strncpy(out[i].name, c->kprof[i].name, 31);
    out[i].launches = c->kprof[i].launches;
    out[i].ms = c->kprof[i].ms;
    out[i].bytes = c->kprof[i].bytes;
    out[i].flops = c->kprof[i].flops;
  }
  return DT_OK;
}

extern "C" int dt_triangulate_batch(dt_ctx* c, const double* points, const int64_t* offsets, int count, int dim) {
  if (!c) return DT_E_ARG;
  c->err.clear();
  if (!points || !offsets || count < 1 || (dim != 2 && dim != 3))
    return set_err(c, DT_E_ARG, "batch: points, offsets, count >= 1 and dim 2 or 3 required");
  if (offsets[0] != 0) return set_err(c, DT_E_ARG, "batch: offsets[0] must be 0");
  for (int i = 0; i < count; i++)
    if (offsets[i + 1] < offsets[i]) return set_err(c, DT_E_ARG, "batch: offsets must be non-decreasing");
  if (offsets[count] >= (int64_t(1) << 28)) return set_err(c, DT_E_ARG, "batch: total points must be below 2^28");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  c->dim = dim;
  c->n = offsets[count];
  c->nout = 0;
  c->out = nullptr;
  c->batch_count = 0;
  memset(&c->stats, 0, sizeof(c->stats));
  c->stats.n = c->n;
  c->stats.dim = dim;
  c->stats.k = 1;
  c->kprof.clear();
  long long l0 = c->launches;
  cudaEventRecord(c->ev[0], c->stream);
  int rc = run_batch(c, points, offsets, count, dim);
  if (rc) return rc;
  cudaEventRecord(c->ev[1], c->stream);
  cudaError_t e = cudaEventSynchronize(c->ev[1]);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "sync", __FILE__, __LINE__), "final sync");
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
  c->stats.ms_total = ms;
  unsigned long long calls; int range;
  rc = pred_counters_engine(c, &calls, &range, true);
  if (rc) return rc;
  c->stats.exact_calls = (int32_t)std::min<unsigned long long>(calls, 0x7fffffffull);
  c->stats.simplices = c->nout;
  c->stats.launches = c->launches - l0;
  return DT_OK;
}

extern "C" int dt_get_batch_simplices(dt_ctx* c, int32_t* out, int64_t capacity, int64_t* out_offsets,
                                      int64_t* total) {
  if (!c || !total) return DT_E_ARG;
  if (!c->batch_count) return set_err(c, DT_E_ARG, "no batch result");
  *total = c->nout;
  if (out_offsets)
    for (int i = 0; i <= c->batch_count; i++) out_offsets[i] = c->batch_offsets[i];
  if (!out) return DT_OK;
  if (capacity < c->nout) return set_err(c, DT_E_ARG, "capacity too small");
  return copy_out(c, out, c->out, sizeof(int32_t) * (c->dim + 1) * c->nout);
}

extern "C" int dt_get_batch_status(dt_ctx* c, int32_t* status, int count) {
  if (!c || !status) return DT_E_ARG;
  if (count != c->batch_count) return set_err(c, DT_E_ARG, "count differs from the last batch");
  for (int i = 0; i < count; i++) status[i] = c->batch_status[i];
  return DT_OK;
}

extern "C" int dt_get_simplices(dt_ctx* c, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  *count = c->nout;
  if (!out) return DT_OK;
  if (capacity < c->nout) return set_err(c, DT_E_ARG, "capacity too small");
  return copy_out(c, out, c->out, sizeof(int32_t) * (c->dim + 1) * c->nout);
}

extern "C" int dt_get_simplices_device(dt_ctx* c, const int32_t** dptr, int64_t* count) {
  if (!c || !dptr || !count) return DT_E_ARG;
  *dptr = c->out;
  *count = c->nout;
  return DT_OK;
}

// Neighbourhood update of the merge (see include/dt.h).
extern "C" int dt_get_neighbors(dt_ctx* c, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  if (!c->links_ok && !c->rows_only)
    return set_err(c, DT_E_ARG, "no single triangulation result (call dt_triangulate first)");
  *count = c->nout;
  if (!out) return DT_OK;
  if (capacity < c->nout) return set_err(c, DT_E_ARG, "capacity too small");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  int rc = ensure_neighbors(c);
  if (rc) return rc;
  return copy_out(c, out, c->nbr, sizeof(int32_t) * (c->dim + 1) * c->nout);
}

// Certificate of a caller's triangulation (see include/dt.h).
extern "C" int dt_validate(dt_ctx* c, const double* points, int64_t n, int dim, const int32_t* simplices, int64_t m,
                           dt_validation* out) {
  if (!c) return DT_E_ARG;
  if (!points || !out || (dim != 2 && dim != 3) || n < dim + 1 || m < 0 || (m > 0 && !simplices))
    return set_err(c, DT_E_ARG, "bad validation arguments");
  if (n >= (int64_t(1) << 28)) return set_err(c, DT_E_ARG, "n must be below 2^28");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  void* P = nullptr;
  int rc = stage_points(c, points, n, dim, &P, "val.in");
  if (rc) return rc;
  const int32_t* in = m ? (const int32_t*)stage_in(c, simplices, sizeof(int32_t) * (dim + 1) * m, "val.rows_in", &rc)
                        : nullptr;
  if (rc) return rc;
  int32_t* rows = (int32_t*)pool_get(c, "val.rows", sizeof(int32_t) * (dim + 1) * std::max<int64_t>(m, 1));
  if (!rows) return set_err(c, DT_E_NOMEM, "validation rows");
  int64_t bad = 0, nm = 0;
  rc = prepare_rows(c, dim, in, m, n, rows, &bad);
  if (rc) return rc;
  int32_t* nbr = nullptr;
  rc = match_all_facets(c, dim, rows, m, &nbr, &nm);
  if (rc) return rc;
  rc = validate_rows(c, dim, P, n, rows, m, nbr, nm, out);
  if (rc) return rc;
  out->bad_index = bad;
  out->violations += bad;
  // the neighbour buffer is shared with the last result's: recompute it on demand
  c->nbr_ok = false;
  return DT_OK;
}

extern "C" int dt_get_stats(dt_ctx* c, dt_stats* s) {
  if (!c || !s) return DT_E_ARG;
  *s = c->stats;
  return DT_OK;
}

extern "C" int dt_get_labels(dt_ctx* c, int32_t* out, int64_t n) {
  if (!c || !out || n != c->n) return DT_E_ARG;
  if (!c->labels) return set_err(c, DT_E_ARG, "no labels (run dt_triangulate first)");
  return copy_out(c, out, c->labels, sizeof(int32_t) * n);
}

extern "C" int dt_get_sample(dt_ctx* c, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  *count = c->sample ? c->eta : 0;
  if (!out || !c->sample) return DT_OK;
  if (capacity < c->eta) return set_err(c, DT_E_ARG, "capacity too small");
  return copy_out(c, out, c->sample, sizeof(int32_t) * c->eta);
}

extern "C" int dt_get_sample_blocks(dt_ctx* c, int32_t* out, int64_t capacity) {
  if (!c || !out) return DT_E_ARG;
  if (!c->sample_block || capacity < c->eta) return set_err(c, DT_E_ARG, "no sample blocks or capacity too small");
  return copy_out(c, out, c->sample_block, sizeof(int32_t) * c->eta);
}

extern "C" int dt_get_border_vertices(dt_ctx* c, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  *count = c->border_vtx ? c->n_border : 0;
  if (!out || !c->border_vtx) return DT_OK;
  if (capacity < c->n_border) return set_err(c, DT_E_ARG, "capacity too small");
  return copy_out(c, out, c->border_vtx, sizeof(int32_t) * c->n_border);
}

// ---------------------------------------------------------------- predicates entry
namespace gdt {
template <int D>
__global__ void k_eval_pred(const typename PT<D>::T* P, const float4* X, const int* gid, int kind, const int32_t* tup,
                            int64_t m, int npts, int8_t* out, int* bad) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  int w = kind == 0 ? D + 1 : (kind == 3 ? 3 : D + 2);
  int t[5];
  for (int i = 0; i < w; i++) {
    t[i] = tup[r * w + i];
    if ((unsigned)t[i] >= (unsigned)npts) { atomicExch(bad, 1); out[r] = 0; return; }
  }
  int s = 0;
  if (kind == 0) {
    s = orient_px(P, X, t);
  } else if (kind == 1) {
    int v[4] = {t[0], t[1], t[2], t[3]};
    int o = orient_px(P, X, v);
    if (o == 0) { out[r] = 0; return; }
    if (o < 0) { int x = v[0]; v[0] = v[1]; v[1] = x; }
    s = insphere_sos_x(P, X, gid, v, t[D + 1], D);
  } else if (kind == 2) {
    int v[4] = {t[0], t[1], t[2], t[3]};
    // the sign of the raw determinant (both stages evaluate the same one)
    s = insphere_f_p(P, X, v, t[D + 1]);
    if (!s) s = insphere_raw_p(P, v, t[D + 1]);
  } else {
    s = closer(P[t[0]], P[t[1]], P[t[2]], D);
  }
  out[r] = (int8_t)s;
}

__global__ void k_i64_to_i32(const long long* in, int* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)in[i];
}

static __global__ void k_read_pred_counters_capi(unsigned long long* calls, int* range) {
  *calls = g_exact_calls;
  *range = g_range_error;
  g_exact_calls = 0;
}
}  // namespace gdt

extern "C" int dt_eval_predicates(dt_ctx* c, const double* points, int64_t n, int dim, const int64_t* gid,
                                  int kind, const int32_t* tuples, int64_t m, int8_t* out) {
  if (!c) return DT_E_ARG;
  if (!points || !tuples || !out || (dim != 2 && dim != 3) || n < 1 || m < 0 || kind < 0 || kind > 3)
    return set_err(c, DT_E_ARG, "bad predicate arguments");
  if (m == 0) return DT_OK;
  cudaSetDevice(c->device);
  int rc = 0;
  const double* src = (const double*)stage_in(c, points, sizeof(double) * n * dim, "pred.raw", &rc);
  if (rc) return rc;
  size_t psz = dim == 2 ? sizeof(double2) : sizeof(double4_32a);
  void* P = pool_get(c, "pred.pts", psz * n);
  int* g32 = (int*)pool_get(c, "pred.gid", 4 * n);
  int* flags = (int*)pool_get(c, "pred.flags", 16);
  int8_t* o = (int8_t*)pool_get(c, "pred.out", m);
  int w = kind == 0 ? dim + 1 : (kind == 3 ? 3 : dim + 2);
  const int32_t* tup = (const int32_t*)stage_in(c, tuples, sizeof(int32_t) * m * w, "pred.tup", &rc);
  if (rc) return rc;
  if (!P || !g32 || !flags || !o) return set_err(c, DT_E_NOMEM, "predicate buffers");
  CUDA_OK(cudaMemsetAsync(flags, 0, 16, c->stream));
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  if (gid) {
    const long long* g64 = (const long long*)stage_in(c, gid, 8 * n, "pred.g64", &rc);
    if (rc) return rc;
    k_i64_to_i32<<<g, 256, (++c->launches, 0), c->stream>>>(g64, g32, n);
  } else {
    k_iota<<<g, 256, (++c->launches, 0), c->stream>>>(g32, n, 0);
  }
  unsigned gm = (unsigned)ceil_div<int64_t>(m, 128);
  unsigned long long* ctr = (unsigned long long*)pool_get(c, "pred.ctr", 64);
  if (!ctr) return set_err(c, DT_E_NOMEM, "predicate counters");
  k_read_pred_counters_capi<<<1, 1, (++c->launches, 0), c->stream>>>(ctr + 2, (int*)(ctr + 3));
  if (dim == 2) k_pack_points<2><<<g, 256, (++c->launches, 0), c->stream>>>(src, n, (double2*)P, flags);
  else k_pack_points<3><<<g, 256, (++c->launches, 0), c->stream>>>(src, n, (double4_32a*)P, flags);
  float4* X = nullptr;
  std::vector<unsigned long long> hu;
  rc = fp32_points(c, dim, P, nullptr, n, 1, "pred.xs", &X, &hu);
  if (rc) return rc;
  if (dim == 2)
    k_eval_pred<2><<<gm, 128, (++c->launches, 0), c->stream>>>((const double2*)P, X, g32, kind, tup, m, (int)n, o, flags + 1);
  else
    k_eval_pred<3><<<gm, 128, (++c->launches, 0), c->stream>>>((const double4_32a*)P, X, g32, kind, tup, m, (int)n, o,
                                                               flags + 1);
  k_read_pred_counters_capi<<<1, 1, (++c->launches, 0), c->stream>>>(ctr, (int*)(ctr + 1));
  int h[2];
  unsigned long long hc[4];
  CUDA_OK(cudaMemcpyAsync(h, flags, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaMemcpyAsync(hc, ctr, 32, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  c->stats.exact_calls = (int32_t)std::min<unsigned long long>(hc[0], 0x7fffffffull);
  if (h[1]) return set_err(c, DT_E_ARG, "tuple index out of range");
  if ((int)(hc[1] & 0xffffffff) != (int)(hc[3] & 0xffffffff))
    return set_err(c, DT_E_RANGE, "coordinate range too wide for the exact fallback");
  return copy_out(c, out, o, m);
}

// ---------------------------------------------------------------- asynchronous jobs
// (see include/dt.h)
extern "C" int dt_submit(dt_ctx* c, const double* points, int64_t n, int dim, int k, double sample_frac,
                         uint64_t* job) {
  if (!c) return DT_E_ARG;
  if (!points || !job || (dim != 2 && dim != 3)) return set_err(c, DT_E_ARG, "points and job must be non-null, dim 2 or 3");
  if (n < dim + 1 || n >= (int64_t(1) << 28)) return set_err(c, DT_E_ARG, "n must be in [dim+1, 2^28)");
  if (k < 1 || k > 4096) return set_err(c, DT_E_ARG, "k must be in [1, 4096]");
  if (!(sample_frac >= 0.0 && sample_frac <= 1.0)) return set_err(c, DT_E_ARG, "sample_frac must be in [0, 1]");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  gdt::JobInput in;
  in.n = n;
  in.dim = dim;
  in.k = k;
  in.frac = sample_frac;
  in.pts.resize((size_t)n * dim);
  if (gdt::is_device_ptr(points)) {
    CUDA_OK(cudaMemcpyAsync(in.pts.data(), points, sizeof(double) * (size_t)n * dim, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
  } else {
    memcpy(in.pts.data(), points, sizeof(double) * (size_t)n * dim);
  }
  if (!c->jobs) {
    dt_ctx* w = nullptr;
    int rc = dt_create(&w, c->device, nullptr, &c->cfg);
    if (rc) return set_err(c, rc, "job context");
    c->job_ctx = w;
    c->jobs = new gdt::JobQueue([w](const gdt::JobInput& j) {
      gdt::JobResult r;
      r.rc = dt_triangulate(w, j.pts.data(), j.n, j.dim, j.k, j.frac);
      int64_t m = 0;
      if (!r.rc) r.rc = dt_get_simplices(w, nullptr, 0, &m);
      if (!r.rc) {
        r.rows.resize((size_t)m * (j.dim + 1));
        r.rc = dt_get_simplices(w, r.rows.data(), m, &m);
      }
      if (r.rc) {
        r.rows.clear();
        r.err = dt_last_error(w);
      }
      return r;
    });
  }
  *job = c->jobs->submit(std::move(in));
  return DT_OK;
}

extern "C" int dt_poll(dt_ctx* c, uint64_t job, int* done) {
  if (!c) return DT_E_ARG;
  if (!done) return set_err(c, DT_E_ARG, "done must be non-null");
  int rc = 0;
  const int st = c->jobs ? c->jobs->poll(job, &rc) : -1;
  if (st < 0) return set_err(c, DT_E_ARG, "unknown job");
  *done = st;
  if (st && rc) {
    const gdt::JobResult* r = c->jobs->result(job);
    return set_err(c, rc, r ? r->err : std::string("job failed"));
  }
  return DT_OK;
}

extern "C" int dt_get_job_simplices(dt_ctx* c, uint64_t job, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  const gdt::JobResult* r = c->jobs ? c->jobs->result(job) : nullptr;
  if (!r) return set_err(c, DT_E_ARG, "unknown or unfinished job");
  if (r->rc) return set_err(c, r->rc, r->err);
  const int64_t ints = (int64_t)r->rows.size();
  *count = r->dim ? ints / (r->dim + 1) : 0;
  if (!out) return DT_OK;
  if (capacity < *count) return set_err(c, DT_E_ARG, "capacity too small");
  if (ints) memcpy(out, r->rows.data(), sizeof(int32_t) * (size_t)ints);
  return DT_OK;
}

extern "C" int dt_release_job(dt_ctx* c, uint64_t job) {
  if (!c) return DT_E_ARG;
  const int st = c->jobs ? c->jobs->release(job) : -1;
  if (st < 0) return set_err(c, DT_E_ARG, "unknown job");
  if (st == 0) return set_err(c, DT_E_ARG, "job still queued or running");
  return DT_OK;
}
