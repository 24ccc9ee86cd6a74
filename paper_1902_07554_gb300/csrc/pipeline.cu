// pipeline.cu -- Alg. 1 driver.
#include "pipeline.cuh"

namespace gdt {

int collect_finite(dt_ctx* c, const EngineRun& run, const int* gid, const unsigned char* drop, int4** rows,
                   int64_t* nrows, const std::string& tag);

// Base case of Alg. 1 (n < N, or k = 1): one triangulation of all points.
static int run_direct(dt_ctx* c, const void* P, int64_t n, int dim) {
  cudaStream_t s = c->stream;
  int* gid = (int*)pool_get(c, "pl.gid", 4 * n);
  int* pinst = (int*)pool_get(c, "pl.pinst", 4 * n);
  if (!gid || !pinst) return set_err(c, DT_E_NOMEM, "pipeline buffers");
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  k_iota<<<g, 256, 0, s>>>(gid, n, 0);
  CUDA_OK(cudaMemsetAsync(pinst, 0, 4 * n, s));
  std::vector<int64_t> poff = {0, n};
  int rc = engine_run(c, c->run_parts, dim, P, gid, pinst, n, poff, "parts");
  if (rc) return rc;
  if (c->run_parts.h_status[0] == 1) return set_err(c, DT_E_DEGENERATE, "all points are collinear/coplanar");
  if (c->run_parts.h_status[0] != 0) return set_err(c, DT_E_ARG, "too few points");
  c->stats.rounds_max = c->run_parts.rounds;
  int4* rows; int64_t nrows;
  rc = collect_finite(c, c->run_parts, gid, nullptr, &rows, &nrows, "final");
  if (rc) return rc;
  rc = canonicalize_rows(c, dim, rows, nrows, n, &c->out, &c->nout, "final");
  if (rc) return rc;
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

int run_pipeline(dt_ctx* c, const double* points, int64_t n, int dim, int k, double frac) {
  void* P = nullptr;
  int rc = stage_points(c, points, n, dim, &P);
  if (rc) return rc;
  (void)frac;
  if (k == 1 || n / k < c->cfg.base_threshold) return run_direct(c, P, n, dim);
  return set_err(c, DT_E_ARG, "divide step not built yet");
}

}  // namespace gdt

extern "C" int dt_label_points(dt_ctx* c, const double*, int64_t, int, const double*, const int64_t*,
                               const int32_t*, int64_t, int32_t*) {
  return c ? gdt::set_err(c, DT_E_ARG, "not built yet") : DT_E_ARG;
}
extern "C" int dt_partition_graph(dt_ctx* c, const double*, int64_t, int, const int32_t*, const int64_t*, int64_t,
                                  int, double, int, int32_t*) {
  return c ? gdt::set_err(c, DT_E_ARG, "not built yet") : DT_E_ARG;
}
