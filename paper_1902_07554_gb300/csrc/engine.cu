// engine.cu -- the insertion engine for 2D instances, and the functions the
// two dimensions share (profile records, FP32 point copies, predicate
// counters, the dispatch by dimension).  The 3D instantiation is engine3.cu.
#define GDT_ENGINE_SHARED
#include "engine_core.cuh"

namespace gdt {

int engine_run_3d(dt_ctx* c, EngineRun& run, const void* pts, const int* gid, const int* pinst, int64_t npts,
                  const std::vector<int64_t>& poff, const std::string& tag);
int pred_counters_3d(dt_ctx* c, unsigned long long* calls, int* range, bool reset);

// Exact-stage calls and range errors of both engine units (summed).
int pred_counters_engine(dt_ctx* c, unsigned long long* calls, int* range, bool reset) {
  unsigned long long a = 0, b = 0;
  int ra = 0, rb = 0;
  int rc = pred_counters_local(c, &a, &ra, reset);
  if (rc) return rc;
  rc = pred_counters_3d(c, &b, &rb, reset);
  if (rc) return rc;
  *calls = a + b;
  *range = ra + rb;
  return 0;
}

int stream_setup_2d(dt_ctx* c, StreamState& st) { return stream_setup_t<2>(c, st); }
int stream_admit_2d(dt_ctx* c, StreamState& st, StreamJob& j, const void* P) { return stream_admit_t<2>(c, st, j, P); }
int stream_quantum_2d(dt_ctx* c, StreamState& st, int* yield) { return stream_quantum_t<2>(c, st, yield); }
int stream_extract_2d(dt_ctx* c, StreamState& st, StreamJob& j) { return stream_extract_t<2>(c, st, j); }

void stream_release_graph(StreamState& st) {
  if (st.gx) cudaGraphExecDestroy(st.gx);
  if (st.g) cudaGraphDestroy(st.g);
  st.gx = nullptr;
  st.g = nullptr;
}

int engine_run(dt_ctx* c, EngineRun& run, int dim, const void* pts, const int* gid, const int* pinst,
               int64_t npts, const std::vector<int64_t>& poff, const std::string& tag) {
  if (dim == 2) return engine_run_t<2>(c, run, pts, gid, pinst, npts, poff, tag);
  return engine_run_3d(c, run, pts, gid, pinst, npts, poff, tag);
}

}  // namespace gdt
