// engine3.cu -- the insertion engine for 3D instances (engine_core.cuh
// instantiated with D = 3 in a translation unit of its own).
#include "engine_core.cuh"

namespace gdt {

int engine_run_3d(dt_ctx* c, EngineRun& run, const void* pts, const int* gid, const int* pinst, int64_t npts,
                  const std::vector<int64_t>& poff, const std::string& tag) {
  return engine_run_t<3>(c, run, pts, gid, pinst, npts, poff, tag);
}

int stream_setup_3d(dt_ctx* c, StreamState& st) { return stream_setup_t<3>(c, st); }
int stream_admit_3d(dt_ctx* c, StreamState& st, StreamJob& j, const void* P) { return stream_admit_t<3>(c, st, j, P); }
int stream_quantum_3d(dt_ctx* c, StreamState& st, int* yield) { return stream_quantum_t<3>(c, st, yield); }
int stream_extract_3d(dt_ctx* c, StreamState& st, StreamJob& j) { return stream_extract_t<3>(c, st, j); }

int pred_counters_3d(dt_ctx* c, unsigned long long* calls, int* range, bool reset) {
  return pred_counters_local(c, calls, range, reset);
}

}  // namespace gdt
