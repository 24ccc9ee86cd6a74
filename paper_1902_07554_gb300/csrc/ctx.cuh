// ctx.cuh -- the library context: stream, configuration, buffer pool, results.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "engine.cuh"

namespace gdt { class JobQueue; struct StreamState; }

struct dt_ctx {
  int device = 0;
  int sms = 152;                         // streaming multiprocessors of the device (grid sizes)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;     // capture stream of the insertion-round graph
  cudaStream_t aux_stream = nullptr;     // second stream: the label walk beside the partitioner
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
  bool pdl_ok = true;                    // programmatic launches accepted in the round graph
  // instantiated round graphs, keyed by the bytes of every launch parameter
  // captured in them: a run whose buffers, sizes and grids equal an earlier
  // run's relaunches that run's graph instead of capturing a new one
  struct RoundGraph { std::string key; cudaGraph_t g = nullptr; cudaGraphExec_t gx = nullptr; };
  std::vector<RoundGraph> round_graphs;
  long long graphs_built = 0, graphs_reused = 0;
  bool own_stream = false;
  dt_config cfg;
  std::string err;
  // named device buffers, grown on demand and reused across calls
  struct Buf { void* p = nullptr; size_t cap = 0; };
  std::map<std::string, Buf> pool;
  gdt::DevStatus* status = nullptr;      // device status word
  gdt::DevStatus* status_host = nullptr; // pinned mirror
  int* counters_host = nullptr;          // pinned scratch for small read-backs (64 ints)
  cudaEvent_t ev[16];
  cudaEvent_t pev[16];                   // per-kernel profiling events
  std::vector<cudaEvent_t> evpool;       // profile mode: events around every engine launch
  long long launches = 0;                // kernels launched by this context (all calls)
  // per-kernel profile of the last call (profile mode)
  struct KProf { const char* name; long long launches; double ms, bytes, flops; };
  std::vector<KProf> kprof;
  // last result
  int dim = 0;
  int64_t n = 0;
  int32_t* out = nullptr;                // device, canonical simplices
  int64_t nout = 0;
  dt_stats stats;
  std::vector<int32_t> h_labels_dummy;
  // divide-step results of the last call (device)
  int32_t* labels = nullptr;             // n
  int32_t* sample = nullptr;             // eta (global ids, ascending)
  int32_t* sample_block = nullptr;       // eta
  int64_t eta = 0;
  int32_t* border_vtx = nullptr;         // |V_B| global ids, ascending
  int64_t n_border = 0;
  gdt::EngineRun run_sample, run_parts, run_border;
  // provenance of the output rows (neighbourhood update) and its result
  gdt::LinkSources links;
  bool links_ok = false;
  bool rows_only = false;                // a single triangulation without link sources (recursive bisection)
  int32_t* nbr = nullptr;                // device, (dim+1) per output row
  bool nbr_ok = false;
  // batched call: per-instance row offsets (count+1) and status
  std::vector<int64_t> batch_offsets;
  std::vector<int> batch_status;
  int batch_count = 0;
  // asynchronous jobs (dt_submit): a second context on the same device and its worker
  dt_ctx* job_ctx = nullptr;
  gdt::JobQueue* jobs = nullptr;
  // continuous-batching stream (dt_stream_open), owned by the context
  gdt::StreamState* stream_state = nullptr;
};

// Frees the context's stream, if one is open (stream_api.cu).
void dt_stream_cleanup(dt_ctx* c);

namespace gdt {

// Returns a device buffer of at least `bytes` bytes under `name`; contents
// are undefined.  Returns nullptr on allocation failure.
void* pool_get(dt_ctx* c, const std::string& name, size_t bytes);
void pool_free_all(dt_ctx* c);

int set_err(dt_ctx* c, int code, const std::string& msg);

// Checks the device status word (synchronises the stream).  Returns 0 or a
// DT_E_* code with the context's error message set.
int check_status(dt_ctx* c, const char* where);

// Generic device helpers (defined in util.cu).
int exclusive_scan_i32(dt_ctx* c, const int* in, int* out, int64_t n, int* total_host);
int exclusive_scan_i64(dt_ctx* c, const long long* in, long long* out, int64_t n);

// Accumulates a per-kernel profile entry (profile mode).
void prof_add(dt_ctx* c, const char* name, double ms, double bytes, double flops);

// FP32 copies of the points for the first predicate stage (engine.cu).
int fp32_points(dt_ctx* c, int dim, const void* pts, const int* pinst, int64_t npts, int ninst, const std::string& tag,
                float4** xs_out, std::vector<unsigned long long>* hu_out, const double** xo_out = nullptr);

// Engine (engine.cu).
int engine_run(dt_ctx* c, EngineRun& run, int dim, const void* pts, const int* gid, const int* pinst,
               int64_t npts, const std::vector<int64_t>& poff, const std::string& tag);

// Canonicalisation of the finite live simplices of `run` whose instances are
// selected: output rows (sorted gid tuples, lexicographic) into *out.
// keep (optional, per slot) filters simplices.
int canonicalize_rows(dt_ctx* c, int dim, const int4* rows, int64_t nrows, int64_t nbuckets,
                      int32_t** out, int64_t* nout, const std::string& tag, const int* src = nullptr,
                      int** src_out = nullptr);
int collect_finite(dt_ctx* c, const EngineRun& run, const int* gid, const unsigned char* flag, int mode,
                   int4** rows, int64_t* nrows, const std::string& tag, int** src = nullptr, int src_base = 0);

}  // namespace gdt
