// stream.cuh -- continuous batching of triangulation jobs in one resident
// insertion engine (stream_api.cu, engine_core.cuh).
//
// A stream owns device buffers for `capacity` points and their simplex
// arenas.  Jobs are queued from any host thread; between insertion rounds the
// engine yields to the host, which admits queued jobs into free ranges of the
// resident buffers (each job one engine instance with its own activation
// schedule), and extracts the jobs whose points are all inserted.  Jobs of
// different sizes therefore share every round's launches, and a job that
// arrives while others run starts at the next round boundary instead of
// waiting for them to finish.
#pragma once
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "ctx.cuh"

namespace gdt {

constexpr int STREAM_NLEV = 96;        // activation levels (the engine's NLEV)
constexpr int STREAM_MAX_JOBS = 1024;  // instances resident at once (one CTA plans them)

// Per resident instance (device).
struct SlotState {
  int status;                    // 0 free, 1 running, 2 finished (awaiting extraction)
  int next_level;                // next activation level (-1: none left)
  int last_batch;                // active count right after the last activation
  int nact;                      // active points
  int loff[STREAM_NLEV + 1];     // absolute offsets of the instance's level lists
};

struct StreamJob {
  uint64_t id = 0;
  std::vector<double> pts;       // host copy until admitted
  int64_t n = 0;
  int slot = -1;
  int64_t p0 = -1;               // first point of its range in the resident buffers
  int status = 0;                // 0 queued, 1 running, 2 done; negative: DT_E_* error
  std::vector<int32_t> rows;     // result: sorted rows of dim+1 input indices
};

struct StreamState {
  int dim = 3, max_jobs = 0;
  int64_t cap = 0;               // points
  int64_t arena_factor = 36;     // simplex slots per point
  int64_t cap_cand = 0;          // nominees per round
  int capC = 0, capB = 0;        // cavity list capacities per nominee
  size_t bytes = 0;              // device bytes held by the stream
  // device buffers
  void* pts = nullptr;
  int *gid = nullptr, *pinst = nullptr, *loc = nullptr, *level = nullptr, *lrank = nullptr, *lsize = nullptr;
  unsigned char* state = nullptr;
  float4* xs = nullptr;
  int *llist = nullptr, *act0 = nullptr, *act1 = nullptr, *walk = nullptr, *nom = nullptr;
  int4 *tv = nullptr, *tn = nullptr;
  unsigned long long *claimA = nullptr, *claimC = nullptr;
  int *toff = nullptr, *tend = nullptr, *tcount = nullptr, *inst_status = nullptr;
  double *xo = nullptr, *glo = nullptr;
  int *gdim = nullptr, *hint = nullptr, *hint2 = nullptr;
  SlotState* ss = nullptr;
  int *seg = nullptr, *kept = nullptr, *cnt = nullptr;
  void* ctl = nullptr;
  CandScratch S;
  int* admit_host = nullptr;     // mapped pinned flag: jobs are waiting (read by the round loop)
  int* admit_dev = nullptr;
  std::vector<void*> owned;      // every cudaMalloc of the stream
  // the round graph (built once per scratch size)
  cudaGraph_t g = nullptr;
  cudaGraphExec_t gx = nullptr;
  bool graph_pdl = true;
  dt_config graph_cfg;           // the context's configuration the graph was built with
  unsigned round = 0;
  long long quanta = 0, rounds_run = 0;
  // host bookkeeping (mu guards queue, jobs and next_id: dt_stream_submit may
  // run on another thread than dt_stream_run)
  std::mutex mu;
  std::deque<uint64_t> queue;
  std::map<uint64_t, StreamJob> jobs;
  std::vector<uint64_t> slot_job;                        // job per instance slot (0: free)
  std::vector<std::pair<int64_t, int64_t>> free_ranges;  // free [begin, end) of the point index space
  uint64_t next_id = 1;
};

// Per dimension (engine.cu: 2D, engine3.cu: 3D).
int stream_setup_2d(dt_ctx* c, StreamState& st);
int stream_setup_3d(dt_ctx* c, StreamState& st);
int stream_admit_2d(dt_ctx* c, StreamState& st, StreamJob& j, const void* P);
int stream_admit_3d(dt_ctx* c, StreamState& st, StreamJob& j, const void* P);
int stream_quantum_2d(dt_ctx* c, StreamState& st, int* yield);
int stream_quantum_3d(dt_ctx* c, StreamState& st, int* yield);
int stream_extract_2d(dt_ctx* c, StreamState& st, StreamJob& j);
int stream_extract_3d(dt_ctx* c, StreamState& st, StreamJob& j);
void stream_release_graph(StreamState& st);

}  // namespace gdt
