// stream_api.cu -- C ABI of the continuous-batching stream (stream.cuh):
// open, submit (any thread), run, job status, fetch, release, info, close.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ctx.cuh"
#include "pipeline.cuh"
#include "stream.cuh"

using namespace gdt;

namespace {

// First fit of `len` points in the free ranges; -1 when nothing fits.
int64_t take_range(StreamState& st, int64_t len) {
  for (size_t i = 0; i < st.free_ranges.size(); i++) {
    auto& r = st.free_ranges[i];
    if (r.second - r.first >= len) {
      const int64_t p0 = r.first;
      r.first += len;
      if (r.first == r.second) st.free_ranges.erase(st.free_ranges.begin() + i);
      return p0;
    }
  }
  return -1;
}

// Returns [p0, p0 + len) to the free ranges, merging neighbours.
void give_range(StreamState& st, int64_t p0, int64_t len) {
  st.free_ranges.push_back({p0, p0 + len});
  std::sort(st.free_ranges.begin(), st.free_ranges.end());
  std::vector<std::pair<int64_t, int64_t>> m;
  for (auto& r : st.free_ranges) {
    if (!m.empty() && m.back().second >= r.first) m.back().second = std::max(m.back().second, r.second);
    else m.push_back(r);
  }
  st.free_ranges.swap(m);
}

// Points a job of n points occupies: n, plus enough that its simplex arena
// ([A p0, A (p0 + n) + 32)) ends before the next range's arena starts.
int64_t range_len(const StreamState& st, int64_t n) { return n + 1 + (32 + st.arena_factor - 1) / st.arena_factor; }

int free_slot(const StreamState& st) {
  for (int i = 0; i < st.max_jobs; i++)
    if (st.slot_job[i] == 0) return i;
  return -1;
}

void stream_free(dt_ctx* c) {
  StreamState* st = c->stream_state;
  if (!st) return;
  cudaStreamSynchronize(c->stream);
  stream_release_graph(*st);
  for (void* p : st->owned) cudaFree(p);
  if (st->admit_host) cudaFreeHost(st->admit_host);
  delete st;
  c->stream_state = nullptr;
}

// Ends every running job with `code` and returns the stream to empty.
int stream_fail_running(dt_ctx* c, int code) {
  StreamState& st = *c->stream_state;
  {
    std::lock_guard<std::mutex> lk(st.mu);
    for (auto& kv : st.jobs)   // running, or admitted but not yet set up
      if (kv.second.status == 1 || (kv.second.status == 0 && kv.second.slot >= 0)) kv.second.status = code;
    st.slot_job.assign(st.max_jobs, 0);
    st.free_ranges.assign(1, {0, st.cap});
  }
  cudaGetLastError();
  stream_release_graph(st);
  return st.dim == 2 ? stream_setup_2d(c, st) : stream_setup_3d(c, st);
}

}  // namespace

void dt_stream_cleanup(dt_ctx* c) { stream_free(c); }

extern "C" int dt_stream_open(dt_ctx* c, int dim, int64_t capacity, int max_jobs) {
  if (!c) return DT_E_ARG;
  c->err.clear();
  if (c->stream_state) return set_err(c, DT_E_ARG, "a stream is already open on this context");
  if ((dim != 2 && dim != 3) || capacity < 16 || capacity >= (int64_t(1) << 26) || max_jobs < 1 ||
      max_jobs > STREAM_MAX_JOBS)
    return set_err(c, DT_E_ARG, "stream: dim 2 or 3, 16 <= capacity < 2^26, 1 <= max_jobs <= 1024");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  StreamState* st = new StreamState();
  st->dim = dim;
  st->cap = capacity;
  st->max_jobs = max_jobs;
  st->arena_factor = c->cfg.arena_factor > 0 ? c->cfg.arena_factor : (dim == 2 ? 8 : 36);
  st->cap_cand = std::min<int64_t>(capacity, int64_t(1) << 20);
  st->capC = dim == 2 ? 32 : 96;
  st->capB = dim == 2 ? 48 : 192;
  if (st->arena_factor * capacity + 64 >= (int64_t(1) << 31)) {
    delete st;
    return set_err(c, DT_E_ARG, "stream: capacity x arena factor must stay below 2^31 simplices");
  }
  st->slot_job.assign(max_jobs, 0);
  st->free_ranges.assign(1, {0, capacity});
  if (cudaHostAlloc((void**)&st->admit_host, 16, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&st->admit_dev, st->admit_host, 0) != cudaSuccess) {
    cudaGetLastError();
    if (st->admit_host) cudaFreeHost(st->admit_host);
    delete st;
    return set_err(c, DT_E_NOMEM, "stream: mapped flag");
  }
  *st->admit_host = 0;
  c->stream_state = st;
  int rc = dim == 2 ? stream_setup_2d(c, *st) : stream_setup_3d(c, *st);
  if (rc) { std::string e = c->err; stream_free(c); return set_err(c, rc, e); }
  return DT_OK;
}

extern "C" int dt_stream_submit(dt_ctx* c, const double* points, int64_t n, uint64_t* job) {
  if (!c || !job) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st || !points || n < 1) return DT_E_ARG;
  if (range_len(*st, n) > st->cap) return DT_E_NOMEM;   // larger than the whole stream
  StreamJob j;
  j.n = n;
  j.pts.assign(points, points + n * st->dim);
  std::lock_guard<std::mutex> lk(st->mu);
  j.id = st->next_id++;
  *job = j.id;
  st->queue.push_back(j.id);
  st->jobs.emplace(j.id, std::move(j));
  *st->admit_host = 1;                     // the running round loop yields at its next boundary
  return DT_OK;
}

extern "C" int dt_stream_run(dt_ctx* c, int quanta, int* pending) {
  if (!c) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st) return set_err(c, DT_E_ARG, "no stream open");
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return set_err(c, DT_E_CUDA, "cudaSetDevice"); }
  c->err.clear();
  const int dim = st->dim;
  int rc = 0;
  for (int q = 0; q < std::max(1, quanta); q++) {
    // admission: queued jobs, in arrival order, into free ranges and slots;
    // a job that does not fit yet is passed over by smaller ones behind it
    std::vector<uint64_t> admit;
    {
      std::lock_guard<std::mutex> lk(st->mu);
      *st->admit_host = 0;
      for (auto it = st->queue.begin(); it != st->queue.end();) {
        StreamJob& j = st->jobs[*it];
        const int slot = free_slot(*st);
        if (slot < 0) break;
        const int64_t p0 = take_range(*st, range_len(*st, j.n));
        if (p0 < 0) { ++it; continue; }
        j.slot = slot;
        j.p0 = p0;
        st->slot_job[slot] = j.id;
        admit.push_back(j.id);
        it = st->queue.erase(it);
      }
    }
    for (uint64_t id : admit) {
      StreamJob* j;
      {
        std::lock_guard<std::mutex> lk(st->mu);
        j = &st->jobs[id];
      }
      void* P = nullptr;
      int arc = stage_points(c, j->pts.data(), j->n, dim, &P, "stream.in");
      if (arc == 0) arc = dim == 2 ? stream_admit_2d(c, *st, *j, P) : stream_admit_3d(c, *st, *j, P);
      if (arc == DT_E_CUDA || arc == DT_E_NOMEM || arc == DT_E_INTERNAL) {
        rc = arc;
        break;
      }
      std::lock_guard<std::mutex> lk(st->mu);
      if (arc) j->status = arc;                 // a bad input (duplicate, non-finite): that job alone fails
      if (j->status != 1) {                     // failed, or too small / flat to triangulate
        if (j->status == 0) j->status = arc ? arc : DT_E_ARG;
        st->slot_job[j->slot] = 0;
        give_range(*st, j->p0, range_len(*st, j->n));
      }
      std::vector<double>().swap(j->pts);
    }
    if (rc) break;
    int running = 0;
    for (int i = 0; i < st->max_jobs; i++) running += st->slot_job[i] != 0;
    if (!running) break;
    int yield = 0;
    rc = dim == 2 ? stream_quantum_2d(c, *st, &yield) : stream_quantum_3d(c, *st, &yield);
    if (rc) break;
    // finished instances: extract and free
    std::vector<SlotState> hs(st->max_jobs);
    CUDA_OK(cudaMemcpyAsync(hs.data(), st->ss, sizeof(SlotState) * st->max_jobs, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < st->max_jobs && !rc; i++) {
      if (hs[i].status != 2 || !st->slot_job[i]) continue;
      StreamJob* j;
      {
        std::lock_guard<std::mutex> lk(st->mu);
        j = &st->jobs[st->slot_job[i]];
      }
      rc = dim == 2 ? stream_extract_2d(c, *st, *j) : stream_extract_3d(c, *st, *j);
      if (rc) break;
      SlotState z;
      memset(&z, 0, sizeof(z));
      CUDA_OK(cudaMemcpyAsync(st->ss + i, &z, sizeof(SlotState), cudaMemcpyHostToDevice, c->stream));
      CUDA_OK(cudaStreamSynchronize(c->stream));
      std::lock_guard<std::mutex> lk(st->mu);
      j->status = 2;
      st->slot_job[i] = 0;
      give_range(*st, j->p0, range_len(*st, j->n));
    }
    if (rc) break;
  }
  if (rc) {
    // the engine state is lost: every running job fails, the stream starts empty
    const std::string e = c->err;
    stream_fail_running(c, rc);
    set_err(c, rc, e);
  }
  if (pending) {
    std::lock_guard<std::mutex> lk(st->mu);
    int p = (int)st->queue.size();
    for (int i = 0; i < st->max_jobs; i++) p += st->slot_job[i] != 0;
    *pending = p;
  }
  return rc;
}

extern "C" int dt_stream_job(dt_ctx* c, uint64_t job, int* status, int64_t* count) {
  if (!c || !status) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st) return DT_E_ARG;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->jobs.find(job);
  if (it == st->jobs.end()) return DT_E_ARG;
  *status = it->second.status;
  if (count) *count = it->second.status == 2 ? (int64_t)(it->second.rows.size() / (st->dim + 1)) : 0;
  return DT_OK;
}

extern "C" int dt_stream_fetch(dt_ctx* c, uint64_t job, int32_t* out, int64_t capacity, int64_t* count) {
  if (!c || !count) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st) return DT_E_ARG;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->jobs.find(job);
  if (it == st->jobs.end()) return DT_E_ARG;
  if (it->second.status < 0) return it->second.status;
  if (it->second.status != 2) return DT_E_ARG;
  const int64_t rows = (int64_t)(it->second.rows.size() / (st->dim + 1));
  *count = rows;
  if (!out) return DT_OK;
  if (capacity < rows) return DT_E_ARG;
  if (rows) memcpy(out, it->second.rows.data(), 4 * (size_t)rows * (st->dim + 1));
  return DT_OK;
}

extern "C" int dt_stream_release(dt_ctx* c, uint64_t job) {
  if (!c) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st) return DT_E_ARG;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->jobs.find(job);
  if (it == st->jobs.end() || it->second.status == 0 || it->second.status == 1) return DT_E_ARG;
  st->jobs.erase(it);
  return DT_OK;
}

extern "C" int dt_stream_get_info(dt_ctx* c, dt_stream_info* out) {
  if (!c || !out) return DT_E_ARG;
  StreamState* st = c->stream_state;
  if (!st) return DT_E_ARG;
  std::lock_guard<std::mutex> lk(st->mu);
  memset(out, 0, sizeof(*out));
  out->capacity = st->cap;
  out->device_bytes = (int64_t)st->bytes;
  int64_t fr = 0;
  for (auto& r : st->free_ranges) fr += r.second - r.first;
  out->free_points = fr;
  out->queued = (int32_t)st->queue.size();
  for (int i = 0; i < st->max_jobs; i++) out->running += st->slot_job[i] != 0;
  out->quanta = st->quanta;
  out->rounds = st->rounds_run;
  out->launches = c->launches;
  return DT_OK;
}

extern "C" int dt_stream_close(dt_ctx* c) {
  if (!c) return DT_E_ARG;
  if (!c->stream_state) return DT_E_ARG;
  stream_free(c);
  return DT_OK;
}
