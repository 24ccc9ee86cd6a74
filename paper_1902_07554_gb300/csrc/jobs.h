// jobs.h -- the asynchronous job executor behind dt_submit / dt_poll (host
// code only, no CUDA): a first-in-first-out queue drained by one worker thread
// that runs each job through a caller-supplied function.  Job ids start at 1
// and are never reused.  The destructor lets the running job finish, drops
// the jobs still queued and joins the worker.
#pragma once
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

namespace gdt {

struct JobInput {
  std::vector<double> pts;   // n x dim, row-major (the library's own copy)
  int64_t n = 0;
  int dim = 0, k = 1;
  double frac = 0.0;
};

struct JobResult {
  int dim = 0;                 // the job's dimension (set by the queue)
  int rc = 0;                  // DT_OK or the error the job's triangulation returned
  std::vector<int32_t> rows;   // count x (dim + 1), canonical order
  std::string err;             // the error message when rc != 0
};

class JobQueue {
 public:
  using Runner = std::function<JobResult(const JobInput&)>;

  explicit JobQueue(Runner run) : run_(std::move(run)), worker_([this] { loop(); }) {}

  ~JobQueue() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    worker_.join();
  }

  JobQueue(const JobQueue&) = delete;
  JobQueue& operator=(const JobQueue&) = delete;

  uint64_t submit(JobInput in) {
    auto j = std::make_shared<Job>();
    j->in = std::move(in);
    uint64_t id;
    {
      std::lock_guard<std::mutex> lk(mu_);
      id = next_++;
      j->id = id;
      jobs_[id] = j;
      pending_.push_back(j);
    }
    cv_.notify_one();
    return id;
  }

  // -1: unknown id; 0: queued or running; 1: finished (*rc = its result code).
  int poll(uint64_t id, int* rc) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = jobs_.find(id);
    if (it == jobs_.end()) return -1;
    if (!it->second->done) return 0;
    if (rc) *rc = it->second->out.rc;
    return 1;
  }

  // The finished job's result, or nullptr (unknown id or not finished).  The
  // pointer stays valid until the job is released or the queue destroyed.
  const JobResult* result(uint64_t id) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = jobs_.find(id);
    if (it == jobs_.end() || !it->second->done) return nullptr;
    return &it->second->out;
  }

  // Frees a finished job: 1 on success, 0 while it is queued or running, -1 unknown.
  int release(uint64_t id) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = jobs_.find(id);
    if (it == jobs_.end()) return -1;
    if (!it->second->done) return 0;
    jobs_.erase(it);
    return 1;
  }

  size_t queued() {
    std::lock_guard<std::mutex> lk(mu_);
    return pending_.size();
  }

 private:
  struct Job {
    uint64_t id = 0;
    JobInput in;
    JobResult out;
    bool done = false;
  };

  void loop() {
    for (;;) {
      std::shared_ptr<Job> j;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [this] { return stop_ || !pending_.empty(); });
        if (stop_) return;
        j = pending_.front();
        pending_.pop_front();
      }
      JobResult r = run_(j->in);
      {
        std::lock_guard<std::mutex> lk(mu_);
        j->out = std::move(r);
        j->out.dim = j->in.dim;
        j->in.pts = std::vector<double>();   // the input copy is no longer needed
        j->done = true;
      }
    }
  }

  Runner run_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::shared_ptr<Job>> pending_;
  std::map<uint64_t, std::shared_ptr<Job>> jobs_;
  uint64_t next_ = 1;
  bool stop_ = false;
  std::thread worker_;   // last: starts after every other member is ready
};

}  // namespace gdt
