// Host-only checks of the asynchronous job executor (csrc/jobs.h), compiled
// with the host C++ compiler by tests/test_jobs_host.py.  Exit status 0 and
// "ok" on success; the first failed check prints its line and exits 1.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "jobs.h"

#define CHECK(x)                                                  \
  do {                                                            \
    if (!(x)) {                                                   \
      std::printf("check failed at line %d: %s\n", __LINE__, #x); \
      std::exit(1);                                               \
    }                                                             \
  } while (0)

using gdt::JobInput;
using gdt::JobQueue;
using gdt::JobResult;

static void sleep_ms(int ms) { std::this_thread::sleep_for(std::chrono::milliseconds(ms)); }

// Polls until every id has finished (at most ~10 s).
static void wait_all(JobQueue& q, const std::vector<uint64_t>& ids) {
  for (int it = 0; it < 10000; it++) {
    bool all = true;
    for (uint64_t id : ids) {
      int rc = 0;
      all &= q.poll(id, &rc) == 1;
    }
    if (all) return;
    sleep_ms(1);
  }
  CHECK(!"jobs did not finish");
}

static JobInput job(int tag, int dim = 2) {
  JobInput in;
  in.n = tag;
  in.dim = dim;
  in.pts.assign(4, (double)tag);
  return in;
}

int main() {
  // 1. first in, first out; results, dimensions and error codes travel with their job
  {
    std::mutex mu;
    std::vector<int> order;
    JobQueue q([&](const JobInput& in) {
      {
        std::lock_guard<std::mutex> lk(mu);
        order.push_back((int)in.n);
      }
      JobResult r;
      CHECK(in.pts.size() == 4 && in.pts[0] == (double)in.n);   // the job sees its own input copy
      if (in.n % 7 == 0) {
        r.rc = -2;
        r.err = "duplicate";
      } else {
        r.rows = {(int32_t)in.n, (int32_t)in.n + 1, (int32_t)in.n + 2};
      }
      return r;
    });
    std::vector<uint64_t> ids;
    for (int i = 1; i <= 50; i++) ids.push_back(q.submit(job(i, i % 2 ? 2 : 3)));
    for (size_t i = 0; i < ids.size(); i++) CHECK(ids[i] == i + 1);   // ids start at 1, in order
    wait_all(q, ids);
    CHECK(order.size() == 50);
    for (int i = 0; i < 50; i++) CHECK(order[i] == i + 1);
    for (int i = 1; i <= 50; i++) {
      int rc = 123;
      CHECK(q.poll(ids[i - 1], &rc) == 1);
      const JobResult* r = q.result(ids[i - 1]);
      CHECK(r != nullptr && r->dim == (i % 2 ? 2 : 3));
      if (i % 7 == 0) {
        CHECK(rc == -2 && r->rc == -2 && r->err == "duplicate" && r->rows.empty());
      } else {
        CHECK(rc == 0 && r->rows.size() == 3 && r->rows[0] == i);
      }
    }
    // unknown ids; release frees a finished job once
    int rc = 0;
    CHECK(q.poll(0, &rc) == -1 && q.poll(51, &rc) == -1);
    CHECK(q.result(51) == nullptr);
    CHECK(q.release(ids[3]) == 1);
    CHECK(q.release(ids[3]) == -1 && q.poll(ids[3], &rc) == -1 && q.result(ids[3]) == nullptr);
    CHECK(q.submit(job(60)) == 51);   // ids are never reused
  }
  // 2. a queued or running job cannot be released; its result appears only when done
  {
    std::atomic<bool> go{false};
    JobQueue q([&](const JobInput& in) {
      for (int it = 0; it < 5000 && !go.load(); it++) sleep_ms(1);
      JobResult r;
      r.rows = {(int32_t)in.n};
      return r;
    });
    uint64_t a = q.submit(job(1)), b = q.submit(job(2));
    int rc = 0;
    CHECK(q.poll(a, &rc) == 0 && q.poll(b, &rc) == 0);
    CHECK(q.result(a) == nullptr && q.release(a) == 0 && q.release(b) == 0);
    go = true;
    wait_all(q, {a, b});
    CHECK(q.result(b)->rows[0] == 2 && q.release(a) == 1 && q.release(b) == 1);
    CHECK(q.queued() == 0);
  }
  // 3. destruction lets the running job finish and drops the queued ones
  {
    std::atomic<int> ran{0};
    auto t0 = std::chrono::steady_clock::now();
    {
      JobQueue q([&](const JobInput&) {
        sleep_ms(20);
        ran++;
        return JobResult();
      });
      for (int i = 0; i < 20; i++) q.submit(job(i + 1));
      sleep_ms(5);
    }
    const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    CHECK(ran >= 0 && ran <= 2 && s < 2.0);
  }
  // 4. submissions from several threads at once: every id distinct, every job run once
  {
    std::atomic<int> ran{0};
    JobQueue q([&](const JobInput&) {
      ran++;
      return JobResult();
    });
    std::mutex mu;
    std::set<uint64_t> seen;
    std::vector<uint64_t> all;
    std::vector<std::thread> th;
    for (int t = 0; t < 4; t++)
      th.emplace_back([&, t] {
        for (int i = 0; i < 100; i++) {
          uint64_t id = q.submit(job(t * 100 + i + 1));
          std::lock_guard<std::mutex> lk(mu);
          seen.insert(id);
          all.push_back(id);
        }
      });
    for (auto& x : th) x.join();
    CHECK(seen.size() == 400 && *seen.begin() == 1 && *seen.rbegin() == 400);
    wait_all(q, all);
    CHECK(ran == 400);
  }
  std::printf("ok\n");
  return 0;
}
