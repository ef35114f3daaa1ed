// Serving: continuous batching of suffix-array builds on one GPU.
//
// `slots` worker threads, each with its own non-blocking CUDA stream, take
// requests from one FIFO queue. The head request starts as soon as a worker
// is free and its device footprint fits in the remaining byte budget; it
// then holds its text, SA and workspace on the device until it completes
// (sa_build_host: copy in, all doubling rounds, copy out). Requests that
// arrive while others run are admitted as slots and budget free up, and the
// builds of different workers overlap on the device. Strict FIFO admission:
// the head waits for memory rather than being overtaken, so no request
// starves. A request is forgotten once its result has been handed out
// (sa_server_wait returned, or sa_server_poll reported it done), so a
// long-running server holds only queued, running and uncollected requests.
//
// Each worker holds one stream per priority level, and a request runs on
// the stream of its size class (sa_server_config.size_priority): the block
// scheduler starts a small request's blocks ahead of the waiting blocks of
// large builds in flight, so small requests are not queued behind whole
// kernels of large ones.
//
// The paper has no serving layer; this is the runtime around its method.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbsa.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr uint64_t DEFAULT_BUDGET = 100ull * 1000 * 1000 * 1000;  // 100 GB
constexpr uint32_t DEFAULT_SLOTS = 8;
constexpr uint32_t MAX_SLOTS = 64;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Size classes of the stream priorities: up to 256 KiB, 2 MiB, 16 MiB, more.
constexpr int PRIORITY_CLASSES = 4;
int size_class(uint64_t n) {
  if (n <= (256ull << 10)) return 0;
  if (n <= (2ull << 20)) return 1;
  if (n <= (16ull << 20)) return 2;
  return 3;
}
// Stream priority of size class c in the device's range [least, greatest]
// (greatest is the numerically lowest, the highest priority).
int class_priority(int c, int least, int greatest) {
  const int p = greatest + c;
  return p < least ? p : least;
}

struct Request {
  uint64_t ticket = 0;
  const uint8_t *text = nullptr;
  uint64_t n = 0;
  uint32_t *sa = nullptr;
  size_t footprint = 0;
  sa_request_info info{};
  bool done = false;
  uint32_t waiters = 0;   // threads blocked in sa_server_wait on this request
  bool collected = false; // result handed out; no longer in `requests`
};

}  // namespace

struct sa_server {
  sa_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, Request *> requests;  // not yet collected
  uint64_t next_ticket = 1;
  uint64_t in_use = 0;
  uint32_t in_flight = 0;
  sa_server_stats stats{};
  bool stop = false;
  std::vector<std::thread> workers;

  // Hands the finished request r over: it leaves the table, and the last
  // thread that still refers to it frees it. Called with `mu` held.
  void collect(Request *r) {
    if (!r->collected) {
      requests.erase(r->ticket);
      r->collected = true;
      stats.tracked = (uint32_t)requests.size();
    }
    if (r->waiters == 0) delete r;
  }

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  int prio_least = 0, prio_greatest = -5;  // the simulate-mode range

  int priority_of(int c) const {
    return cfg.size_priority == 0 ? class_priority(c, prio_least, prio_greatest) : 0;
  }

  void worker(uint32_t slot) {
    cudaStream_t streams[PRIORITY_CLASSES] = {};
    if (!cfg.simulate) {
      cudaSetDevice(device);
      for (int c = 0; c < PRIORITY_CLASSES; ++c)
        cudaStreamCreateWithPriority(&streams[c], cudaStreamNonBlocking, priority_of(c));
    }
    for (;;) {
      Request *r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop && queue.empty()) return true;
          return !queue.empty() && in_use + queue.front()->footprint <= cfg.budget_bytes;
        });
        if (queue.empty()) break;  // stopping and drained
        r = queue.front();
        queue.pop_front();
        in_use += r->footprint;
        ++in_flight;
        stats.bytes_in_use = in_use;
        if (in_use > stats.peak_bytes_in_use) stats.peak_bytes_in_use = in_use;
        if (in_flight > stats.peak_in_flight) stats.peak_in_flight = in_flight;
        stats.queued = (uint32_t)queue.size();
        r->info.start_s = now();
        r->info.slot = slot;
        r->info.priority = priority_of(size_class(r->n));
      }
      sa_status status = SA_OK;
      if (cfg.simulate) {
        const double ns = (double)r->n * cfg.simulate_ns_per_byte;
        std::this_thread::sleep_for(std::chrono::nanoseconds((int64_t)ns));
      } else {
        status = sa_build_host(r->text, r->n, r->sa, (gbsa_stream_t)streams[size_class(r->n)]);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= r->footprint;
        --in_flight;
        stats.bytes_in_use = in_use;
        ++stats.completed;
        r->info.status = status;
        r->info.done_s = now();
        r->done = true;
      }
      cv_done.notify_all();
      cv_work.notify_all();  // memory and a slot were freed
    }
    for (cudaStream_t st : streams)
      if (st) cudaStreamDestroy(st);
  }
};

GBSA_API size_t sa_request_footprint(uint64_t n) {
  return align256(n) + align256(n * 4) + sa_workspace_bytes(n);
}

GBSA_API sa_status sa_server_create(const sa_server_config *cfg, sa_server **out) {
  if (!out) return SA_ERR_INVALID_ARG;
  *out = nullptr;
  sa_server *s = new (std::nothrow) sa_server();
  if (!s) return SA_ERR_OOM;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.budget_bytes == 0) s->cfg.budget_bytes = DEFAULT_BUDGET;
  if (s->cfg.slots == 0) s->cfg.slots = DEFAULT_SLOTS;
  if (s->cfg.slots > MAX_SLOTS) s->cfg.slots = MAX_SLOTS;
  s->device = s->cfg.device;
  if (!s->cfg.simulate && s->device < 0 && cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return SA_ERR_CUDA;
  }
  if (!s->cfg.simulate) {
    int dev0 = 0;
    if (cudaGetDevice(&dev0) != cudaSuccess || cudaSetDevice(s->device) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest) != cudaSuccess ||
        cudaSetDevice(dev0) != cudaSuccess) {
      delete s;
      return SA_ERR_CUDA;
    }
  }
  s->t0 = std::chrono::steady_clock::now();
  for (uint32_t k = 0; k < s->cfg.slots; ++k) s->workers.emplace_back(&sa_server::worker, s, k);
  *out = s;
  return SA_OK;
}

GBSA_API sa_status sa_server_submit(sa_server *s, const uint8_t *host_text, uint64_t n,
                                    uint32_t *host_sa, uint64_t *ticket) {
  if (!s || !ticket) return SA_ERR_INVALID_ARG;
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!host_text || !host_sa)) return SA_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request();
  if (!r) return SA_ERR_OOM;
  r->text = host_text;
  r->n = n;
  r->sa = host_sa;
  r->footprint = sa_request_footprint(n);
  r->info.n = n;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->footprint > s->cfg.budget_bytes || s->stop) {
      delete r;
      return SA_ERR_OOM;
    }
    r->ticket = s->next_ticket++;
    r->info.submit_s = s->now();
    s->requests[r->ticket] = r;
    s->stats.tracked = (uint32_t)s->requests.size();
    s->queue.push_back(r);
    ++s->stats.submitted;
    s->stats.queued = (uint32_t)s->queue.size();
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return SA_OK;
}

GBSA_API int sa_server_poll(sa_server *s, uint64_t ticket, sa_request_info *info) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return -1;
  Request *r = it->second;
  if (!r->done) return 0;
  if (info) *info = r->info;
  s->collect(r);
  return 1;
}

GBSA_API sa_status sa_server_wait(sa_server *s, uint64_t ticket, sa_request_info *info) {
  if (!s) return SA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return SA_ERR_INVALID_ARG;
  Request *r = it->second;
  ++r->waiters;
  s->cv_done.wait(lk, [&] { return r->done; });
  --r->waiters;
  if (info) *info = r->info;
  const sa_status status = r->info.status;
  s->collect(r);
  return status;
}

GBSA_API void sa_server_get_stats(sa_server *s, sa_server_stats *out) {
  if (!s || !out) return;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
}

GBSA_API void sa_server_destroy(sa_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &w : s->workers) w.join();
  for (auto &kv : s->requests) delete kv.second;
  delete s;
}
