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
// Merged builds (sa_server_config.merge_requests >= 2): a worker that takes a
// small head request also takes the small requests queued directly behind
// it and builds them all as one batch (sa_build_batched_host). They share
// one launch sequence and its doubling rounds; each text drops out of the
// rounds as soon as its suffixes are unique, so the batch costs about one
// small build instead of one per request. A worker takes only its share of
// the queue (the queued requests divided among it and the workers idle
// beside it), so requests that idle workers can start at once on their own
// streams are not serialised behind one batch: merging sets in when the
// queue outgrows the idle workers. Only requests already queued join: a
// request that arrives while a batch runs waits for the next free worker.
//
// The paper has no serving layer; this is the runtime around its method.
#include <algorithm>
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
// Merging: requests of up to MERGE_MAX_N characters (the highest-priority
// size class), at most MERGE_TOTAL_MAX in one build (the largest batch whose
// host copies run as kernels), at most MAX_MERGE requests (one copy launch
// per direction). Off by default (DEFAULT_MERGE = 1): on a GB300 it raised a
// burst of 2000 requests of 10-256 KiB from 23k to 79k requests/s, but it did
// not help an overloaded mix of small and large requests.
constexpr uint64_t MERGE_MAX_N = 256ull << 10;
constexpr uint64_t MERGE_TOTAL_MAX = 4ull << 20;
constexpr uint32_t DEFAULT_MERGE = 1;
constexpr uint32_t MAX_MERGE = 64;

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

// Device bytes of one batched build of texts with these offsets (text, SA
// and the batched workspace), the merged counterpart of sa_request_footprint.
size_t merged_footprint(const std::vector<uint64_t> &off) {
  const uint64_t N = off.back();
  return align256(N) + align256(N * 4) +
         sa_batched_workspace_bytes(off.data(), (uint32_t)(off.size() - 1));
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
  uint32_t busy = 0;  // workers running a build
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

  // Takes the head request and, when it is small, the small requests
  // queued directly behind it while the merged build fits the budget, up to
  // this worker's share of the queue. Called with `mu` held, the head
  // admissible and this worker not yet counted in `busy`; returns the bytes
  // to charge against the budget.
  size_t take_batch(std::vector<Request *> &batch, std::vector<uint64_t> &off) {
    const uint64_t queued = queue.size();
    const uint64_t idle = cfg.slots > busy ? cfg.slots - busy : 1;  // this worker included
    const uint64_t share = (queued + idle - 1) / idle;
    Request *head = queue.front();
    queue.pop_front();
    batch.assign(1, head);
    size_t charge = head->footprint;
    const uint64_t limit = std::min<uint64_t>(cfg.merge_requests, share);
    if (limit <= 1 || head->n > MERGE_MAX_N) return charge;
    off.assign({0, head->n});
    while (!queue.empty() && batch.size() < limit) {
      Request *q = queue.front();
      if (q->n > MERGE_MAX_N || off.back() + q->n > MERGE_TOTAL_MAX) break;
      off.push_back(off.back() + q->n);
      const size_t f = merged_footprint(off);
      if (in_use + f > cfg.budget_bytes) {
        off.pop_back();
        break;
      }
      queue.pop_front();
      batch.push_back(q);
      charge = f;
    }
    return charge;
  }

  void worker(uint32_t slot) {
    cudaStream_t streams[PRIORITY_CLASSES] = {};
    if (!cfg.simulate) {
      cudaSetDevice(device);
      for (int c = 0; c < PRIORITY_CLASSES; ++c)
        cudaStreamCreateWithPriority(&streams[c], cudaStreamNonBlocking, priority_of(c));
    }
    std::vector<Request *> batch;
    std::vector<uint64_t> off;
    std::vector<const uint8_t *> texts;
    std::vector<uint64_t> lens;
    std::vector<uint32_t *> sas;
    for (;;) {
      size_t charge = 0;
      uint64_t total = 0;
      int cls = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop && queue.empty()) return true;
          return !queue.empty() && in_use + queue.front()->footprint <= cfg.budget_bytes;
        });
        if (queue.empty()) break;  // stopping and drained
        charge = take_batch(batch, off);
        ++busy;
        for (Request *r : batch) {
          total += r->n;
          cls = std::max(cls, size_class(r->n));
        }
        in_use += charge;
        in_flight += (uint32_t)batch.size();
        stats.in_flight = in_flight;
        ++stats.builds;
        if (batch.size() > 1) stats.merged += batch.size();
        stats.bytes_in_use = in_use;
        if (in_use > stats.peak_bytes_in_use) stats.peak_bytes_in_use = in_use;
        if (in_flight > stats.peak_in_flight) stats.peak_in_flight = in_flight;
        stats.queued = (uint32_t)queue.size();
        const double t = now();
        for (Request *r : batch) {
          r->info.start_s = t;
          r->info.slot = slot;
          r->info.priority = priority_of(cls);
          r->info.batch = (uint32_t)batch.size();
        }
      }
      sa_status status = SA_OK;
      if (cfg.simulate) {
        const double ns = (double)total * cfg.simulate_ns_per_byte;
        std::this_thread::sleep_for(std::chrono::nanoseconds((int64_t)ns));
      } else if (batch.size() == 1) {
        Request *r = batch[0];
        status = sa_build_host(r->text, r->n, r->sa, (gbsa_stream_t)streams[cls]);
      } else {
        texts.clear();
        lens.clear();
        sas.clear();
        for (Request *r : batch) {
          texts.push_back(r->text);
          lens.push_back(r->n);
          sas.push_back(r->sa);
        }
        status = sa_build_batched_host(texts.data(), lens.data(), sas.data(),
                                       (uint32_t)batch.size(), (gbsa_stream_t)streams[cls]);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= charge;
        in_flight -= (uint32_t)batch.size();
        --busy;
        stats.in_flight = in_flight;
        stats.bytes_in_use = in_use;
        stats.completed += batch.size();
        const double t = now();
        for (Request *r : batch) {
          r->info.status = status;
          r->info.done_s = t;
          r->done = true;
        }
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
  if (s->cfg.merge_requests == 0) s->cfg.merge_requests = DEFAULT_MERGE;
  if (s->cfg.merge_requests > MAX_MERGE) s->cfg.merge_requests = MAX_MERGE;
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
