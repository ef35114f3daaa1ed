// Round driver and C-ABI of gbsa: prefix doubling with discarding in
// inverse-suffix-array form (Section 2.1, Algorithms 1, 4 and 5).
//
// Round 0 (initial names, Algorithm 1's first lines):
//   byte histogram -> alphabet (host) -> packed keys -> radix sort ->
//   rename/unique/compact.
// Round r >= 1 (one doubling step, h = c0 * 2^(r-1) characters resolved):
//   large groups: partner-name gather -> radix sort of (group, partner)
//   keys; small groups: tile-local refine (k_refine.cu); then the rename of
//   the large groups, the queued ISA updates and the classification of the
//   new groups.
// With sa_options.multiplier a = 3 or 4 (Section 2.1, Prefix Quadrupling) a
// round ranks the names of i, i + h, .., i + (a-1)h and h grows a-fold: the
// sorts become two stable sorts (later partners, then group and first
// partner) and the boundary tests compare the whole tuple.
// The loop ends when no suffix is active (every name unique; the paper's
// loop bound is one round short, so the count decides). SA is complete then:
// each suffix wrote SA[name] = i when its name became unique.
//
// Host <-> device per round: one 64-byte read of the control block (active
// and group counts of both producers, large-group counts, pass count, error
// word) at the end of the round.
//
// Data layout in HBM (N characters in S texts, gapped positions N + S):
//   keys A/B u64[N], vals A/B u32[N] (radix sort of round 0 and of large
//   groups), active lists u64[N] x2 (g << 32 | i', current and next), queued
//   ISA updates u64[N], ISA u32[N + S + 1] (end slots hold 0xFFFFFFFF),
//   group starts, names and head ranks u32[N/2+1] x2 each, parent names
//   u32[N/2+1], large-group lists, the refine tile map, look-back status,
//   control block, plan, histograms: about 67 bytes per character.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbsa.h"
#include "launch.h"
#include "segcopy.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {
namespace {

constexpr uint32_t DEFAULT_SPIN_LIMIT = 1u << 20;  // ~1 s with the 1 us back-off cap
// ISA writes are bucketed by position when this many may be pending (the
// default discard threshold; sa_options.bucket_min and the tuning table
// override it).
constexpr uint32_t BUCKET_MIN = 1u << 22;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// NVTX ranges (header-only NVTX 3: without a profiler attached a push or
// pop is a call through a pointer to a function that returns at once).
// A build is one range, each round a range inside it, each kernel launch
// a range named for its class, so a profiler's launch list attributes
// every kernel to its round and step.
const char *const KERNEL_RANGE[SA_K_CLASSES] = {
    "gbsa:byte_hist", "gbsa:pack",     "gbsa:digit_hist", "gbsa:plan",     "gbsa:onesweep",
    "gbsa:rename",    "gbsa:gather",   "gbsa:output",     "gbsa:refine",   "gbsa:scatter",
    "gbsa:classify",  "gbsa:apply",    "gbsa:bucket",     "gbsa:reorder"};

struct NvtxRange {
  bool open = true;
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  void end() {
    if (open) nvtxRangePop();
    open = false;
  }
  ~NvtxRange() { end(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Layout {
  size_t ctrl, plan, hist, dbase, bytehist, code, segoff;
  size_t ka, kb, va, vb, act0, act1, upd, isa, gs0, gs1, gn0, gn1, gh0, gh1, gold;
  size_t lg, loff, lbase, lold, tfirst, bcount, pm1;
  size_t st_sort, st_ren, total;
  size_t st_sort_bytes, st_ren_bytes;
  uint32_t max_groups, max_large, max_tiles;
};

Layout make_layout(uint64_t N, uint32_t S) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += align256(bytes);
    return r;
  };
  const uint64_t Nm = N ? N : 1;
  L.ctrl = take(sizeof(Ctrl));
  L.plan = take(sizeof(SortPlan));
  L.hist = take(MAX_PASSES * RADIX * 4);
  L.dbase = take(MAX_PASSES * RADIX * 4);
  L.bytehist = take(RADIX * 4);
  L.code = take(RADIX);
  L.segoff = take(((size_t)S + 1) * 4);
  L.ka = take(Nm * 8);
  L.kb = take(Nm * 8);
  L.va = take(Nm * 4);
  L.vb = take(Nm * 4);
  L.act0 = take(Nm * 8);
  L.act1 = take(Nm * 8);
  L.upd = take(Nm * 8);
  L.isa = take((N + S + 1) * 4);
  L.max_groups = (uint32_t)(Nm / 2 + 1);
  L.gs0 = take(((size_t)L.max_groups + 1) * 4);
  L.gs1 = take(((size_t)L.max_groups + 1) * 4);
  L.gn0 = take((size_t)L.max_groups * 4);
  L.gn1 = take((size_t)L.max_groups * 4);
  L.gh0 = take((size_t)L.max_groups * 4);
  L.gh1 = take((size_t)L.max_groups * 4);
  L.gold = take((size_t)L.max_groups * 4);
  L.max_large = (uint32_t)(Nm / (REFINE_MIN_NOMINAL + 1) + 1);
  L.lg = take((size_t)L.max_large * 4);
  L.loff = take((size_t)L.max_large * 4);
  L.lbase = take((size_t)L.max_large * 4);
  L.lold = take((size_t)L.max_large * 4);
  L.bcount = take((size_t)BUCKET_BLOCKS_MAX * RADIX * 4);
  L.pm1 = take(8);
  L.max_tiles = (uint32_t)((Nm + REFINE_MIN_NOMINAL - 1) / REFINE_MIN_NOMINAL);
  L.tfirst = take(((size_t)L.max_tiles + 1) * 4);
  const uint64_t ts = std::max<uint64_t>(1, (N + SORT_TILE_MIN - 1) / SORT_TILE_MIN);
  L.st_sort_bytes = ts * RADIX * 8;
  L.st_sort = take(L.st_sort_bytes);
  const uint64_t tr = std::max<uint64_t>(1, (N + RENAME_TILE - 1) / RENAME_TILE);
  L.st_ren_bytes = tr * 3 * 8;
  L.st_ren = take(L.st_ren_bytes);
  L.total = o;
  return L;
}

uint32_t bits_for(uint64_t v) {  // bits to hold values 0..v
  uint32_t b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

int sm_count() { return device_sm_count(); }

// Library-private stream-ordered pools, one per device (never trimmed, so
// repeated builds reuse their memory without touching the process-wide
// default pool).
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
  std::mutex &mu = g_pool_mu;
  std::map<int, cudaMemPool_t> &pools = g_pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = pools.find(dev);
    if (it == pools.end()) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

struct PoolBuf {
  void *p = nullptr;
  cudaStream_t st = nullptr;
  ~PoolBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return SA_ERR_CUDA; \
  } while (0)

// Mirror of the first 64 bytes of Ctrl.
// Pinned host staging for the small readbacks of a build (control block,
// byte histogram): a kernel writes them into pinned host memory, so a
// readback does not wait on a copy engine behind the large copies of
// builds on other streams (a server's concurrent requests). Blocks are
// allocated once (mapped into every device's address space) and reused.
constexpr size_t STAGE_BYTES = 16 << 10;
std::mutex g_stage_mu;
std::vector<void *> g_stage_free;

struct PinnedStage {
  void *p = nullptr;
  cudaError_t get() {
    if (p) return cudaSuccess;
    {
      std::lock_guard<std::mutex> g(g_stage_mu);
      if (!g_stage_free.empty()) {
        p = g_stage_free.back();
        g_stage_free.pop_back();
        return cudaSuccess;
      }
    }
    const cudaError_t e = cudaHostAlloc(&p, STAGE_BYTES, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) p = nullptr;  // nothing to hand back to the free list
    return e;
  }
  ~PinnedStage() {
    if (!p) return;
    std::lock_guard<std::mutex> g(g_stage_mu);
    g_stage_free.push_back(p);
  }
};

struct HostCtrl {
  uint32_t error, err_where, passes, pass_mask;
  uint32_t m_s, g_s, m_l, g_l, upd, pad;
  unsigned long long large;
  uint32_t zero[4];
  uint32_t m_next() const { return m_s + m_l; }
  uint32_t g_next() const { return g_s + g_l; }
  uint32_t m_large() const { return (uint32_t)large; }
  uint32_t g_large() const { return (uint32_t)(large >> 32); }
};
static_assert(sizeof(HostCtrl) == 64, "HostCtrl mirrors the head of Ctrl");

struct Build {
  PinnedStage stage;            // small readbacks (fetch)
  bool stage_readbacks = true;  // false: copy-engine readbacks (no host allocation)
  // inputs
  const uint8_t *text = nullptr;
  uint64_t N = 0;
  uint32_t S = 1;
  std::vector<uint32_t> off;  // S+1 ungapped offsets
  uint32_t *sa = nullptr;
  uint32_t *isa_out = nullptr;
  sa_options opt{};
  sa_stats *stats = nullptr;
  cudaStream_t st = nullptr;
  // workspace
  uint8_t *ws = nullptr;
  Layout L{};
  Ctrl *ctrl = nullptr;
  SortPlan *plan = nullptr;
  uint32_t *hist = nullptr, *dbase = nullptr, *bytehist = nullptr, *segoff = nullptr;
  uint8_t *code = nullptr;
  uint64_t *ka = nullptr, *kb = nullptr, *act[2] = {nullptr, nullptr}, *upd = nullptr;
  uint64_t *st_sort = nullptr, *st_ren = nullptr;
  uint32_t *va = nullptr, *vb = nullptr, *isa = nullptr;
  uint32_t *gstart[2] = {nullptr, nullptr}, *gname[2] = {nullptr, nullptr};
  uint32_t *ghead[2] = {nullptr, nullptr}, *gold = nullptr;
  uint32_t *lg = nullptr, *loff = nullptr, *lbase = nullptr, *lold = nullptr, *tfirst = nullptr;
  uint32_t *bcount = nullptr;  // position-bucketing counts (BUCKET_BLOCKS_MAX x 256)
  uint32_t *pm1 = nullptr;     // (passes, pass mask) of the first sort of an a-tuple round
  // launch bookkeeping
  uint32_t epoch = 0, slot = 0;
  uint32_t spin = DEFAULT_SPIN_LIMIT;
  bool inject_pending = false;
  uint64_t bytes = 0;
  uint32_t launches = 0;
  uint32_t naming = NAMES_RETAIN;
  uint32_t shape = 0, nominal = 512;  // refine tile shape and window
  uint32_t sort_items = SORT_ITEMS_DEFAULT;  // keys per thread of the radix pass
  uint32_t bucket_min = BUCKET_MIN;  // pending ISA writes that are bucketed first
  uint32_t mult = 2;  // a: names ranked per round (2: doubling, 4: quadrupling)
  // per-kernel profiling (events on the build's stream)
  struct Rec {
    int cls, pass;
    uint64_t bytes;
    cudaEvent_t a, b;
  };
  bool prof = false;
  // Launches whose byte counts wait for the round's control block.
  static constexpr uint64_t PENDING = ~0ull;
  struct Pending {
    uint32_t scatter = 0, apply = 0, bucket_upd = 0, bucket_surv = 0;
  } pend;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  std::vector<Rec> recs;

  ~Build() {
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
  }

  template <class T>
  T *at(size_t off_) {
    return reinterpret_cast<T *>(ws + off_);
  }

  void carve() {
    ctrl = at<Ctrl>(L.ctrl);
    plan = at<SortPlan>(L.plan);
    hist = at<uint32_t>(L.hist);
    dbase = at<uint32_t>(L.dbase);
    bytehist = at<uint32_t>(L.bytehist);
    code = at<uint8_t>(L.code);
    segoff = at<uint32_t>(L.segoff);
    ka = at<uint64_t>(L.ka);
    kb = at<uint64_t>(L.kb);
    va = at<uint32_t>(L.va);
    vb = at<uint32_t>(L.vb);
    act[0] = at<uint64_t>(L.act0);
    act[1] = at<uint64_t>(L.act1);
    upd = at<uint64_t>(L.upd);
    isa = at<uint32_t>(L.isa);
    gstart[0] = at<uint32_t>(L.gs0);
    gstart[1] = at<uint32_t>(L.gs1);
    gname[0] = at<uint32_t>(L.gn0);
    gname[1] = at<uint32_t>(L.gn1);
    ghead[0] = at<uint32_t>(L.gh0);
    ghead[1] = at<uint32_t>(L.gh1);
    gold = at<uint32_t>(L.gold);
    lg = at<uint32_t>(L.lg);
    loff = at<uint32_t>(L.loff);
    lbase = at<uint32_t>(L.lbase);
    lold = at<uint32_t>(L.lold);
    bcount = at<uint32_t>(L.bcount);
    pm1 = at<uint32_t>(L.pm1);
    tfirst = at<uint32_t>(L.tfirst);
    st_sort = at<uint64_t>(L.st_sort);
    st_ren = at<uint64_t>(L.st_ren);
  }

  cudaError_t event(cudaEvent_t &e) {
    if (evused == evpool.size()) {
      cudaEvent_t x;
      cudaError_t r = cudaEventCreate(&x);
      if (r != cudaSuccess) return r;
      evpool.push_back(x);
    }
    e = evpool[evused++];
    return cudaEventRecord(e, st);
  }

  // Issues one kernel launch; with profiling, brackets it with events.
  // `bytes` is the launch's algorithmic traffic (radix passes: counted only
  // if the device plan kept the pass; rename: settled at the round's sync).
  template <class F>
  sa_status launch(int cls, int pass, uint64_t nbytes, F f) {
    NvtxRange range(KERNEL_RANGE[cls]);
    ++launches;
    cudaEvent_t a = nullptr, b = nullptr;
    if (prof) CK(event(a));
    CK(f());
    if (prof) {
      CK(event(b));
      recs.push_back({cls, pass, nbytes, a, b});
    }
    return SA_OK;
  }

  // After a stream sync: fold the recorded launches into the statistics.
  sa_status flush(uint32_t pass_mask, uint64_t rename_bytes_now, uint32_t mask1 = 0) {
    if (!prof || !stats) {
      recs.clear();
      evused = 0;
      return SA_OK;
    }
    for (const Rec &r : recs) {
      if (r.cls == SA_K_ONESWEEP &&
          !(((r.pass >= 32 ? mask1 : pass_mask) >> (r.pass & 31)) & 1u))
        continue;
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      stats->kernel_ms[r.cls] += ms;
      stats->kernel_launches[r.cls] += 1;
      stats->kernel_bytes[r.cls] += r.cls == SA_K_RENAME ? rename_bytes_now : r.bytes;
    }
    recs.clear();
    evused = 0;
    return SA_OK;
  }

  sa_status next_launch(uint32_t *&ctr, uint32_t &ep) {
    if (slot == (uint32_t)TILE_COUNTERS) {
      CK(cudaMemsetAsync(ctrl->tile_ctr, 0, sizeof(ctrl->tile_ctr), st));
      slot = 0;
    }
    ctr = &ctrl->tile_ctr[slot++];
    ep = ++epoch;
    return SA_OK;
  }

  // bytes of device memory into host memory, synchronising `st`: through
  // the pinned stage by a kernel (a multiple of 4 bytes, at most
  // STAGE_BYTES), else, or without a stage, on the copy engine.
  cudaError_t fetch(void *host, const void *dev, size_t bytes) {
    if (stage_readbacks && bytes <= STAGE_BYTES && bytes % 4 == 0 && stage.get() != cudaSuccess) {
      cudaGetLastError();  // no pinned block to be had: the copy engine instead
      stage_readbacks = false;
    }
    if (!stage_readbacks || bytes > STAGE_BYTES || bytes % 4) {
      cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st);
      return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
    }
    cudaError_t e = launch_copy_words(reinterpret_cast<uint32_t *>(stage.p),
                                      reinterpret_cast<const uint32_t *>(dev), bytes / 4, st);
    if (e == cudaSuccess) ++launches;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) memcpy(host, stage.p, bytes);
    return e;
  }

  sa_status read_ctrl(HostCtrl &hc) {
    CK(fetch(&hc, ctrl, sizeof(HostCtrl)));
    if (hc.error == ERR_TIMEOUT) return SA_ERR_TIMEOUT;
    if (hc.error != ERR_NONE) return SA_ERR_INTERNAL;
    return SA_OK;
  }

  // Radix sort of (ka, va)[0, m) by the digits of spec; result where the
  // device plan says (plan->kfinal / vfinal).
  // chain 1: the first of the two sorts of an a-tuple round (its kept
  // passes are copied to pm1 afterwards; profile records tag pass + 32).
  // from_text (round 0, one text): pass 0 builds the keys from the text
  // (the pack wrote only the histograms), so it is kept even if constant.
  sa_status sort(uint32_t m, const DigitSpec &spec, bool hist_ready = false, int chain = 0,
                 const PackArgs *from_text = nullptr) {
    sa_status s = SA_OK;
    if (!hist_ready) {
      CK(cudaMemsetAsync(hist, 0, (size_t)spec.P * RADIX * 4, st));
      s = launch(SA_K_DIGIT_HIST, 0, 8ull * m, [&] {
        return launch_digit_histogram(ka, m, spec, hist, sm_count(), st);
      });
      if (s != SA_OK) return s;
      bytes += 8ull * m;  // histogram read
    }
    s = launch(SA_K_PLAN, 0, (uint64_t)spec.P * RADIX * 8, [&] {
      return launch_sort_plan(hist, dbase, spec, m, ka, kb, va, vb, plan, ctrl, st, nullptr,
                              from_text != nullptr);
    });
    if (s != SA_OK) return s;
    for (uint32_t p = 0; p < spec.P; ++p) {
      PassArgs pa{};
      pa.plan = plan;
      pa.p = (int)p;
      pa.shift = spec.shift[p];
      pa.bits = spec.bits[p];
      pa.digit_base = dbase + p * RADIX;
      pa.m = m;
      pa.status = st_sort;
      s = next_launch(pa.tile_ctr, pa.epoch);
      if (s != SA_OK) return s;
      pa.ctrl = ctrl;
      pa.spin_limit = spin;
      pa.inject = inject_pending ? 1u : 0u;
      pa.items = sort_items;
      uint64_t pass_bytes = 24ull * m;
      if (from_text && p == 0) {
        pa.text = from_text->text;
        pa.code = from_text->code;
        pa.b = from_text->b;
        pa.c0 = from_text->c0;
        pa.cb = from_text->cb;
        pa.tails = std::min(m, from_text->c0 - 1);
        pass_bytes = 13ull * m;  // the text read, the sorted keys and positions written
      }
      s = launch(SA_K_ONESWEEP, (int)p + 32 * chain, pass_bytes,
                 [&] { return launch_onesweep(pa, st); });
      if (s != SA_OK) return s;
    }
    inject_pending = false;
    if (chain == 1) CK(cudaMemcpyAsync(pm1, &ctrl->passes, 8, cudaMemcpyDeviceToDevice, st));
    return SA_OK;
  }

  static DigitSpec spec_for(uint32_t total_bits) {
    DigitSpec s{};
    s.P = (total_bits + RADIX_BITS - 1) / RADIX_BITS;
    for (uint32_t p = 0; p < s.P; ++p) {
      s.shift[p] = (uint8_t)(p * RADIX_BITS);
      s.bits[p] = (uint8_t)std::min<uint32_t>(RADIX_BITS, total_bits - p * RADIX_BITS);
    }
    return s;
  }

  // Rename of round 0 (all suffixes) or of the large groups of a later
  // round; writes the next active list at the device-side offsets `off_in`.
  sa_status rename(uint32_t m, bool round0, uint32_t cb, uint32_t c0, uint32_t W,
                   const uint32_t *base_in, const uint32_t *old_in, uint32_t g_in, int out,
                   const uint32_t *off_in, bool wide = false) {
    RenameArgs ra{};
    ra.sec_buf[0] = wide ? ka : nullptr;
    ra.sec_buf[1] = wide ? kb : nullptr;
    ra.plan = plan;
    ra.m = m;
    ra.round0 = round0 ? 1u : 0u;
    ra.cb = cb;
    ra.c0 = c0;
    ra.seg_off = segoff;
    ra.S = S;
    ra.W = W;
    ra.base_in = base_in;
    ra.old_in = old_in;
    ra.g_in = g_in;
    ra.isa = isa;
    ra.upd = upd;
    ra.isa_len = N + S + 1;
    ra.N = (uint32_t)N;
    ra.sa = sa;
    ra.act_out = act[out];
    ra.gstart_out = gstart[out];
    ra.ghead_out = ghead[out];
    ra.gold_out = gold;
    ra.off_in = off_in;
    ra.cnt_out = &ctrl->rc.m_l;
    ra.status = st_ren;
    sa_status s = next_launch(ra.tile_ctr, ra.epoch);
    if (s != SA_OK) return s;
    ra.ctrl = ctrl;
    ra.spin_limit = spin;
    return launch(SA_K_RENAME, 0, 0, [&] { return launch_rename(ra, st); });
  }

  // Large groups and the refine tile map of the list just written.
  sa_status classify(int out, uint64_t cap_groups, uint32_t apply_bound) {
    ClassifyArgs ca{};
    ca.gstart = gstart[out];
    ca.gname = gname[out];
    ca.ghead = ghead[out];
    ca.gold = gold;
    ca.naming = naming;
    ca.lg = lg;
    ca.loff = loff;
    ca.lbase = lbase;
    ca.lold = lold;
    ca.tfirst = tfirst;
    ca.nominal = nominal;
    ca.max_groups = L.max_groups;
    ca.max_tiles = L.max_tiles;
    ca.ctrl = ctrl;
    sa_status s = launch(SA_K_CLASSIFY, 0, 16 * cap_groups,
                         [&] { return launch_classify(ca, sm_count(), st); });
    if (s != SA_OK) return s;
    // ISA entries of the rename's survivors whose name changed, bucketed by
    // position first when there can be many.
    if (apply_bound == 0) return SA_OK;
    const uint64_t *src = act[out];
    const uint32_t *lo = &ctrl->rc.m_s;
    const uint32_t *count = &ctrl->rc.m_l;
    uint32_t translated = 0;
    if (apply_bound >= bucket_min) {
      // The partition reads the group names while the entries are still in
      // group order and keeps only the changed ones, as (name, i').
      s = bucket(src, lo, &ctrl->rc.m_l, apply_bound, 2, gname[out]);
      if (s != SA_OK) return s;
      src = kb;
      lo = ctrl->zero;
      count = &ctrl->bucket_total;
      translated = 1;
    }
    ++pend.apply;
    return launch(SA_K_APPLY, 0, PENDING, [&] {
      return launch_apply_names(src, lo, count, apply_bound, gname[out], gold, isa, N + S + 1,
                                st, translated);
    });
  }

  // Position bucketing of `count` entries starting at `lo` into keys
  // buffer B (free whenever ISA writes are pending). `src_tag` tells the
  // byte settlement which count applies (0: queued updates, 2: survivors).
  sa_status bucket(const uint64_t *in, const uint32_t *lo, const uint32_t *count,
                   uint32_t max_count, int src_tag, const uint32_t *translate_names = nullptr) {
    BucketArgs ba{};
    if (translate_names) {
      ba.gname = translate_names;
      ba.gold = gold;
      ba.total_out = &ctrl->bucket_total;
    }
    ba.in = in;
    ba.lo = lo;
    ba.count = count;
    ba.max_count = max_count;
    const uint32_t bits = bits_for(N + S);
    ba.shift = bits > 8 ? bits - 8 : 0;
    ba.blocks = std::min<uint32_t>(BUCKET_BLOCKS_MAX, 4 * sm_count());
    ba.counts = bcount;
    ba.out = kb;
    ++(src_tag ? pend.bucket_surv : pend.bucket_upd);
    sa_status s = launch(SA_K_BUCKET, src_tag, PENDING,
                         [&] { return launch_bucket_count(ba, st); });
    if (s != SA_OK) return s;
    s = launch(SA_K_BUCKET, src_tag, 0, [&] { return launch_bucket_offsets(ba, st); });
    if (s != SA_OK) return s;
    return launch(SA_K_BUCKET, src_tag | 1, PENDING,
                  [&] { return launch_bucket_scatter(ba, st); });
  }

  // ISA[i'] = new for the queued updates (at most `bound` of them).
  sa_status scatter(uint32_t bound) {
    if (bound == 0) return SA_OK;
    const uint64_t *src = upd;
    if (bound >= bucket_min) {
      sa_status s = bucket(upd, nullptr, &ctrl->rc.upd, bound, 0);
      if (s != SA_OK) return s;
      src = kb;
    }
    ++pend.scatter;
    return launch(SA_K_SCATTER, 0, PENDING, [&] {
      return launch_scatter_updates(src, bound, isa, N + S + 1, ctrl, st);
    });
  }

  // Byte counts of the launches whose sizes are known only from this
  // round's control block: scatter and apply read 8 and write 4 bytes per
  // entry; bucketing reads 8 (histogram), then reads and writes 8.
  void settle(const HostCtrl &hc) {
    bytes += pend.scatter * 12ull * hc.upd + pend.apply * 12ull * hc.m_l +
             pend.bucket_upd * 24ull * hc.upd + pend.bucket_surv * 24ull * hc.m_l;
    pend = Pending{};
    for (Rec &r : recs) {
      if (r.bytes != PENDING) continue;
      if (r.cls == SA_K_SCATTER) r.bytes = 12ull * hc.upd;
      if (r.cls == SA_K_APPLY) r.bytes = 12ull * hc.m_l;
      if (r.cls == SA_K_BUCKET)
        r.bytes = ((r.pass & 1) ? 16ull : 8ull) * ((r.pass & 2) ? hc.m_l : hc.upd);
    }
  }

  // Rename (round 0 or large groups) reads 12 bytes per item; writes 4
  // (SA) + 8 (queued ISA entry) per unique item, 8 per survivor and 12 per
  // surviving group (start, head rank, parent name).
  static uint64_t rename_bytes(uint32_t m, uint32_t surv, uint32_t groups) {
    const uint64_t u = m - surv;
    return 12ull * m + 12 * u + 8ull * surv + 12ull * groups;
  }

  // Refine: 8 bytes read and a - 1 4-byte gathers per item, 8 bytes of
  // group table per input group, 8 per survivor and per new group, 4 (SA)
  // per unique item, 8 per queued update.
  static uint64_t refine_bytes(uint32_t m, uint32_t G, uint32_t surv, uint32_t groups,
                               uint32_t upd_n, uint32_t a) {
    const uint64_t u = m - surv;
    return (8ull + 4ull * (a - 1)) * m + 8ull * G + 8ull * surv + 8ull * groups + 4 * u +
           8ull * upd_n;
  }

  // Device-driven rounds: only for doubling (a = 2), without the per-launch
  // profile or the per-round name trace; sa_options.device_rounds 1 asks
  // for them, 2 refuses them, 0 leaves the choice to the library.
  bool device_rounds_wanted() const {
    if (mult != 2 || prof || (opt.trace_isa && opt.trace_cap > 1)) return false;
    if (opt.device_rounds == 1) return true;
    if (opt.device_rounds == 2) return false;
    return false;
  }

  // Adds an if-node at the capture point of `outer` (handle h, created on
  // the graph being captured) and starts capturing its body on `inner`.
  static cudaError_t begin_if(cudaStream_t outer, cudaStream_t inner,
                              cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(outer, &cst, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
    if (e != cudaSuccess) return e;
    e = cudaStreamUpdateCaptureDependencies(outer, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    return cudaStreamBeginCaptureToGraph(inner, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed);
  }

  static cudaError_t end_capture(cudaStream_t s) {
    cudaGraph_t g = nullptr;
    return cudaStreamEndCapture(s, &g);
  }

  struct RoundHandles {
    cudaGraphConditionalHandle sort, rename, bucket_upd, bucket_surv;
  };

  // Captures one round (active list and group tables in buffer `cur`) on
  // stream cs, its optional steps in if-nodes captured on cs2. Grids are
  // sized for m1 items (the most any round after round 0 can have) and
  // capped, the kernels looping over their work.
  cudaError_t capture_round(cudaStream_t cs, cudaStream_t cs2, int cur, const RoundHandles &hd,
                            uint32_t m1, uint32_t W) {
    const int nxt = cur ^ 1;
    const uint32_t sms = (uint32_t)sm_count();
    const RoundState *rs = &ctrl->rs;
    RoundBeginArgs rb{};
    rb.ctrl = ctrl;
    rb.hist = hist;
    rb.W = W;
    rb.nominal = nominal;
    rb.bucket_min = bucket_min;
    rb.N = (uint32_t)N;
    rb.if_sort = hd.sort;
    rb.if_rename = hd.rename;
    rb.if_bucket_upd = hd.bucket_upd;
    rb.if_bucket_surv = hd.bucket_surv;
    cudaError_t e = launch_round_begin(rb, cs);
    if (e != cudaSuccess) return e;

    // Large groups: partner names and the global radix sort.
    if ((e = begin_if(cs, cs2, hd.sort)) != cudaSuccess) return e;
    GatherLargeArgs ga{};
    ga.act = act[cur];
    ga.gstart = gstart[cur];
    ga.lg = lg;
    ga.loff = loff;
    ga.mL = m1;
    ga.W = W;
    ga.mult = 2;
    ga.isa = isa;
    ga.isa_len = N + S + 1;
    ga.keys = ka;
    ga.vals = va;
    ga.rs = rs;
    ga.grid_cap = 8 * sms;
    if ((e = launch_gather_large(ga, cs2)) != cudaSuccess) return e;
    const DigitSpec none{};
    if ((e = launch_digit_histogram(ka, m1, none, hist, (int)sms, cs2, rs)) != cudaSuccess) return e;
    if ((e = launch_sort_plan(hist, dbase, none, m1, ka, kb, va, vb, plan, ctrl, cs2, rs)) !=
        cudaSuccess)
      return e;
    for (int p = 0; p < MAX_PASSES; ++p) {
      PassArgs pa{};
      pa.plan = plan;
      pa.p = p;
      pa.digit_base = dbase + p * RADIX;
      pa.m = m1;
      pa.status = st_sort;
      pa.epoch = (uint32_t)p;  // offset from the round's epoch base
      pa.tile_ctr = &ctrl->tile_ctr[p];
      pa.ctrl = ctrl;
      pa.spin_limit = spin;
      pa.items = sort_items;
      pa.rs = rs;
      pa.grid_cap = sms * (sort_items >= 16 ? 3u : (sort_items >= 12 ? 4u : 5u));
      if ((e = launch_onesweep(pa, cs2)) != cudaSuccess) return e;
    }
    if ((e = end_capture(cs2)) != cudaSuccess) return e;

    // Small groups: the tile-local refine.
    RefineArgs rf{};
    rf.act = act[cur];
    rf.gstart = gstart[cur];
    rf.gname = gname[cur];
    rf.ghead = ghead[cur];
    rf.naming = naming;
    rf.tfirst = tfirst;
    rf.m = m1;
    rf.shape = shape;
    rf.tiles = (m1 + nominal - 1) / nominal;
    rf.W = W;
    rf.mult = 2;
    rf.isa = isa;
    rf.isa_len = N + S + 1;
    rf.N = (uint32_t)N;
    rf.sa = sa;
    rf.seg_off = segoff;
    rf.S = S;
    rf.act_out = act[nxt];
    rf.gstart_out = gstart[nxt];
    rf.gname_out = gname[nxt];
    rf.ghead_out = ghead[nxt];
    rf.upd = upd;
    rf.ctrl = ctrl;
    rf.rs = rs;
    {  // two waves of the resident blocks (k_refine's launch bounds)
      const RefineShape sh = REFINE_SHAPE[shape];
      rf.grid_cap = 2 * sms * ((sh.cap / sh.block > 8 ? 512u : 1024u) / sh.block);
    }
    if ((e = launch_refine(rf, cs)) != cudaSuccess) return e;

    // The large groups' rename (after every gather of the round).
    if ((e = begin_if(cs, cs2, hd.rename)) != cudaSuccess) return e;
    RenameArgs ra{};
    ra.plan = plan;
    ra.m = m1;
    ra.W = W;
    ra.seg_off = segoff;
    ra.S = S;
    ra.base_in = lbase;
    ra.old_in = lold;
    ra.g_in = L.max_large;
    ra.isa = isa;
    ra.upd = upd;
    ra.isa_len = N + S + 1;
    ra.N = (uint32_t)N;
    ra.sa = sa;
    ra.act_out = act[nxt];
    ra.gstart_out = gstart[nxt];
    ra.ghead_out = ghead[nxt];
    ra.gold_out = gold;
    ra.off_in = &ctrl->rc.m_s;
    ra.cnt_out = &ctrl->rc.m_l;
    ra.status = st_ren;
    ra.epoch = MAX_PASSES;  // offset from the round's epoch base
    ra.tile_ctr = &ctrl->tile_ctr[MAX_PASSES];
    ra.ctrl = ctrl;
    ra.spin_limit = spin;
    ra.rs = rs;
    ra.grid_cap = 4 * sms;
    if ((e = launch_rename(ra, cs2)) != cudaSuccess) return e;
    if ((e = end_capture(cs2)) != cudaSuccess) return e;

    // The round's queued ISA updates, bucketed by position when many.
    BucketArgs ba{};
    const uint32_t bits = bits_for(N + S);
    ba.shift = bits > 8 ? bits - 8 : 0;
    ba.blocks = std::min<uint32_t>(BUCKET_BLOCKS_MAX, 4 * sms);
    ba.counts = bcount;
    ba.out = kb;
    ba.in = upd;
    ba.count = &ctrl->rc.upd;
    ba.max_count = m1;
    if ((e = begin_if(cs, cs2, hd.bucket_upd)) != cudaSuccess) return e;
    if ((e = launch_bucket_count(ba, cs2)) != cudaSuccess) return e;
    if ((e = launch_bucket_offsets(ba, cs2)) != cudaSuccess) return e;
    if ((e = launch_bucket_scatter(ba, cs2)) != cudaSuccess) return e;
    if ((e = end_capture(cs2)) != cudaSuccess) return e;
    if ((e = launch_scatter_updates(upd, m1, isa, N + S + 1, ctrl, cs, kb, rs, 8 * sms)) !=
        cudaSuccess)
      return e;

    // The new groups, and the ISA entries of the rename's survivors.
    ClassifyArgs ca{};
    ca.gstart = gstart[nxt];
    ca.gname = gname[nxt];
    ca.ghead = ghead[nxt];
    ca.gold = gold;
    ca.naming = naming;
    ca.lg = lg;
    ca.loff = loff;
    ca.lbase = lbase;
    ca.lold = lold;
    ca.tfirst = tfirst;
    ca.nominal = nominal;
    ca.max_groups = L.max_groups;
    ca.max_tiles = L.max_tiles;
    ca.ctrl = ctrl;
    ca.rs = rs;
    if ((e = launch_classify(ca, (int)sms, cs)) != cudaSuccess) return e;
    ba.in = act[nxt];
    ba.lo = &ctrl->rc.m_s;
    ba.count = &ctrl->rc.m_l;
    ba.gname = gname[nxt];  // translating: (name, i') of the changed names only
    ba.gold = gold;
    ba.total_out = &ctrl->bucket_total;
    if ((e = begin_if(cs, cs2, hd.bucket_surv)) != cudaSuccess) return e;
    if ((e = launch_bucket_count(ba, cs2)) != cudaSuccess) return e;
    if ((e = launch_bucket_offsets(ba, cs2)) != cudaSuccess) return e;
    if ((e = launch_bucket_scatter(ba, cs2)) != cudaSuccess) return e;
    if ((e = end_capture(cs2)) != cudaSuccess) return e;
    return launch_apply_names(act[nxt], &ctrl->rc.m_s, &ctrl->rc.m_l, m1, gname[nxt], gold, isa,
                              N + S + 1, cs, 0, kb, ctrl->zero, &ctrl->bucket_total, rs, 8 * sms);
  }

  // Rounds >= 1 as one graph: while (suffixes active) { round; round }.
  // `round` returns the number of rounds including round 0.
  sa_status run_device_rounds(const HostCtrl &hc0, uint32_t W, uint32_t h1, int cur,
                              uint32_t &round) {
    const uint32_t m1 = hc0.m_next();
    RoundState rs0{};
    rs0.live = 1;
    rs0.round = 0;
    rs0.h_next = h1;
    rs0.epoch = epoch + ROUND_EPOCHS;
    CK(cudaMemcpyAsync(&ctrl->rs, &rs0, sizeof(rs0), cudaMemcpyHostToDevice, st));
    // Round 0's kernels already set the attributes of the sort and rename
    // kernels; the refine's are set when it is first captured (a host call
    // that capture allows).
    cudaStream_t cs = nullptr, cs2 = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
      if (exec) cudaGraphExecDestroy(exec);
      if (g) cudaGraphDestroy(g);
      if (cs2) cudaStreamDestroy(cs2);
      if (cs) cudaStreamDestroy(cs);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle loop{};
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cudaGraphNodeParams p{};
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = loop;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      cudaGraphNode_t node;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
      if (e == cudaSuccess) body = p.conditional.phGraph_out[0];
    }
    RoundHandles hd[2];
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      cudaGraphConditionalHandle *hs[4] = {&hd[k].sort, &hd[k].rename, &hd[k].bucket_upd,
                                           &hd[k].bucket_surv};
      for (cudaGraphConditionalHandle *hp : hs)
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(hp, body, 0, 0);
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ce = capture_round(cs, cs2, cur, hd[0], m1, W);
      if (ce == cudaSuccess) ce = capture_round(cs, cs2, cur ^ 1, hd[1], m1, W);
      if (ce == cudaSuccess) ce = launch_round_end(ctrl, loop, cs);
      cudaStreamCaptureStatus c2 = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(cs2, &c2) == cudaSuccess && c2 != cudaStreamCaptureStatusNone)
        end_capture(cs2);
      e = end_capture(cs);
      if (ce != cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return SA_ERR_CUDA;
    }
    launches += 1;  // the graph (its kernels are counted below)
    // One readback of the whole control block (a few KB): error word, the
    // last round's counters, the round state and the per-round records.
    std::vector<uint8_t> raw(sizeof(Ctrl));
    static_assert(sizeof(Ctrl) <= STAGE_BYTES && sizeof(Ctrl) % 4 == 0, "Ctrl fits the stage");
    e = fetch(raw.data(), ctrl, sizeof(Ctrl));
    cleanup();
    if (e != cudaSuccess) return SA_ERR_CUDA;
    const Ctrl &hctrl = *reinterpret_cast<const Ctrl *>(raw.data());
    HostCtrl hc{};
    memcpy(&hc, raw.data(), sizeof(HostCtrl));
    if (hc.error == ERR_TIMEOUT) return SA_ERR_TIMEOUT;
    if (hc.error != ERR_NONE) return SA_ERR_INTERNAL;
    // Statistics and byte counts from the device records.
    const uint32_t last = hctrl.rs.round;
    if (last >= (uint32_t)DEV_MAX_ROUNDS) return SA_ERR_INTERNAL;
    std::vector<RoundRecord> rec(hctrl.rec, hctrl.rec + last + 1);
    if (last >= 1) {  // the last round's outputs are still in the counters
      RoundRecord &r = rec[last];
      r.m_s = hc.m_s;
      r.g_s = hc.g_s;
      r.m_l = hc.m_l;
      r.g_l = hc.g_l;
      r.upd = hc.upd;
      r.passes = hc.passes;
    }
    for (uint32_t r = 1; r <= last; ++r) {
      const RoundRecord &x = rec[r];
      const uint32_t kbits = x.mL ? W + (x.GL > 1 ? bits_for(x.GL - 1) : 0) : 0;
      const uint64_t rbl = x.mL ? rename_bytes(x.mL, x.m_l, x.g_l) : 0;
      const uint64_t rfb = refine_bytes(x.m - x.mL, x.G - x.GL, x.m_s, x.g_s, x.upd, 2);
      bytes += (x.mL ? (uint64_t)x.passes * 24 * x.mL + 32ull * x.mL : 0) + rbl + rfb + 8ull * x.G +
               12ull * x.upd + (x.m >= bucket_min ? 24ull * x.upd : 0) +
               (x.mL ? 12ull * x.m_l + (x.mL >= bucket_min ? 24ull * x.m_l : 0) : 0);
      launches += 5 + (x.mL ? 12 + MAX_PASSES - 1 : 0) + (x.m >= bucket_min ? 3 : 0) +
                  (x.mL && x.mL >= bucket_min ? 3 : 0);
      if (stats && r < SA_MAX_ROUNDS) {
        stats->active[r] = x.m;
        stats->unique[r] = x.m - (x.m_s + x.m_l);
        stats->passes[r] = x.mL ? x.passes : 0;
        stats->key_bits[r] = kbits;
        stats->groups[r] = x.g_s + x.g_l;
      }
    }
    launches += (last + 1) / 2;  // k_round_end, once per body
    round = last + 1;
    return SA_OK;
  }

  // The groups of the active list `cur` (hc: its counts) copied to the
  // other buffer set in order of their smallest member position, then
  // classified again (large groups, refine tile map); hc is re-read.
  sa_status reorder_groups(int cur, HostCtrl &hc) {
    const uint32_t G = hc.g_next(), m = hc.m_next();
    const int nxt = cur ^ 1;
    const int sms = sm_count();
    // Buffers: the records go to the update queue (free now, 8 N bytes >=
    // 16 G); after the sort only its order (the final value buffer) is
    // needed, so both key buffers are free: the records in the new order
    // go to one, the sizes and scan sums to the other.
    uint4 *info = reinterpret_cast<uint4 *>(upd);
    sa_status s = launch(SA_K_REORDER, 0, 8ull * m + 44ull * G, [&] {
      return launch_group_minpos(act[cur], gstart[cur], gname[cur], ghead[cur], G, ka, va, info,
                                 sms, st);
    });
    if (s != SA_OK) return s;
    bytes += 8ull * m + 44ull * G;
    // By the 32 position bits (constant digits skipped); the order is in the
    // plan's final value buffer.
    s = sort(G, spec_for(32));
    if (s != SA_OK) return s;
    uint4 *info_new = reinterpret_cast<uint4 *>(ka);
    uint32_t *sizes = reinterpret_cast<uint32_t *>(kb);
    uint32_t *sums = sizes + G;
    if (2ull * G > N || inclusive_scan_sums_words(G) + G > 2ull * N) return SA_ERR_INTERNAL;
    s = launch(SA_K_REORDER, 1, 40ull * G, [&] {
      return launch_group_sizes(plan, info, G, info_new, sizes, ctrl, sms, st);
    });
    if (s != SA_OK) return s;
    s = launch(SA_K_REORDER, 2, 8ull * G,
               [&] { return launch_inclusive_scan(sizes, sizes, G, sums, st); });
    if (s != SA_OK) return s;
    RegroupArgs ra{};
    ra.info = info_new;
    ra.act_in = act[cur];
    ra.ends = sizes;
    ra.G = G;
    ra.m = m;
    ra.act_out = act[nxt];
    ra.gstart_out = gstart[nxt];
    ra.gname_out = gname[nxt];
    ra.ghead_out = ghead[nxt];
    ra.ctrl = ctrl;
    s = launch(SA_K_REORDER, 3, 16ull * m + 32ull * G,
               [&] { return launch_regroup(ra, sms, st); });
    if (s != SA_OK) return s;
    bytes += 40ull * G + 8ull * G + 16ull * m + 32ull * G;
    // Every group is now a "refine" group with its final name.
    RoundCounts rc{};
    rc.m_s = m;
    rc.g_s = G;
    CK(cudaMemcpyAsync(&ctrl->rc, &rc, sizeof(rc), cudaMemcpyHostToDevice, st));
    s = classify(nxt, G, 0);
    if (s != SA_OK) return s;
    HostCtrl h2{};
    s = read_ctrl(h2);
    if (s != SA_OK) return s;
    const uint32_t passes = h2.passes;
    s = flush(h2.pass_mask, 0);
    if (s != SA_OK) return s;
    bytes += (uint64_t)passes * 24 * G + 8ull * G;
    h2.passes = hc.passes;
    h2.pass_mask = hc.pass_mask;
    h2.upd = hc.upd;
    hc = h2;
    return SA_OK;
  }

  void record(uint32_t r, uint32_t m, const HostCtrl &hc, uint32_t kbits) {
    if (!stats || r >= SA_MAX_ROUNDS) return;
    stats->active[r] = m;
    stats->unique[r] = m - hc.m_next();
    stats->passes[r] = kbits ? hc.passes : 0;
    stats->key_bits[r] = kbits;
    stats->groups[r] = hc.g_next();
  }

  sa_status run() {
    char label[96];
    snprintf(label, sizeof(label), "gbsa:build n=%llu texts=%u", (unsigned long long)N, S);
    NvtxRange build_range(label);
    const uint32_t N32 = (uint32_t)N;
    carve();
    prof = opt.profile != 0 && stats != nullptr;
    naming = opt.paper_names ? NAMES_HEAD : NAMES_RETAIN;
    mult = opt.multiplier ? opt.multiplier : 2;  // checked by the entry points
    // Clear what must start at zero; the ISA starts all-ones so every end
    // slot reads as the sentinel.
    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    CK(cudaMemsetAsync(st_sort, 0, L.st_sort_bytes, st));
    CK(cudaMemsetAsync(st_ren, 0, L.st_ren_bytes, st));
    CK(cudaMemsetAsync(bytehist, 0, RADIX * 4, st));
    CK(cudaMemsetAsync(isa, 0xFF, (N + S + 1) * 4, st));
    CK(cudaMemcpyAsync(segoff, off.data(), ((size_t)S + 1) * 4, cudaMemcpyHostToDevice, st));

    // ---- A0: alphabet ----
    sa_status s = launch(SA_K_BYTE_HIST, 0, N, [&] {
      return launch_byte_histogram(text, N, bytehist, sm_count(), st);
    });
    if (s != SA_OK) return s;
    uint32_t hh[RADIX];
    CK(fetch(hh, bytehist, sizeof(hh)));
    s = flush(0, 0);
    if (s != SA_OK) return s;
    uint8_t hcode[RADIX];
    uint32_t sigma = 0;
    for (int c = 0; c < RADIX; ++c) {
      hcode[c] = (uint8_t)sigma;  // order-preserving dense code
      if (hh[c]) ++sigma;
    }
    const uint32_t b = std::max<uint32_t>(1, bits_for(sigma - 1));
    const uint32_t segbits = S > 1 ? bits_for(S - 1) : 0;
    // Parameters: the caller's options, else the tuning table's entry for
    // this class (batch or not, bits per character, size), else defaults:
    // 16 keys per radix thread, the 128 x 1024 refine (8 blocks per SM),
    // keys as wide as fit, bucketing from 2^22 pending ISA writes.
    sa_tuned tuned{};
    tuned_params(S > 1, b, N, &tuned);
    bool from_table = false;
    auto pick = [&](uint32_t given, uint32_t table, uint32_t dflt, bool ok_given, bool ok_table) {
      if (given && ok_given) return given;
      if (table && ok_table) {
        from_table = true;
        return table;
      }
      return dflt;
    };
    auto items_ok = [](uint32_t v) { return v == 8 || v == 12 || v == 16; };
    auto shape_ok = [](uint32_t v) { return v >= 1 && v <= (uint32_t)REFINE_SHAPES; };
    sort_items = pick(opt.sort_items, tuned.sort_items, SORT_ITEMS_DEFAULT,
                      items_ok(opt.sort_items), items_ok(tuned.sort_items));
    shape = pick(opt.refine_shape, tuned.refine_shape, 1, shape_ok(opt.refine_shape),
                 shape_ok(tuned.refine_shape)) - 1;
    nominal = REFINE_SHAPE[shape].cap / 2;
    bucket_min = pick(opt.bucket_min, tuned.bucket_min, BUCKET_MIN, true, true);
    const uint32_t h0 = pick(opt.h0_chars, tuned.h0_chars, 0, true, true);
    uint32_t c0 = (64 - segbits) / b;
    if (h0) c0 = std::min(c0, h0);
    const uint32_t cb = c0 * b;
    CK(cudaMemcpyAsync(code, hcode, sizeof(hcode), cudaMemcpyHostToDevice, st));
    bytes += N;
    if (stats) {
      stats->sigma = sigma;
      stats->bits_per_char = b;
      stats->chars_per_key = c0;
      stats->sort_items = sort_items;
      stats->refine_shape = shape + 1;
      stats->bucket_min = bucket_min;
      stats->tuned = from_table ? 1u : 0u;
    }

    // ---- round 0: initial names ----
    snprintf(label, sizeof(label), "gbsa:round 0 m=%u", N32);
    NvtxRange round0_range(label);
    PackArgs pk{};
    pk.text = text;
    pk.N = N32;
    pk.seg_off = segoff;
    pk.S = S;
    pk.code = code;
    pk.b = b;
    pk.c0 = c0;
    pk.cb = cb;
    pk.keys = ka;
    pk.vals = va;
    const uint32_t bits0 = cb + segbits;
    pk.spec = spec_for(bits0);
    pk.hist = hist;
    pk.top_only = (S == 1 && 8 % b == 0 && cb % 8 == 0 && c0 <= 64 && pk.spec.P * 8 == cb) ? 1u : 0u;
    // One text with whole-character digits: the first radix pass forms the
    // keys from the text and the pack only counts (no packed copy written
    // and read back).
    const bool keys_in_pass = pk.top_only && opt.initial_keys != 2;
    if (keys_in_pass) {
      pk.keys = nullptr;
      pk.vals = nullptr;
    }
    const uint64_t pack_bytes = keys_in_pass ? (uint64_t)N : 13ull * N;
    CK(cudaMemsetAsync(hist, 0, (size_t)pk.spec.P * RADIX * 4, st));
    s = launch(SA_K_PACK, 0, pack_bytes, [&] { return launch_pack(pk, st); });
    if (s != SA_OK) return s;
    bytes += pack_bytes;
    inject_pending = opt.inject_stall != 0;
    s = sort(N32, pk.spec, true, 0, keys_in_pass ? &pk : nullptr);
    if (s != SA_OK) return s;
    int cur = 0;  // the active list, group starts and names of this round
    s = rename(N32, true, cb, c0, 0, nullptr, nullptr, 0, cur, ctrl->zero);
    if (s != SA_OK) return s;
    s = classify(cur, N / 2 + 1, N32);
    if (s != SA_OK) return s;
    HostCtrl hc{};
    s = read_ctrl(hc);
    if (s != SA_OK) return s;
    uint32_t m = N32;
    const uint64_t rb0 = rename_bytes(m, hc.m_next(), hc.g_next());
    settle(hc);
    s = flush(hc.pass_mask, rb0);
    if (s != SA_OK) return s;
    record(0, m, hc, bits0);
    bytes += (uint64_t)hc.passes * 24 * m - (keys_in_pass ? 11ull * m : 0ull) + rb0;
    // The unique suffixes' ISA entries are needed only by a later round, the
    // ISA output or the trace; a text resolved in round 0 skips them.
    const bool want_trace = opt.trace_isa && opt.trace_cap > 0 && S == 1;
    if (hc.m_next() > 0 || isa_out || want_trace) {
      // Its records settle with round 0's counts, before round 1 reads new ones.
      s = scatter(hc.upd);
      if (s != SA_OK) return s;
      settle(hc);
    }
    if (want_trace) CK(cudaMemcpyAsync(opt.trace_isa, isa, N * 4, cudaMemcpyDeviceToDevice, st));
    if (hc.m_next() > 0 && opt.group_order != 2) {
      // The later rounds read partner names through the ISA: groups in
      // position order make those reads of neighbouring groups neighbours.
      s = reorder_groups(cur, hc);
      if (s != SA_OK) return s;
      cur ^= 1;
    }
    round0_range.end();

    // ---- rounds r >= 1: one doubling step each ----
    const uint32_t W = bits_for(N);  // r2 in [0, N]
    uint64_t h = c0;
    uint32_t round = 1;
    if (hc.m_next() > 0 && device_rounds_wanted()) {
      // The whole loop as one graph launch; rounds, statistics and byte
      // counts come back from the device records.
      s = run_device_rounds(hc, W, (uint32_t)c0, cur, round);
      if (s != SA_OK) return s;
      hc = HostCtrl{};  // no suffix left active
    }
    while (hc.m_next() > 0) {
      if (round >= SA_MAX_ROUNDS || h > N) return SA_ERR_INTERNAL;
      m = hc.m_next();
      snprintf(label, sizeof(label), "gbsa:round %u m=%u", round, m);
      NvtxRange round_range(label);
      const uint32_t G = hc.g_next();
      const uint32_t mL = hc.m_large(), GL = hc.g_large();
      const int nxt = cur ^ 1;
      CK(cudaMemsetAsync(&ctrl->rc, 0, sizeof(RoundCounts), st));
      // Large groups: keys for the global radix sort (gathered before any
      // name of this round changes).
      uint32_t kbits = 0;
      if (mL > 0) {
        GatherLargeArgs ga{};
        ga.act = act[cur];
        ga.gstart = gstart[cur];
        ga.lg = lg;
        ga.loff = loff;
        ga.mL = mL;
        ga.GL = GL;
        ga.h = (uint32_t)h;
        ga.W = W;
        ga.mult = mult;
        ga.isa = isa;
        ga.isa_len = N + S + 1;
        ga.keys = ka;
        ga.vals = va;
        // a > 2: the queued-update list and the next active list are free
        // until the refine below, and hold the per-item keys until then.
        ga.key1_stash = upd;
        ga.sec_stash = act[nxt];
        const uint64_t gb = mult == 2 ? 24ull * mL : (32ull + 4ull * (mult - 1) + 16ull) * mL;
        s = launch(SA_K_GATHER, 0, gb, [&] { return launch_gather_large(ga, st); });
        if (s != SA_OK) return s;
        bytes += gb;
        kbits = W + (GL > 1 ? bits_for(GL - 1) : 0);
        if (mult > 2) {
          // LSD over the tuple: later partners first, then (group, r2).
          s = sort(mL, spec_for(mult == 4 ? 2 * W : W), false, 1);
          if (s != SA_OK) return s;
          WideArgs wa{};
          wa.plan = plan;
          wa.m = m;
          wa.mL = mL;
          wa.GL = GL;
          wa.W = W;
          wa.act = act[cur];
          wa.gstart = gstart[cur];
          wa.lg = lg;
          wa.loff = loff;
          wa.key1_stash = upd;
          wa.sec_stash = act[nxt];
          wa.ka = ka;
          wa.kb = kb;
          wa.va = va;
          wa.ctrl = ctrl;
          s = launch(SA_K_GATHER, 1, 24ull * mL, [&] { return launch_wide_rekey(wa, st); });
          if (s != SA_OK) return s;
          s = sort(mL, spec_for(kbits));
          if (s != SA_OK) return s;
          s = launch(SA_K_GATHER, 2, 40ull * mL, [&] { return launch_wide_finish(wa, st); });
          if (s != SA_OK) return s;
          bytes += 64ull * mL;
        } else {
          s = sort(mL, spec_for(kbits));
          if (s != SA_OK) return s;
        }
      }
      // Small groups: refined tile by tile; name changes are queued.
      RefineArgs rf{};
      rf.act = act[cur];
      rf.gstart = gstart[cur];
      rf.gname = gname[cur];
      rf.ghead = ghead[cur];
      rf.naming = naming;
      rf.tfirst = tfirst;
      rf.m = m;
      rf.G = G;
      rf.shape = shape;
      rf.tiles = (m + nominal - 1) / nominal;
      rf.h = (uint32_t)h;
      rf.W = W;
      rf.mult = mult;
      rf.isa = isa;
      rf.isa_len = N + S + 1;
      rf.N = N32;
      rf.sa = sa;
      rf.seg_off = segoff;
      rf.S = S;
      rf.act_out = act[nxt];
      rf.gstart_out = gstart[nxt];
      rf.gname_out = gname[nxt];
      rf.ghead_out = ghead[nxt];
      rf.upd = upd;
      rf.ctrl = ctrl;
      s = launch(SA_K_REFINE, 0, 0, [&] { return launch_refine(rf, st); });
      if (s != SA_OK) return s;
      if (mL > 0) {
        s = rename(mL, false, 0, 0, W, lbase, lold, GL, nxt, &ctrl->rc.m_s, mult > 2);
        if (s != SA_OK) return s;
      }
      s = scatter(m);
      if (s != SA_OK) return s;
      s = classify(nxt, G, mL);
      if (s != SA_OK) return s;
      if (opt.trace_isa && round < opt.trace_cap && S == 1)
        CK(cudaMemcpyAsync(opt.trace_isa + (size_t)round * N, isa, N * 4,
                           cudaMemcpyDeviceToDevice, st));
      uint32_t p1[2] = {0, 0};  // the first sort's (passes, mask) in a-tuple rounds
      if (mL > 0 && mult > 2) CK(cudaMemcpyAsync(p1, pm1, 8, cudaMemcpyDeviceToHost, st));
      s = read_ctrl(hc);
      if (s != SA_OK) return s;
      hc.passes += p1[0];
      // Settle the byte counts that depend on this round's results.
      const uint64_t rbl = mL ? rename_bytes(mL, hc.m_l, hc.g_l) : 0;
      const uint64_t rfb = refine_bytes(m - mL, G - GL, hc.m_s, hc.g_s, hc.upd, mult);
      for (Rec &r : recs)
        if (r.cls == SA_K_REFINE) r.bytes = rfb;
      settle(hc);
      s = flush(hc.pass_mask, rbl, p1[1]);
      if (s != SA_OK) return s;
      record(round, m, hc, kbits);
      bytes += (mL ? (uint64_t)hc.passes * 24 * mL : 0) + rbl + rfb + 8ull * G;
      cur = nxt;
      h *= mult;
      ++round;
    }
    // ---- output ----
    if (isa_out) {
      s = launch(SA_K_OUTPUT, 0, 8ull * N, [&] {
        return launch_isa_to_local(isa, isa_out, N32, segoff, S, st);
      });
      if (s != SA_OK) return s;
      bytes += 8ull * N;
    }
    if (prof) {
      CK(cudaStreamSynchronize(st));
      s = flush(0, 0);
      if (s != SA_OK) return s;
    }
    if (stats) {
      stats->rounds = round;
      stats->bytes_model = bytes;
      stats->launches = launches;
    }
    return SA_OK;
  }
};

sa_status check_offsets(const uint64_t *offsets, uint32_t count) {
  if (!offsets || count == 0) return SA_ERR_INVALID_ARG;
  if (offsets[0] != 0) return SA_ERR_INVALID_ARG;
  for (uint32_t k = 0; k < count; ++k)
    if (offsets[k + 1] < offsets[k]) return SA_ERR_INVALID_ARG;
  if (offsets[count] > SA_MAX_N) return SA_ERR_TOO_LARGE;
  return SA_OK;
}

bool bad_options(const sa_options *opt) {
  if (!opt) return false;
  if (opt->multiplier != 0 && (opt->multiplier < 2 || opt->multiplier > 4)) return true;
  if (opt->sort_items != 0 && opt->sort_items != 8 && opt->sort_items != 12 &&
      opt->sort_items != 16)
    return true;
  if (opt->refine_shape > (uint32_t)REFINE_SHAPES) return true;
  return opt->initial_keys > 2;
}

sa_status run_with_workspace(Build &B, void *workspace, size_t ws_bytes) {
  B.L = make_layout(B.N, B.S);
  if (B.opt.spin_limit) B.spin = B.opt.spin_limit;
  PoolBuf own;
  if (workspace) {
    if (ws_bytes < B.L.total || ((uintptr_t)workspace & 255)) return SA_ERR_OOM;
    B.ws = (uint8_t *)workspace;
  } else {
    own.st = B.st;
    if (pool_alloc(&own.p, B.L.total, B.st) != cudaSuccess) {
      own.p = nullptr;
      cudaGetLastError();
      return SA_ERR_OOM;
    }
    B.ws = (uint8_t *)own.p;
  }
  if (B.stats) memset(B.stats, 0, sizeof(sa_stats));
  return B.run();
}

}  // namespace

// The library's private stream-ordered pool, for the other entry points.
cudaError_t library_pool_alloc(void **p, size_t bytes, cudaStream_t st) {
  return pool_alloc(p, bytes, st);
}

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 1;  // not cached: a later call may succeed
  }
  cache[dev] = n;
  return n;
}

namespace {

// Identity of the CUDA context current on this thread (cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime's driver entry points so that
// the library needs no link against libcuda); 0 when it cannot be told.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace

cudaError_t ensure_smem_attributes(const void *fn, int smem_bytes, bool max_carveout) {
  static std::mutex mu;
  static std::set<std::pair<const void *, unsigned long long>> done;
  const unsigned long long ctx = current_context_id();
  if (ctx) {
    std::lock_guard<std::mutex> g(mu);
    if (done.count({fn, ctx})) return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  if (max_carveout) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  if (ctx) {  // unknown context: set again next time rather than trust a stale entry
    std::lock_guard<std::mutex> g(mu);
    done.insert({fn, ctx});
  }
  return cudaSuccess;
}
}  // namespace gbsa

using namespace gbsa;

GBSA_API size_t sa_workspace_bytes(uint64_t n) { return make_layout(n, 1).total; }

GBSA_API sa_status sa_pool_usage(uint64_t *used, uint64_t *reserved) {
  if (!used || !reserved) return SA_ERR_INVALID_ARG;
  *used = *reserved = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it == g_pools.end()) return SA_OK;  // nothing was ever taken from it
  uint64_t u = 0, r = 0;  // the pool attributes are 64-bit values
  if (cudaMemPoolGetAttribute(it->second, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
      cudaMemPoolGetAttribute(it->second, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  *used = u;
  *reserved = r;
  return SA_OK;
}

GBSA_API sa_status sa_pool_trim(uint64_t keep_bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it == g_pools.end()) return SA_OK;
  if (cudaMemPoolTrimTo(it->second, (size_t)keep_bytes) != cudaSuccess) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  return SA_OK;
}

GBSA_API size_t sa_batched_workspace_bytes(const uint64_t *offsets, uint32_t count) {
  if (check_offsets(offsets, count) != SA_OK) return 0;
  return make_layout(offsets[count], count).total;
}

GBSA_API sa_status sa_build_ex(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                               uint32_t *isa_out, void *workspace, size_t ws_bytes,
                               const sa_options *opt, sa_stats *stats, gbsa_stream_t stream) {
  return gbsa::build_single(text, n, sa_out, isa_out, workspace, ws_bytes, opt, stats, stream,
                            true);
}

namespace gbsa {
sa_status build_single(const uint8_t *text, uint64_t n, uint32_t *sa_out, uint32_t *isa_out,
                       void *workspace, size_t ws_bytes, const sa_options *opt, sa_stats *stats,
                       gbsa_stream_t stream, bool stage_readbacks) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  if (bad_options(opt)) return SA_ERR_INVALID_ARG;
  if (stats) memset(stats, 0, sizeof(sa_stats));
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return SA_OK;
  if (n == 1) {
    if (cudaMemsetAsync(sa_out, 0, 4, st) != cudaSuccess) return SA_ERR_CUDA;
    if (isa_out && cudaMemsetAsync(isa_out, 0, 4, st) != cudaSuccess) return SA_ERR_CUDA;
    if (stats) stats->rounds = 1;
    return SA_OK;
  }
  Build B;
  B.stage_readbacks = stage_readbacks;
  B.text = text;
  B.N = n;
  B.S = 1;
  B.off = {0u, (uint32_t)n};
  B.sa = sa_out;
  B.isa_out = isa_out;
  if (opt) B.opt = *opt;
  B.stats = stats;
  B.st = st;
  return run_with_workspace(B, workspace, ws_bytes);
}
}  // namespace gbsa

GBSA_API sa_status sa_build(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                            gbsa_stream_t stream) {
  return sa_build_ex(text, n, sa_out, nullptr, nullptr, 0, nullptr, nullptr, stream);
}

GBSA_API sa_status sa_build_batched_ex(const uint8_t *texts, const uint64_t *offsets,
                                       uint32_t count, uint32_t *sa_out, void *workspace,
                                       size_t ws_bytes, const sa_options *opt,
                                       sa_stats *stats, gbsa_stream_t stream) {
  sa_status s = check_offsets(offsets, count);
  if (s != SA_OK) return s;
  if (count > (1u << 20)) return SA_ERR_TOO_LARGE;
  if (bad_options(opt)) return SA_ERR_INVALID_ARG;
  const uint64_t N = offsets[count];
  if (stats) memset(stats, 0, sizeof(sa_stats));
  if (N == 0) return SA_OK;
  if (!texts || !sa_out) return SA_ERR_INVALID_ARG;
  Build B;
  B.text = texts;
  B.N = N;
  B.S = count;
  B.off.resize((size_t)count + 1);
  for (uint32_t k = 0; k <= count; ++k) B.off[k] = (uint32_t)offsets[k];
  B.sa = sa_out;
  if (opt) {
    B.opt = *opt;
    B.opt.trace_isa = nullptr;
    B.opt.trace_cap = 0;
  }
  B.stats = stats;
  B.st = (cudaStream_t)stream;
  return run_with_workspace(B, workspace, ws_bytes);
}

GBSA_API sa_status sa_build_batched(const uint8_t *texts, const uint64_t *offsets, uint32_t count,
                                    uint32_t *sa_out, gbsa_stream_t stream) {
  return sa_build_batched_ex(texts, offsets, count, sa_out, nullptr, 0, nullptr, nullptr, stream);
}

// Largest request whose host copies run as kernels (sa_build_host).
constexpr uint64_t HOST_KERNEL_COPY_MAX = 4ull << 20;

GBSA_API sa_status sa_build_host(const uint8_t *host_text, uint64_t n, uint32_t *host_sa,
                                 gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!host_text || !host_sa)) return SA_ERR_INVALID_ARG;
  if (n == 0) return SA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t tb = align256(n), sb = align256(n * 4);
  const size_t wb = sa_workspace_bytes(n);
  PoolBuf buf;
  buf.st = st;
  if (pool_alloc(&buf.p, tb + sb + wb, st) != cudaSuccess) {
    buf.p = nullptr;
    cudaGetLastError();
    return SA_ERR_OOM;
  }
  uint8_t *d_text = (uint8_t *)buf.p;
  uint32_t *d_sa = (uint32_t *)((uint8_t *)buf.p + tb);
  void *d_ws = (uint8_t *)buf.p + tb + sb;
  // Small requests with pinned host buffers copy by kernels, which read and
  // write the buffers through their device mapping: a copy engine runs the
  // copies of all streams in order, so a server's small request would
  // otherwise wait behind the large copies of concurrent builds. Larger or
  // pageable buffers take the copy engine.
  const uint8_t *src_dev = nullptr;
  uint32_t *dst_dev = nullptr;
  if (n <= HOST_KERNEL_COPY_MAX) {
    cudaPointerAttributes at{}, as{};
    if (cudaPointerGetAttributes(&at, host_text) == cudaSuccess &&
        cudaPointerGetAttributes(&as, host_sa) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        as.type == cudaMemoryTypeHost && at.devicePointer && as.devicePointer) {
      src_dev = (const uint8_t *)at.devicePointer;
      dst_dev = (uint32_t *)as.devicePointer;
    }
    cudaGetLastError();  // a pageable pointer is not an error here
  }
  if (src_dev) {
    if (launch_copy_bytes(d_text, src_dev, n, st) != cudaSuccess) return SA_ERR_CUDA;
  } else if (cudaMemcpyAsync(d_text, host_text, n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    return SA_ERR_CUDA;
  }
  sa_status s = sa_build_ex(d_text, n, d_sa, nullptr, d_ws, wb, nullptr, nullptr, stream);
  if (s != SA_OK) return s;
  if (dst_dev) {
    if (launch_copy_words(dst_dev, d_sa, n, st) != cudaSuccess) return SA_ERR_CUDA;
  } else if (cudaMemcpyAsync(host_sa, d_sa, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    return SA_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return SA_ERR_CUDA;
  return SA_OK;
}

GBSA_API sa_status sa_build_batched_host(const uint8_t *const *host_texts, const uint64_t *lengths,
                                         uint32_t *const *host_sas, uint32_t count,
                                         gbsa_stream_t stream) {
  if (count == 0 || !host_texts || !lengths || !host_sas) return SA_ERR_INVALID_ARG;
  if (count > (1u << 20)) return SA_ERR_TOO_LARGE;
  std::vector<uint64_t> off((size_t)count + 1, 0);
  for (uint32_t k = 0; k < count; ++k) {
    if (lengths[k] > SA_MAX_N) return SA_ERR_TOO_LARGE;
    if (lengths[k] > 0 && (!host_texts[k] || !host_sas[k])) return SA_ERR_INVALID_ARG;
    off[k + 1] = off[k] + lengths[k];
    if (off[k + 1] > SA_MAX_N) return SA_ERR_TOO_LARGE;
  }
  const uint64_t N = off[count];
  if (N == 0) return SA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t tb = align256(N), sb = align256(N * 4);
  const size_t wb = sa_batched_workspace_bytes(off.data(), count);
  PoolBuf buf;
  buf.st = st;
  if (pool_alloc(&buf.p, tb + sb + wb, st) != cudaSuccess) {
    buf.p = nullptr;
    cudaGetLastError();
    return SA_ERR_OOM;
  }
  uint8_t *d_text = (uint8_t *)buf.p;
  uint32_t *d_sa = (uint32_t *)((uint8_t *)buf.p + tb);
  void *d_ws = (uint8_t *)buf.p + tb + sb;
  // As in sa_build_host: a small batch whose buffers are all pinned copies
  // by kernels (one launch per SegCopy::MAX texts each way), so it does not
  // queue behind the copy-engine traffic of other streams; otherwise one
  // copy-engine copy per text and direction.
  std::vector<void *> src_dev, dst_dev;
  bool mapped = N <= HOST_KERNEL_COPY_MAX;
  if (mapped) {
    src_dev.assign(count, nullptr);
    dst_dev.assign(count, nullptr);
    for (uint32_t k = 0; k < count && mapped; ++k) {
      if (lengths[k] == 0) continue;
      cudaPointerAttributes at{}, as{};
      mapped = cudaPointerGetAttributes(&at, host_texts[k]) == cudaSuccess &&
               cudaPointerGetAttributes(&as, host_sas[k]) == cudaSuccess &&
               at.type == cudaMemoryTypeHost && as.type == cudaMemoryTypeHost &&
               at.devicePointer && as.devicePointer;
      src_dev[k] = at.devicePointer;
      dst_dev[k] = as.devicePointer;
    }
    cudaGetLastError();  // a pageable pointer is not an error here
  }
  auto kernel_copies = [&](bool to_flat) -> cudaError_t {
    for (uint32_t k0 = 0; k0 < count; k0 += SegCopy::MAX) {
      SegCopy t{};
      t.count = std::min<uint32_t>(SegCopy::MAX, count - k0);
      for (uint32_t j = 0; j < t.count; ++j) t.ext[j] = to_flat ? src_dev[k0 + j] : dst_dev[k0 + j];
      for (uint32_t j = 0; j <= t.count; ++j) t.off[j] = off[k0 + j];
      const cudaError_t e = launch_copy_segments(to_flat ? (void *)d_text : (void *)d_sa, t,
                                                 to_flat ? 1 : 4, to_flat, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (mapped) {
    if (kernel_copies(true) != cudaSuccess) return SA_ERR_CUDA;
  } else {
    for (uint32_t k = 0; k < count; ++k)
      if (lengths[k] && cudaMemcpyAsync(d_text + off[k], host_texts[k], lengths[k],
                                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SA_ERR_CUDA;
  }
  const sa_status s =
      sa_build_batched_ex(d_text, off.data(), count, d_sa, d_ws, wb, nullptr, nullptr, stream);
  if (s != SA_OK) return s;
  if (mapped) {
    if (kernel_copies(false) != cudaSuccess) return SA_ERR_CUDA;
  } else {
    for (uint32_t k = 0; k < count; ++k)
      if (lengths[k] && cudaMemcpyAsync(host_sas[k], d_sa + off[k], lengths[k] * 4,
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SA_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return SA_ERR_CUDA;
  return SA_OK;
}

GBSA_API size_t sa_sort_workspace_bytes(uint64_t m) {
  const uint64_t mm = m ? m : 1;
  const uint64_t tiles = (mm + SORT_TILE_MIN - 1) / SORT_TILE_MIN;
  return align256(sizeof(Ctrl)) + align256(sizeof(SortPlan)) + 2 * align256(MAX_PASSES * RADIX * 4) +
         align256(mm * 8) + align256(mm * 4) + align256(tiles * RADIX * 8);
}

GBSA_API sa_status sa_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t m, uint32_t begin_bit,
                                 uint32_t end_bit, void *workspace, size_t ws_bytes,
                                 gbsa_stream_t stream) {
  if (m > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (begin_bit >= end_bit || end_bit > 64) return SA_ERR_INVALID_ARG;
  if (m > 0 && (!keys || !vals)) return SA_ERR_INVALID_ARG;
  if (m <= 1) return SA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = sa_sort_workspace_bytes(m);
  PoolBuf own;
  uint8_t *ws = (uint8_t *)workspace;
  if (ws) {
    if (ws_bytes < need || ((uintptr_t)ws & 255)) return SA_ERR_OOM;
  } else {
    own.st = st;
    if (pool_alloc(&own.p, need, st) != cudaSuccess) {
      own.p = nullptr;
      cudaGetLastError();
      return SA_ERR_OOM;
    }
    ws = (uint8_t *)own.p;
  }
  const uint64_t tiles = (m + SORT_TILE_MIN - 1) / SORT_TILE_MIN;
  size_t o = 0;
  auto take = [&](size_t bytes) { uint8_t *r = ws + o; o += align256(bytes); return r; };
  Build B;
  B.st = st;
  B.ctrl = (Ctrl *)take(sizeof(Ctrl));
  B.plan = (SortPlan *)take(sizeof(SortPlan));
  B.hist = (uint32_t *)take(MAX_PASSES * RADIX * 4);
  B.dbase = (uint32_t *)take(MAX_PASSES * RADIX * 4);
  B.kb = (uint64_t *)take(m * 8);
  B.vb = (uint32_t *)take(m * 4);
  B.st_sort = (uint64_t *)take(tiles * RADIX * 8);
  B.ka = keys;
  B.va = vals;
  CK(cudaMemsetAsync(B.ctrl, 0, sizeof(Ctrl), st));
  CK(cudaMemsetAsync(B.st_sort, 0, tiles * RADIX * 8, st));
  DigitSpec spec{};
  const uint32_t span = end_bit - begin_bit;
  spec.P = (span + RADIX_BITS - 1) / RADIX_BITS;
  for (uint32_t p = 0; p < spec.P; ++p) {
    spec.shift[p] = (uint8_t)(begin_bit + p * RADIX_BITS);
    spec.bits[p] = (uint8_t)std::min<uint32_t>(RADIX_BITS, end_bit - spec.shift[p]);
  }
  sa_status s = B.sort((uint32_t)m, spec);
  if (s != SA_OK) return s;
  CK(launch_copy_back(B.plan, keys, vals, (uint32_t)m, sm_count(), st));
  HostCtrl hc{};
  return B.read_ctrl(hc);
}

GBSA_API const char *sa_status_string(sa_status s) {
  switch (s) {
    case SA_OK: return "SA_OK";
    case SA_ERR_INVALID_ARG: return "SA_ERR_INVALID_ARG";
    case SA_ERR_TOO_LARGE: return "SA_ERR_TOO_LARGE";
    case SA_ERR_OOM: return "SA_ERR_OOM";
    case SA_ERR_CUDA: return "SA_ERR_CUDA";
    case SA_ERR_TIMEOUT: return "SA_ERR_TIMEOUT";
    case SA_ERR_INTERNAL: return "SA_ERR_INTERNAL";
  }
  return "SA_ERR_UNKNOWN";
}
