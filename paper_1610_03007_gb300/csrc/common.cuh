// Shared device-side definitions of the gbsa kernels (sm_103a).
//
// Decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", NVIDIA TR 2016) is used by the radix passes and
// by the rename/compaction kernel. Each tile publishes a 64-bit status word
//   [63:34] epoch (30 bits) | [33:32] state | [31:0] value
// in one store, so value and state are always read together. The epoch is
// unique per launch within a build; a word whose epoch differs from the
// current launch reads as "not ready", so status arrays need clearing only
// once per build. Tiles are numbered by an atomic counter in launch order,
// so every predecessor a tile waits on is already resident or finished.
// Every wait is bounded: after `spin_limit` polls (or when another tile has
// already failed) the kernel records ERR_TIMEOUT in the control block and
// returns without writing its outputs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbsa {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 8;  // 64-bit keys, 8-bit digits
constexpr uint32_t EPOCH_MASK = 0x3FFFFFFFu;
constexpr uint32_t ST_AGG = 1;  // value = the tile's own aggregate
constexpr uint32_t ST_INC = 2;  // value = inclusive prefix through the tile
constexpr int TILE_COUNTERS = 1024;

enum DevError : uint32_t { ERR_NONE = 0, ERR_TIMEOUT = 1, ERR_INTERNAL = 2 };

// Counters of one doubling round (cleared when the round starts). The next
// active list is written by two producers: the small-group refine first
// (survivors [0, m_s), groups [0, g_s)), then the rename of round 0 or of
// the large groups (survivors [m_s, m_s + m_l), groups [g_s, g_s + g_l)).
struct RoundCounts {
  uint32_t m_s, g_s;        // survivors / groups written by the refine
  uint32_t m_l, g_l;        // survivors / groups written by the rename
  uint32_t upd;             // deferred ISA updates queued by the refine
  uint32_t pad;
  unsigned long long large; // classify: (large groups << 32) | large items
};

// Digit positions of one sort: pass p covers key bits [shift[p], shift[p]+bits[p]).
struct DigitSpec {
  uint32_t P;
  uint8_t shift[MAX_PASSES];
  uint8_t bits[MAX_PASSES];
};

constexpr int DEV_MAX_ROUNDS = 64;  // SA_MAX_ROUNDS

// Device-driven rounds (rounds >= 1 run as one CUDA graph with no host
// round trip): the sizes the host round driver otherwise passes as kernel
// arguments. k_round_begin writes them from the previous round's counters;
// every kernel of a round reads them here.
struct RoundState {
  uint32_t m, G, mL, GL;  // active items and groups; items and groups of the large groups
  uint32_t tiles;         // refine tiles: ceil(m / refine window)
  uint32_t h;             // characters the current names resolve (partner offset)
  uint32_t h_next;        // h of the next round
  uint32_t round;         // index of the current round
  uint32_t live;          // 0 once no suffix is active or an error was raised
  uint32_t epoch;         // look-back epoch base of the round's launches
  uint32_t bucket_upd;    // 1: the round's queued ISA updates are bucketed by position
  uint32_t bucket_surv;   // 1: the large groups' ISA entries are bucketed by position
  DigitSpec spec;         // digits of the large-group sort
};

// What one device-driven round saw (the host fills sa_stats from it).
struct RoundRecord {
  uint32_t m, G, mL, GL;              // inputs
  uint32_t m_s, g_s, m_l, g_l, upd;   // outputs (RoundCounts of the round)
  uint32_t passes;                    // radix passes the large-group sort kept
};

// Device-resident control block of one build (cleared at build start).
struct Ctrl {
  uint32_t error;      // first DevError raised by any kernel
  uint32_t err_where;  // kernel id that raised it
  uint32_t passes;     // radix passes the last plan kept
  uint32_t pass_mask;  // bit p set iff pass p of the last plan was kept
  RoundCounts rc;
  uint32_t zero[4];    // constant zeros (output offsets of round 0)
  uint32_t bucket_total;  // entries a translating position partition kept
  uint32_t tile_ctr[TILE_COUNTERS];  // one dynamic tile counter per launch
  RoundState rs;                     // device-driven rounds only
  RoundRecord rec[DEV_MAX_ROUNDS];
};
static_assert(sizeof(RoundCounts) == 32, "RoundCounts layout");

// Where each radix pass reads and writes; written on the device by the plan
// kernel after the digit histograms are known (constant digits are skipped).
struct SortPlan {
  const uint64_t *ksrc[MAX_PASSES];
  uint64_t *kdst[MAX_PASSES];
  const uint32_t *vsrc[MAX_PASSES];
  uint32_t *vdst[MAX_PASSES];
  uint32_t active[MAX_PASSES];
  uint32_t n_active;
  uint32_t final_idx;  // 0: result in buffer A, 1: in buffer B
  const uint64_t *kfinal;
  const uint32_t *vfinal;
  uint32_t match_mask;  // bit p: pass p ranks with match.any (low-entropy digit)
};

__device__ __forceinline__ uint32_t digit_of(uint64_t key, uint32_t shift, uint32_t bits) {
  return (uint32_t)(key >> shift) & ((1u << bits) - 1u);
}

__device__ __forceinline__ uint64_t status_word(uint32_t epoch, uint32_t state, uint32_t value) {
  return ((uint64_t)(((epoch & EPOCH_MASK) << 2) | state) << 32) | value;
}

__device__ __forceinline__ void status_store(uint64_t *p, uint64_t w) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ uint64_t status_load(const uint64_t *p) {
  uint64_t w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

__device__ __forceinline__ uint32_t load_volatile_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void raise_error(Ctrl *ctrl, uint32_t code, uint32_t where) {
  if (atomicCAS(&ctrl->error, 0u, code) == 0u) ctrl->err_where = where;
}

__device__ __forceinline__ bool has_error(const Ctrl *ctrl) {
  return load_volatile_u32(&ctrl->error) != 0u;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---- TMA bulk copies (global -> shared) behind an mbarrier -----------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory (and
// those of the threads a barrier ordered before it) before its following
// async-proxy (TMA) accesses: a bulk copy into a buffer that ordinary
// stores wrote before.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 1-D bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier guarding this block's own
// bulk copies. On expiry the error is recorded, and the wait continues (again
// bounded) so the block never leaves while its copies may still land.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, Ctrl *ctrl,
                                                  uint32_t spin_limit) {
  for (uint32_t i = 0; i < spin_limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(256);
  }
  raise_error(ctrl, ERR_TIMEOUT, 5);
  for (uint32_t i = 0; i < spin_limit; ++i) {
    if (mbar_try_wait(bar, parity)) return false;
    __nanosleep(1024);
  }
  return false;
}

// Waits until status word `p` carries this launch's epoch and a non-zero
// state; returns false if the wait gave up (bounded).
__device__ __forceinline__ bool status_wait(const uint64_t *p, uint32_t epoch, uint64_t &w,
                                            Ctrl *ctrl, uint32_t spin_limit) {
  uint32_t spins = 0;
  uint32_t ns = 32;
  for (;;) {
    w = status_load(p);
    uint32_t tag = (uint32_t)(w >> 32);
    if ((tag >> 2) == (epoch & EPOCH_MASK) && (tag & 3u) != 0u) return true;
    if (++spins > spin_limit) {
      raise_error(ctrl, ERR_TIMEOUT, 1);
      return false;
    }
    if ((spins & 15u) == 0u && has_error(ctrl)) return false;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
}

// Sequential look-back of one thread over tiles tile-1, tile-2, ...:
// combines predecessor values with `op` until an inclusive prefix is found.
// Returns false if a wait gave up.
template <class Op>
__device__ __forceinline__ bool look_back(const uint64_t *status, uint32_t stride, uint32_t slot,
                                          uint32_t tile, uint32_t epoch, Op op, uint32_t &carry,
                                          Ctrl *ctrl, uint32_t spin_limit) {
  int64_t pred = (int64_t)tile - 1;
  while (pred >= 0) {
    uint64_t w;
    if (!status_wait(status + (size_t)pred * stride + slot, epoch, w, ctrl, spin_limit)) return false;
    carry = op(carry, (uint32_t)w);
    if (((uint32_t)(w >> 32) & 3u) == ST_INC) return true;
    --pred;
  }
  return true;
}

// Look-back with an associative operator that reads a window of W
// predecessors per round trip (W independent loads): a chain of tiles that
// have published only their aggregates costs 1/W of the dependent
// latencies. Bounded like status_wait.
template <int W, class Op>
__device__ __forceinline__ bool look_back_w(const uint64_t *status, uint32_t stride, uint32_t slot,
                                            uint32_t tile, uint32_t epoch, Op op, uint32_t &carry,
                                            Ctrl *ctrl, uint32_t spin_limit) {
  int64_t p = (int64_t)tile - 1;
  uint32_t spins = 0, ns = 32;
  const uint32_t ep = epoch & EPOCH_MASK;
  while (p >= 0) {
    uint64_t w[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
      w[k] = (p - k >= 0) ? status_load(status + (size_t)(p - k) * stride + slot) : 0ull;
    int used = 0;
    bool done = false, blocked = false;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      if (!done && !blocked && p - k >= 0) {
        const uint32_t tag = (uint32_t)(w[k] >> 32);
        if ((tag >> 2) != ep || (tag & 3u) == 0u) {
          blocked = true;
        } else {
          carry = op(carry, (uint32_t)w[k]);
          ++used;
          if ((tag & 3u) == ST_INC) done = true;
        }
      }
    }
    if (done) return true;
    p -= used;
    if (used == 0) {
      if (++spins > spin_limit) {
        raise_error(ctrl, ERR_TIMEOUT, 1);
        return false;
      }
      if ((spins & 15u) == 0u && has_error(ctrl)) return false;
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
  }
  return true;
}

template <class Op>
__device__ __forceinline__ bool look_back4(const uint64_t *status, uint32_t stride, uint32_t slot,
                                           uint32_t tile, uint32_t epoch, Op op, uint32_t &carry,
                                           Ctrl *ctrl, uint32_t spin_limit) {
  return look_back_w<4>(status, stride, slot, tile, epoch, op, carry, ctrl, spin_limit);
}

// Sum look-back that reads a window of 4 predecessors per round trip
// (independent loads), so a chain of tiles that have only published their
// aggregates costs a quarter of the dependent latencies. `stride`/`slot`
// address the status word of this thread's digit in each tile.
__device__ __forceinline__ bool look_back_sum4(const uint64_t *status, uint32_t stride,
                                               uint32_t slot, uint32_t tile, uint32_t epoch,
                                               uint32_t &carry, Ctrl *ctrl, uint32_t spin_limit) {
  int64_t p = (int64_t)tile - 1;
  uint32_t spins = 0, ns = 32;
  const uint32_t ep = epoch & EPOCH_MASK;
  while (p >= 0) {
    uint64_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = (p - k >= 0) ? status_load(status + (size_t)(p - k) * stride + slot) : 0ull;
    int used = 0;
    bool done = false, blocked = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!done && !blocked && p - k >= 0) {
        const uint32_t tag = (uint32_t)(w[k] >> 32);
        if ((tag >> 2) != ep || (tag & 3u) == 0u) {
          blocked = true;
        } else {
          carry += (uint32_t)w[k];
          ++used;
          if ((tag & 3u) == ST_INC) done = true;
        }
      }
    }
    if (done) return true;
    p -= used;
    if (used == 0) {
      if (++spins > spin_limit) {
        raise_error(ctrl, ERR_TIMEOUT, 1);
        return false;
      }
      if ((spins & 15u) == 0u && has_error(ctrl)) return false;
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
  }
  return true;
}

struct OpAdd {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};
struct OpMax {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

// Text of ungapped position (or rank) j: the largest s < S with
// seg_off[s] <= j, so empty texts sharing an offset are skipped.
__device__ __forceinline__ uint32_t segment_of(const uint32_t *seg_off, uint32_t S, uint32_t j) {
  uint32_t lo = 0, hi = S - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(seg_off + mid) <= j)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Stable rank of digit d among the lanes of a warp, plus the warp's running
// per-digit count. Peers holding the same digit are found with a
// shared-memory atomicOr mask (on GB300 about 2.7x the rate of eight
// ballots). `match` (this warp's 256 masks) is all-zero on entry and left
// all-zero; `wh` (this warp's 256 counters) accumulates. Every lane of the
// warp must call it.
__device__ __forceinline__ uint32_t warp_rank_digit(uint32_t d, uint32_t *match, uint16_t *wh,
                                                    uint32_t lane, uint32_t lt) {
  atomicOr(&match[d], 1u << lane);
  __syncwarp();
  const uint32_t peers = match[d];
  const uint32_t before = wh[d];
  __syncwarp();
  const uint32_t lower = peers & lt;
  if (lower == 0) {
    wh[d] = (uint16_t)(before + __popc(peers));
    match[d] = 0u;
  }
  __syncwarp();
  return before + __popc(lower);
}

// The same rank with the peers found by match.any: faster than the masks
// when a warp's digits take few distinct values (their atomics then
// serialise on a few words), slower when they take many.
__device__ __forceinline__ uint32_t warp_rank_digit_match(uint32_t d, uint16_t *wh, uint32_t lt) {
  const uint32_t peers = __match_any_sync(0xffffffffu, d);
  const uint32_t before = wh[d];
  __syncwarp();
  if ((peers & lt) == 0) wh[d] = (uint16_t)(before + __popc(peers));
  __syncwarp();
  return before + __popc(peers & lt);
}

// Local index of gapped position ip: text s occupies the gapped positions
// [seg_off[s] + s, seg_off[s+1] + s) (the slot after it is its end
// sentinel), so gapped starts increase strictly even across empty texts.
__device__ __forceinline__ uint32_t local_index(uint32_t ip, const uint32_t *seg_off, uint32_t S) {
  if (S <= 1) return ip;
  uint32_t lo = 0, hi = S - 1;  // the last s with seg_off[s] + s <= ip
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(seg_off + mid) + mid <= ip)
      lo = mid;
    else
      hi = mid - 1;
  }
  return ip - (__ldg(seg_off + lo) + lo);
}

// Inclusive warp scan.
template <class Op>
__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v, Op op) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v = op(v, o);
  }
  return v;
}

// Exclusive block scan for BLOCK threads (BLOCK/32 <= 32). `tmp` holds at
// least BLOCK/32 + 1 words of shared memory. Returns the exclusive prefix
// (identity for thread 0) and the block total in `total`.
template <int BLOCK, class Op>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, Op op, uint32_t identity,
                                                    uint32_t *tmp, uint32_t &total) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = warp_inclusive(v, op);
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < WARPS ? tmp[lane] : identity;
    uint32_t ti = warp_inclusive(t, op);
    if (lane < WARPS) tmp[lane] = ti;  // inclusive over warps
  }
  __syncthreads();
  uint32_t warp_prefix = warp == 0 ? identity : tmp[warp - 1];
  total = tmp[WARPS - 1];
  uint32_t excl_in_warp = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl_in_warp = identity;
  uint32_t r = op(warp_prefix, excl_in_warp);
  __syncthreads();  // tmp may be reused by the caller
  return r;
}

// Exclusive suffix minimum over the threads of a block: min of v over the
// threads with a larger index (0xFFFFFFFF for the last thread). `tmp`
// holds at least BLOCK/32 + 1 words of shared memory.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_suffix_min_exclusive(uint32_t v, uint32_t *tmp) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_down_sync(0xffffffffu, incl, d);
    if (lane + d < 32) incl = o < incl ? o : incl;
  }
  if (lane == 0) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < WARPS ? tmp[lane] : 0xFFFFFFFFu;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_down_sync(0xffffffffu, t, d);
      if (lane + d < 32) t = o < t ? o : t;
    }
    if (lane < WARPS) tmp[lane] = t;  // suffix over warps, inclusive
  }
  __syncthreads();
  const uint32_t later = warp + 1 < WARPS ? tmp[warp + 1] : 0xFFFFFFFFu;
  uint32_t next = __shfl_down_sync(0xffffffffu, incl, 1);
  if (lane == 31) next = 0xFFFFFFFFu;
  const uint32_t r = later < next ? later : next;
  __syncthreads();
  return r;
}

}  // namespace gbsa
