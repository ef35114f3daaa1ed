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

// Device-resident control block of one build (cleared at build start).
struct Ctrl {
  uint32_t error;      // first DevError raised by any kernel
  uint32_t err_where;  // kernel id that raised it
  uint32_t m_next;     // active suffixes after the last rename
  uint32_t g_next;     // groups among them
  uint32_t passes;     // radix passes the last plan kept
  uint32_t pass_mask;  // bit p set iff pass p of the last plan was kept
  uint32_t pad[2];
  uint32_t tile_ctr[TILE_COUNTERS];  // one dynamic tile counter per launch
};

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
};

// Digit positions of one sort: pass p covers key bits [shift[p], shift[p]+bits[p]).
struct DigitSpec {
  uint32_t P;
  uint8_t shift[MAX_PASSES];
  uint8_t bits[MAX_PASSES];
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

}  // namespace gbsa
