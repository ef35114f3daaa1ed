// Steps A3 + A4 — new names, uniqueness and discarding, in one pass over the
// sorted (key, position) pairs of a round.
//
//  - Boundary flag (CmpName, Section 2.1, Algorithm 2): f_j = 1 iff key_j
//    differs from key_{j-1} (f_0 = 1). In round 0 every tail suffix (fewer
//    than c0 characters left; see k_pack.cu) and the item after it also get
//    f = 1, so each tail is a group of its own.
//  - Head rank (PrefixSum with max, Algorithm 1): s_j = max over j' <= j of
//    (f_j' ? j' : 0). It is read only where f_j = 1 (a unique item, or the
//    head of a surviving group, whose members take their names from the
//    head's record in k_classify / k_apply_names), and there s_j = j, so the
//    max-scan itself is never materialised.
//  - New name (NameDiscarding, Algorithms 5/6, in head-rank form): round 0
//    new_j = s_j; later rounds new_j = r + (s_j - group start), stored as
//    base[g] + s_j with base[g] = r - group start of group g (this kernel
//    renames the large groups after rounds >= 1; k_refine.cu renames the
//    small ones).
//  - Unique (Algorithm 6): new_j differs from both neighbours, i.e.
//    f_j and f_{j+1} (f_m = 1).
//  - Discarding (Algorithm 5): a unique item is final: it writes SA[pos] = i
//    and queues ISA[i] = pos (applied by k_scatter_updates when a later
//    round or an output reads the ISA); the others are compacted, in order, into
//    the next active list with their group ordinal g', and each group's head
//    records its start in that list, its head rank and its parent's name
//    (the group's own name and the ISA entries of its members follow in
//    k_classify / k_apply_names, once group sizes are known).
//    Offsets come from two device-wide sums (survivors, group heads) with
//    decoupled look-back, added to output offsets read from the device (the
//    small-group refine of the same round writes first).
//
// All partner names of a round were gathered by an earlier kernel, so the
// ISA writes here never race with reads of the same round.
//
// Bound: HBM. 12 bytes read per item; per unique item 4 bytes of SA (in
// rank order: sequential in round 0) and 8 queued bytes; 8 bytes per
// survivor.
#include "launch.h"

namespace gbsa {

constexpr int RN_BLOCK = 256;
constexpr int RN_ITEMS = GBSA_RN_ITEMS;
constexpr int RN_TILE = RN_BLOCK * RN_ITEMS;
constexpr int RN_WARPS = RN_BLOCK / 32;
#ifndef GBSA_RN_LB_WINDOW
#define GBSA_RN_LB_WINDOW 4
#endif
// Predecessors read per look-back round trip.
constexpr int RN_LB_WINDOW = GBSA_RN_LB_WINDOW;
static_assert(RN_TILE == RENAME_TILE, "tile size mismatch");

// Item e of a tile (e = k * 256 + thread, k < RN_ITEMS) is the k-th item of
// its thread: a warp's 32 lanes hold 32 consecutive items, so neighbours
// are one shuffle away, counts come from ballots, and every output is
// written by consecutive lanes to consecutive (or, for the compacted lists,
// ballot-ranked) addresses straight from registers. The tile's order is
// row-major: (k, warp, lane). Its segment (k, warp) of 32 items has its
// counts in `cnt` and, after one warp's scan, its exclusive prefixes in
// `pre`.
constexpr int RN_SEGS = RN_ITEMS * RN_WARPS;
static_assert(RN_SEGS == 64, "one scanning warp holds two segments per lane (8 items)");

struct RnSmem {
  // Per segment: unique | survivors << 21 | surviving-group heads << 42.
  unsigned long long cnt[RN_SEGS];
  unsigned long long pre[RN_SEGS];
  uint32_t carry[2];  // survivors and groups of the tiles before this one
  uint32_t tile, bail, upd_base;
};

__device__ __forceinline__ uint32_t lanemask_le_u32() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}

// One rename tile; every thread of the block calls it. Returns false when
// the block must stop (a wait gave up). m, g_in and epoch as in the kernel.
__device__ __forceinline__ bool rename_tile(RnSmem &S, const RenameArgs &a, const uint32_t tile,
                                            const uint32_t m, const uint32_t g_in,
                                            const uint32_t epoch) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t *__restrict__ K = a.plan->kfinal;
  const uint32_t *__restrict__ V = a.plan->vfinal;
  // a-tuple rounds: items with equal keys are still apart if their later
  // partners differ (sorted alongside, in the other key buffer).
  const uint64_t *SEC = a.sec_buf[0] ? a.sec_buf[a.plan->final_idx ^ 1u] : nullptr;
  const uint32_t base = tile * RN_TILE;
  const uint32_t count = min((uint32_t)RN_TILE, m - base);

  // Round 0: does the suffix at gapped position v (key k) have fewer than
  // c0 characters left in its text?
  auto tail = [&](uint64_t k, uint32_t v) -> bool {
    if (a.S <= 1) return a.N - v < a.c0;  // one text: gapped = plain positions
    const uint32_t s = (uint32_t)(k >> a.cb);
    const uint32_t off = __ldg(a.seg_off + s);
    const uint32_t len = __ldg(a.seg_off + s + 1) - off;
    return len - (v - (off + s)) < a.c0;
  };

  uint64_t key[RN_ITEMS];
  uint32_t val[RN_ITEMS];
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    const uint32_t e = k * RN_BLOCK + tid;
    key[k] = e < count ? K[base + e] : 0ull;
    val[k] = e < count ? V[base + e] : 0u;
  }
  // Boundary flags f (item j starts a new group: Algorithm 2's CmpName, and
  // in round 0 the tail rule) and fn = f of the next item, as bit k of each.
  uint32_t fbits = 0, fnbits = 0;
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    const uint32_t e = k * RN_BLOCK + tid;
    const uint32_t j = base + e;  // < 2^32: m fits 32 bits
    const bool valid = e < count;
    const bool tl = a.round0 && valid && tail(key[k], val[k]);
    const uint64_t sc = SEC && valid ? SEC[j] : 0ull;
    // the item before: lane - 1, or (lane 0) read from memory
    uint64_t pk = __shfl_up_sync(0xffffffffu, key[k], 1);
    bool ptl = __shfl_up_sync(0xffffffffu, (uint32_t)tl, 1) != 0u;
    uint64_t ps = __shfl_up_sync(0xffffffffu, sc, 1);
    if (lane == 0 && valid && j > 0) {
      pk = K[j - 1];
      ptl = a.round0 && tail(pk, V[j - 1]);
      ps = SEC ? SEC[j - 1] : 0ull;
    }
    const bool f = !valid || j == 0 || key[k] != pk || (a.round0 && (tl || ptl)) ||
                   (SEC && sc != ps);
    // the item after: lane + 1's flag, or (lane 31) computed from memory
    bool fn = __shfl_down_sync(0xffffffffu, (uint32_t)f, 1) != 0u;
    if (lane == 31 && valid) {
      if (j + 1 >= m) {
        fn = true;
      } else {
        const uint64_t nk = K[j + 1];
        fn = nk != key[k] || (a.round0 && (tl || tail(nk, V[j + 1]))) ||
             (SEC && SEC[j + 1] != sc);
      }
    }
    if (f) fbits |= 1u << k;
    if (fn) fnbits |= 1u << k;
  }
  // Per segment: unique items (f and fn), survivors, heads of surviving
  // groups (f, not fn).
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    const bool valid = (uint32_t)(k * RN_BLOCK + tid) < count;
    const bool f = (fbits >> k) & 1u, fn = (fnbits >> k) & 1u;
    const uint32_t U = __ballot_sync(0xffffffffu, valid && f && fn);
    const uint32_t Sv = __ballot_sync(0xffffffffu, valid && !(f && fn));
    const uint32_t H = __ballot_sync(0xffffffffu, valid && f && !fn);
    if (lane == 0)
      S.cnt[k * RN_WARPS + warp] = (unsigned long long)__popc(U) |
                                   ((unsigned long long)__popc(Sv) << 21) |
                                   ((unsigned long long)__popc(H) << 42);
  }
  __syncthreads();
  // One warp scans the segments (two per lane), publishes the tile's
  // survivors and groups for the device-wide sums, and reserves the queued
  // updates' space.
  if (warp == 0) {
    const unsigned long long c0 = S.cnt[2 * lane], c1 = S.cnt[2 * lane + 1];
    unsigned long long incl = c0 + c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += o;
    }
    const unsigned long long tot = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned long long ex = incl - c0 - c1;
    S.pre[2 * lane] = ex;
    S.pre[2 * lane + 1] = ex + c0;
    const uint32_t tot_u = (uint32_t)(tot & 0x1FFFFFu);
    const uint32_t tot_s = (uint32_t)((tot >> 21) & 0x1FFFFFu), tot_h = (uint32_t)(tot >> 42);
    if (lane < 2)
      status_store(a.status + (uint64_t)tile * 2 + lane,
                   status_word(epoch, tile == 0 ? ST_INC : ST_AGG, lane == 0 ? tot_s : tot_h));
    if (lane == 2) S.upd_base = tot_u ? atomicAdd(&a.ctrl->rc.upd, tot_u) : 0u;
  }
  __syncthreads();

  // Unique items (Algorithm 5 discards them): name = rank, final. The
  // queued ISA entry and the SA entry (the index local to the suffix's own
  // text) need no offsets from earlier tiles, so they go before the
  // look-back.
  const uint32_t lt = lanemask_lt(), le = lanemask_le_u32();
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    const uint32_t e = k * RN_BLOCK + tid;
    const bool valid = e < count;
    const bool f = (fbits >> k) & 1u, fn = (fnbits >> k) & 1u;
    const bool uniq = valid && f && fn;
    const uint32_t U = __ballot_sync(0xffffffffu, uniq);
    if (!uniq) continue;
    const uint32_t j = base + e, ip = val[k];
    const uint32_t g = a.round0 ? 0u : (uint32_t)(key[k] >> a.W);
    if (!a.round0 && g >= g_in) {  // never taken unless a logic error
      raise_error(a.ctrl, ERR_INTERNAL, 4);
      continue;
    }
    const uint32_t head = a.round0 ? j : __ldg(a.base_in + g) + j;
    if (head >= a.N || ip >= a.isa_len) {  // never taken unless a logic error
      raise_error(a.ctrl, ERR_INTERNAL, 3);
      continue;
    }
    const uint32_t slot = S.upd_base + (uint32_t)(S.pre[k * RN_WARPS + warp] & 0x1FFFFFu) +
                          __popc(U & lt);
    a.upd[slot] = ((uint64_t)head << 32) | ip;
    uint32_t local = ip;
    if (a.S > 1) {
      if (a.round0) {
        const uint32_t s = (uint32_t)(key[k] >> a.cb);
        local = ip - (__ldg(a.seg_off + s) + s);
      } else {
        local = local_index(ip, a.seg_off, a.S);
      }
    }
    a.sa[head] = local;
  }

  // Device-wide offsets of the tile's survivors and groups.
  if (tid < 2) {
    uint32_t carry = 0;
    bool ok = true;
    if (tile > 0) {
      ok = look_back_w<RN_LB_WINDOW>(a.status, 2, tid, tile, epoch, OpAdd(), carry, a.ctrl,
                                     a.spin_limit);
      if (ok) {
        const unsigned long long tot = S.pre[RN_SEGS - 1] + S.cnt[RN_SEGS - 1];
        const uint32_t mine =
            tid == 0 ? (uint32_t)((tot >> 21) & 0x1FFFFFu) : (uint32_t)(tot >> 42);
        status_store(a.status + (uint64_t)tile * 2 + tid, status_word(epoch, ST_INC, carry + mine));
      }
    }
    if (!ok) S.bail = 1;
    S.carry[tid] = carry;
  }
  __syncthreads();
  if (S.bail) return false;
  const uint32_t m_off = __ldg(a.off_in), g_off = __ldg(a.off_in + 1);
  const uint32_t surv0 = m_off + S.carry[0], grp0 = g_off + S.carry[1];
  if (tid == 0 && base + count == m) {
    const unsigned long long tot = S.pre[RN_SEGS - 1] + S.cnt[RN_SEGS - 1];
    a.cnt_out[0] = S.carry[0] + (uint32_t)((tot >> 21) & 0x1FFFFFu);
    a.cnt_out[1] = S.carry[1] + (uint32_t)(tot >> 42);
  }
  // Survivors: compacted, in order, into the next active list with their
  // group ordinal g' (the surviving-group heads at or before them, minus
  // one); each group's head records its start there, its head rank (its own
  // sorted index) and its parent's name. Their names and ISA entries follow
  // once the group sizes are known (k_classify, k_apply_names).
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    const uint32_t e = k * RN_BLOCK + tid;
    const bool valid = e < count;
    const bool f = (fbits >> k) & 1u, fn = (fnbits >> k) & 1u;
    const bool surv = valid && !(f && fn);
    const uint32_t Sv = __ballot_sync(0xffffffffu, surv);
    const uint32_t H = __ballot_sync(0xffffffffu, valid && f && !fn);
    if (!surv) continue;
    const unsigned long long pr = S.pre[k * RN_WARPS + warp];
    const uint32_t sidx = (uint32_t)((pr >> 21) & 0x1FFFFFu) + __popc(Sv & lt);
    const uint32_t ord = grp0 + (uint32_t)(pr >> 42) + __popc(H & le) - 1u;
    const uint32_t ip = val[k];
    if (ip >= a.isa_len) {  // never taken unless a logic error
      raise_error(a.ctrl, ERR_INTERNAL, 3);
      continue;
    }
    a.act_out[surv0 + sidx] = ((uint64_t)ord << 32) | ip;
    if (f) {  // the head of a surviving group
      const uint32_t j = base + e;
      const uint32_t g = a.round0 ? 0u : (uint32_t)(key[k] >> a.W);
      if (!a.round0 && g >= g_in) {  // never taken unless a logic error
        raise_error(a.ctrl, ERR_INTERNAL, 4);
        continue;
      }
      const uint32_t head = a.round0 ? j : __ldg(a.base_in + g) + j;
      if (head >= a.N) {  // never taken unless a logic error
        raise_error(a.ctrl, ERR_INTERNAL, 3);
        continue;
      }
      a.gstart_out[ord] = surv0 + sidx;
      a.ghead_out[ord] = head;
      a.gold_out[ord] = a.round0 ? NO_NAME : __ldg(a.old_in + g);
    }
  }
  return true;
}

// 8 items per thread, 4 blocks of 256 threads per SM. Tiles are taken from the launch's
// counter until it passes the last one, so any grid works (a grid smaller
// than the tile count makes the blocks persistent); in device-driven
// rounds the item and group counts and the epoch base come from the round
// state.
template <bool PERSIST>
__global__ void __launch_bounds__(RN_BLOCK, 4) k_rename(RenameArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  RnSmem &S = *reinterpret_cast<RnSmem *>(smem_raw);
  uint32_t m = a.m, g_in = a.g_in, epoch = a.epoch;
  if (a.rs) {
    if (!a.rs->live) return;
    m = a.rs->mL;
    g_in = a.rs->GL;
    epoch = a.rs->epoch + a.epoch;
  }
  const uint32_t tiles = (uint32_t)(((uint64_t)m + RN_TILE - 1) / RN_TILE);
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      S.tile = atomicAdd(a.tile_ctr, 1u);
      S.bail = has_error(a.ctrl) ? 1u : 0u;
    }
    __syncthreads();
    if (S.bail || S.tile >= tiles) return;
    if (!rename_tile(S, a, S.tile, m, g_in, epoch)) return;
    if constexpr (!PERSIST) return;  // one tile per block: no second claim
    __syncthreads();  // the next tile reuses the shared buffers
  }
}

cudaError_t launch_rename(const RenameArgs &a, cudaStream_t stream) {
  if (a.m == 0) return cudaSuccess;
  const int smem = (int)sizeof(RnSmem);
  // One tile per block unless the grid is capped (persistent blocks loop).
  const uint32_t tiles = (a.m + RN_TILE - 1) / RN_TILE;
  const bool persist = a.grid_cap && tiles > a.grid_cap;
  const void *fn = persist ? reinterpret_cast<const void *>(&k_rename<true>)
                           : reinterpret_cast<const void *>(&k_rename<false>);
  cudaError_t e = ensure_smem_attributes(fn, smem, false);
  if (e != cudaSuccess) return e;
  if (persist)
    k_rename<true><<<a.grid_cap, RN_BLOCK, smem, stream>>>(a);
  else
    k_rename<false><<<tiles, RN_BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace gbsa
