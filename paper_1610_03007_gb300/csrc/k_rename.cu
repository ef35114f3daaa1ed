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

struct RnSmem {
  // Loading: the tile's keys and values; writing: staged queued updates
  // (keys) and, in round 0, the SA entries by tile index (vals).
  uint64_t keys[RN_TILE + RN_TILE / 16];  // element e at e + e/16 (no bank conflicts)
  uint32_t vals[RN_TILE + RN_TILE / 32];  // element e at e + e/32
  uint64_t surv[RN_TILE];                 // staged next-list entries of the survivors
  uint64_t prev_key, next_key;
  uint32_t prev_val, next_val;
  uint32_t tmp[RN_WARPS + 1];
  uint32_t carry[2];
  uint32_t tile, bail, upd_local, upd_base;
};

__device__ __forceinline__ uint32_t kidx(uint32_t e) { return e + (e >> 4); }
__device__ __forceinline__ uint32_t vidx(uint32_t e) { return e + (e >> 5); }

// One rename tile; every thread of the block calls it. Returns false when
// the block must stop (a wait gave up). m, g_in and epoch as in the kernel.
__device__ __forceinline__ bool rename_tile(RnSmem &S, const RenameArgs &a, const uint32_t tile,
                                            const uint32_t m, const uint32_t g_in,
                                            const uint32_t epoch) {
  const int tid = threadIdx.x;
  const uint64_t *__restrict__ K = a.plan->kfinal;
  const uint32_t *__restrict__ V = a.plan->vfinal;
  const uint32_t base = tile * RN_TILE;
  const uint32_t count = min((uint32_t)RN_TILE, m - base);

  // Coalesced load of the tile plus one item of halo on each side.
  for (int k = 0; k < RN_ITEMS; ++k) {
    const uint32_t e = k * RN_BLOCK + tid;
    if (e < count) {
      S.keys[kidx(e)] = K[base + e];
      S.vals[vidx(e)] = V[base + e];
    }
  }
  if (tid == 0) {
    S.prev_key = base > 0 ? K[base - 1] : 0ull;
    S.prev_val = base > 0 ? V[base - 1] : 0u;
    const bool has_next = base + count < m;
    S.next_key = has_next ? K[base + count] : 0ull;
    S.next_val = has_next ? V[base + count] : 0u;
  }
  __syncthreads();

  // Items tid*16 .. tid*16+15 of the tile, with neighbours -1 and +16.
  const uint32_t l0 = tid * RN_ITEMS;
  uint64_t key[RN_ITEMS + 2];
  uint32_t val[RN_ITEMS + 2];
#pragma unroll
  for (int k = 0; k < RN_ITEMS + 2; ++k) {
    const int64_t l = (int64_t)l0 + k - 1;
    if (l < 0) {
      key[k] = S.prev_key;
      val[k] = S.prev_val;
    } else if (l < (int64_t)count) {
      key[k] = S.keys[kidx((uint32_t)l)];
      val[k] = S.vals[vidx((uint32_t)l)];
    } else {
      key[k] = S.next_key;
      val[k] = S.next_val;
    }
  }
  // Round 0: does the suffix at gapped position v (key k) have fewer than
  // c0 characters left in its text?
  auto tail = [&](uint64_t k, uint32_t v) -> bool {
    if (a.S <= 1) return a.N - v < a.c0;  // one text: gapped = plain positions
    const uint32_t s = (uint32_t)(k >> a.cb);
    const uint32_t off = __ldg(a.seg_off + s);
    const uint32_t len = __ldg(a.seg_off + s + 1) - off;
    return len - (v - (off + s)) < a.c0;
  };
  // f[k] = boundary flag of item l0 + k (k = 0..16).
  bool f[RN_ITEMS + 1];
  bool is_tail[RN_ITEMS + 2];
  if (a.round0) {
#pragma unroll
    for (int k = 0; k < RN_ITEMS + 2; ++k) is_tail[k] = tail(key[k], val[k]);
  }
  // a-tuple rounds: items with equal keys are still apart if their later
  // partners differ (sorted alongside, in the other key buffer).
  const uint64_t *SEC = a.sec_buf[0] ? a.sec_buf[a.plan->final_idx ^ 1u] : nullptr;
#pragma unroll
  for (int k = 0; k <= RN_ITEMS; ++k) {
    const uint64_t j = (uint64_t)base + l0 + k;
    bool b = (j == 0) || (j >= m) || key[k + 1] != key[k];
    if (a.round0 && j > 0 && j < m) b = b || is_tail[k + 1] || is_tail[k];
    if (SEC && !b) b = SEC[j] != SEC[j - 1];
    f[k] = b;
  }
  uint32_t th_surv = 0, th_hs = 0, th_uniq = 0;
#pragma unroll
  for (int k = 0; k < RN_ITEMS; ++k) {
    if (l0 + k < count) {
      const bool uniq = f[k] && f[k + 1];
      if (!uniq) {
        ++th_surv;
        if (f[k]) ++th_hs;
      } else {
        ++th_uniq;
      }
    }
  }
  // ISA entries of new unique suffixes are queued (in any order) and applied
  // only when a later round, the ISA output or the trace reads them.
  const uint32_t my_upd = th_uniq ? atomicAdd(&S.upd_local, th_uniq) : 0u;
  uint32_t tot_surv, tot_hs;
  const uint32_t ex_surv = block_exclusive<RN_BLOCK>(th_surv, OpAdd(), 0u, S.tmp, tot_surv);
  const uint32_t ex_hs = block_exclusive<RN_BLOCK>(th_hs, OpAdd(), 0u, S.tmp, tot_hs);

  // The tile's survivors and surviving groups, published for the device-wide
  // sums (decoupled look-back); the look-back itself runs after the staging
  // below, which needs only tile-local offsets.
  uint64_t *st_tile = a.status + (uint64_t)tile * 2;
  if (tid < 2) status_store(st_tile + tid, status_word(epoch, tile == 0 ? ST_INC : ST_AGG,
                                                        tid == 0 ? tot_surv : tot_hs));
  if (tid == 0) S.upd_base = S.upd_local ? atomicAdd(&a.ctrl->rc.upd, S.upd_local) : 0u;
  // Outputs are staged in shared memory and written with consecutive
  // addresses afterwards: queued updates in the keys area, survivors' list
  // entries (with tile-local group ordinals) in `surv`, and (round 0, where a
  // unique item's name is its own position in the sorted order) SA entries
  // by tile index in the vals area. Every item's new group starts at a head
  // (f = 1) whose head rank is that head's own sorted index, so no head rank
  // from an earlier tile is needed.
  uint64_t *st_upd = S.keys;
  uint32_t *st_sa = S.vals;
  if (a.round0)
    for (uint32_t e = tid; e < count; e += RN_BLOCK) st_sa[e] = NO_NAME;
  __syncthreads();
  {
    uint32_t run_upd = my_upd, run_surv = ex_surv, run_hs = ex_hs;
#pragma unroll
    for (int k = 0; k < RN_ITEMS; ++k) {
      if (l0 + k < count) {
        const uint32_t j = base + l0 + k;
        const uint64_t kk = key[k + 1];
        const uint32_t ip = val[k + 1];
        if (ip >= a.isa_len) {  // never taken unless a logic error
          raise_error(a.ctrl, ERR_INTERNAL, 3);
          continue;
        }
        if (f[k] && f[k + 1]) {
          // Unique: its name is its rank, final (Algorithm 5 discards it). SA
          // holds the index local to the suffix's own text.
          const uint32_t g = a.round0 ? 0u : (uint32_t)(kk >> a.W);
          if (!a.round0 && g >= g_in) {  // never taken unless a logic error
            raise_error(a.ctrl, ERR_INTERNAL, 4);
            continue;
          }
          const uint32_t head = a.round0 ? j : __ldg(a.base_in + g) + j;
          if (head >= a.N) {  // never taken unless a logic error
            raise_error(a.ctrl, ERR_INTERNAL, 3);
            continue;
          }
          st_upd[run_upd++] = ((uint64_t)head << 32) | ip;
          uint32_t local = ip;
          if (a.S > 1) {
            if (a.round0) {
              const uint32_t s = (uint32_t)(kk >> a.cb);
              local = ip - (__ldg(a.seg_off + s) + s);
            } else {
              local = local_index(ip, a.seg_off, a.S);
            }
          }
          if (a.round0)
            st_sa[l0 + k] = local;  // head == j here
          else
            a.sa[head] = local;
        } else {
          // Survivors get their names, and their ISA entries, once the group
          // sizes are known (k_classify, k_apply_names).
          if (f[k]) ++run_hs;
          S.surv[run_surv++] = ((uint64_t)(run_hs - 1) << 32) | ip;
        }
      }
    }
  }

  // Device-wide offsets of the tile's survivors and groups.
  if (tid < 2) {
    uint32_t carry = 0;
    bool ok = true;
    if (tile > 0) {
      ok = look_back_w<RN_LB_WINDOW>(a.status, 2, tid, tile, epoch, OpAdd(), carry, a.ctrl,
                                     a.spin_limit);
      if (ok)
        status_store(st_tile + tid,
                     status_word(epoch, ST_INC, carry + (tid == 0 ? tot_surv : tot_hs)));
    }
    if (!ok) S.bail = 1;
    S.carry[tid] = carry;
  }
  __syncthreads();
  if (S.bail) return false;
  const uint32_t m_off = __ldg(a.off_in), g_off = __ldg(a.off_in + 1);
  const uint32_t surv0 = m_off + S.carry[0], grp0 = g_off + S.carry[1];
  if (tid == 0 && base + count == m) {
    a.cnt_out[0] = S.carry[0] + tot_surv;
    a.cnt_out[1] = S.carry[1] + tot_hs;
  }
  // Surviving groups: start in the next list, head rank, parent's name.
  {
    uint32_t run_surv = ex_surv, run_hs = ex_hs;
#pragma unroll
    for (int k = 0; k < RN_ITEMS; ++k) {
      if (l0 + k < count && !(f[k] && f[k + 1])) {
        if (f[k]) {
          const uint32_t j = base + l0 + k;
          const uint32_t g = a.round0 ? 0u : (uint32_t)(key[k + 1] >> a.W);
          if (!a.round0 && g >= g_in) {  // never taken unless a logic error
            raise_error(a.ctrl, ERR_INTERNAL, 4);
            continue;
          }
          const uint32_t head = a.round0 ? j : __ldg(a.base_in + g) + j;
          if (head >= a.N) {  // never taken unless a logic error
            raise_error(a.ctrl, ERR_INTERNAL, 3);
            continue;
          }
          const uint32_t o = grp0 + run_hs;
          a.gstart_out[o] = surv0 + run_surv;
          a.ghead_out[o] = head;
          a.gold_out[o] = a.round0 ? NO_NAME : __ldg(a.old_in + g);
          ++run_hs;
        }
        ++run_surv;
      }
    }
  }
  for (uint32_t e = tid; e < S.upd_local; e += RN_BLOCK) a.upd[S.upd_base + e] = st_upd[e];
  const uint64_t gshift = (uint64_t)grp0 << 32;
  for (uint32_t e = tid; e < tot_surv; e += RN_BLOCK) a.act_out[surv0 + e] = S.surv[e] + gshift;
  if (a.round0) {
    for (uint32_t e = tid; e < count; e += RN_BLOCK) {
      const uint32_t v = st_sa[e];
      if (v != NO_NAME) a.sa[base + e] = v;
    }
  }
  return true;
}

// 8 items: 64 registers, 4 blocks of 256 threads per SM (42 KB of shared
// memory each); 4 items: 6 blocks. Tiles are taken from the launch's
// counter until it passes the last one, so any grid works (a grid smaller
// than the tile count makes the blocks persistent); in device-driven
// rounds the item and group counts and the epoch base come from the round
// state.
template <bool PERSIST>
__global__ void __launch_bounds__(RN_BLOCK, RN_ITEMS <= 4 ? 6 : 4) k_rename(RenameArgs a) {
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
      S.upd_local = 0u;
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
