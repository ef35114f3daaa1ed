// Rounds >= 1 of prefix doubling with discarding (Section 2.1, Algorithm 5)
// when most active groups are small.
//
// After round 0 every active suffix belongs to a group of equal names, and
// a group only ever splits into subgroups: the refinement of a round never
// crosses group boundaries. So the sort of a round is a segmented sort, and
// a group that fits one tile can be refined entirely inside one block:
//
//   k_refine (one tile = whole groups whose starts fall in a 2048-item
//   window, at most 4096 items): load the tile's (g, i') from the active
//   list, gather the partner names r2 = ISA[i' + h] + 1 (Algorithm 4), sort
//   by (local group, r2) with a radix sort in shared memory, then rename
//   (CmpName + max PrefixSum inside the tile; NameDiscarding's
//   r + (subgroup start - group start)), write SA for suffixes that became
//   unique, compact the survivors into the next active list and queue every
//   changed name as an (i', new) update. Tiles share nothing but two atomic
//   counters: the next list only needs each group contiguous, not in any
//   particular group order (names are absolute ranks).
//
//   Partner names of a round must all be read before any name of that round
//   changes (a mix of old and new names within one group would order
//   suffixes wrongly), so the refine never writes the ISA itself:
//   k_scatter_updates applies the queued updates after every gather of the
//   round has finished.
//
// Groups larger than REFINE_SMALL_MAX take the global path: k_gather_large
// builds (large-group ordinal, r2) keys, the one-sweep radix sort orders
// them and k_rename renames them (after the refine, so its direct ISA
// writes come after every gather).
//
// k_classify runs at the end of each round over the new group table: it
// lists the large groups (one 64-bit atomic gives each its slot and its
// item offset at once) and maps every refine tile to its first group.
//
// Bound: HBM. Refine per item: 8 bytes read, one 4-byte random gather,
// 8 bytes per survivor, 4 bytes random SA write per unique item, 8 bytes
// queued per changed name; the update scatter reads 8 and writes 4 random
// bytes per changed name.
#include "launch.h"

namespace gbsa {

// ---- classify -------------------------------------------------------------

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t n, uint32_t v) {
  uint32_t lo = 0, hi = n;  // first index with a[i] >= v, or n
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_classify(ClassifyArgs a) {
  if (a.rs && !a.rs->live) return;
  const uint32_t m = a.ctrl->rc.m_s + a.ctrl->rc.m_l;
  const uint32_t gs = a.ctrl->rc.g_s;
  const uint32_t G = gs + a.ctrl->rc.g_l;
  if (G > a.max_groups) {
    raise_error(a.ctrl, ERR_INTERNAL, 6);
    return;
  }
  const uint32_t tiles = (m + a.nominal - 1) / a.nominal;
  if (tiles > a.max_tiles) {
    raise_error(a.ctrl, ERR_INTERNAL, 7);
    return;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t total = (uint64_t)(G > tiles + 1 ? G : tiles + 1);
  // CL_UNROLL groups per thread and iteration, their starts loaded before
  // any is used (independent loads in flight).
  constexpr int CL_UNROLL = 4;
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < total;
       x0 += CL_UNROLL * stride) {
    uint32_t sv[CL_UNROLL], ev[CL_UNROLL];
#pragma unroll
    for (int u = 0; u < CL_UNROLL; ++u) {
      const uint64_t x = x0 + u * stride;
      sv[u] = x < G ? a.gstart[x] : 0u;
      ev[u] = x + 1 < G ? a.gstart[x + 1] : m;
    }
#pragma unroll
    for (int u = 0; u < CL_UNROLL; ++u) {
      const uint64_t x = x0 + u * stride;
      if (x >= total) break;
      if (x < G) {
        const uint32_t size = ev[u] - sv[u];
        uint32_t name = 0;
        if (x >= gs) {
          // A group written by the rename: its name is chosen now that its
          // size (its SA interval [head, head + size)) is known.
          const uint32_t head = a.ghead[x], old = a.gold[x];
          if (a.naming == NAMES_RETAIN)
            name = (old != NO_NAME && old - head < size) ? old : head + size / 2;
          else
            name = head;
          a.gname[x] = name;
        }
        if (size > a.nominal) {
          if (x < gs) name = a.gname[x];
          const unsigned long long old =
              atomicAdd(&a.ctrl->rc.large, (1ull << 32) | (unsigned long long)size);
          const uint32_t k = (uint32_t)(old >> 32), off = (uint32_t)old;
          a.lg[k] = (uint32_t)x;
          a.loff[k] = off;
          a.lbase[k] = a.ghead[x] - off;
          a.lold[k] = name;
        }
      }
      if (x <= tiles) a.tfirst[x] = lower_bound_u32(a.gstart, G, (uint32_t)x * a.nominal);
      if (x == 0) a.gstart[G] = m;
    }
  }
}

cudaError_t launch_classify(const ClassifyArgs &a, int num_sms, cudaStream_t stream) {
  // One full wave (8 blocks of 256 threads per SM).
  k_classify<<<num_sms * 8, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

// ---- large groups: keys for the global radix sort ---------------------------

__device__ __forceinline__ void gather_large_item(const GatherLargeArgs &a, const uint32_t j,
                                                  const uint32_t GL, const uint32_t h);

__global__ void __launch_bounds__(256) k_gather_large(GatherLargeArgs a) {
  uint32_t mL = a.mL, GL = a.GL, h = a.h;
  if (a.rs) {  // device-driven rounds
    if (!a.rs->live) return;
    mL = a.rs->mL;
    GL = a.rs->GL;
    h = a.rs->h;
  }
  for (uint64_t j64 = (uint64_t)blockIdx.x * 256 + threadIdx.x; j64 < mL;
       j64 += (uint64_t)gridDim.x * 256)
    gather_large_item(a, (uint32_t)j64, GL, h);
}

__device__ __forceinline__ void gather_large_item(const GatherLargeArgs &a, const uint32_t j,
                                                  const uint32_t GL, const uint32_t h) {
  // k = the large group holding item j: the last k with loff[k] <= j
  uint32_t lo = 0, hi = GL - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(a.loff + mid) <= j)
      lo = mid;
    else
      hi = mid - 1;
  }
  const uint32_t g = __ldg(a.lg + lo);
  const uint64_t e = a.act[__ldg(a.gstart + g) + (j - __ldg(a.loff + lo))];
  const uint32_t ip = (uint32_t)e;
  const uint64_t at = min((uint64_t)ip + h, a.isa_len - 1);
  const uint32_t r2 = __ldg(a.isa + at) + 1u;
  const uint64_t key1 = ((uint64_t)lo << a.W) | r2;
  if (a.mult == 2) {
    a.keys[j] = key1;
    a.vals[j] = ip;
    return;
  }
  // a-tuples: the later partners are sorted first (keys), item j rides
  // along; (group, r2) and the later partners are kept by item.
  const uint32_t r3 = r2 ? __ldg(a.isa + min((uint64_t)ip + (uint64_t)2 * h, a.isa_len - 1)) + 1u : 0u;
  uint32_t r4 = 0;
  if (a.mult == 4 && r3) r4 = __ldg(a.isa + min((uint64_t)ip + (uint64_t)3 * h, a.isa_len - 1)) + 1u;
  const uint64_t sec = a.mult == 4 ? (((uint64_t)r3 << a.W) | r4) : (uint64_t)r3;
  a.keys[j] = sec;
  a.vals[j] = j;
  a.key1_stash[j] = key1;
  a.sec_stash[j] = sec;
}

cudaError_t launch_gather_large(const GatherLargeArgs &a, cudaStream_t stream) {
  if (a.mL == 0) return cudaSuccess;
  uint64_t grid = ((uint64_t)a.mL + 255) / 256;
  if (a.grid_cap && grid > a.grid_cap) grid = a.grid_cap;
  k_gather_large<<<(unsigned)grid, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

// Between the two sorts of an a-tuple round: the items, in the order of
// their later partners, get their (group, r2) keys back as the input of the
// second (stable) sort.
__global__ void __launch_bounds__(256) k_wide_rekey(WideArgs a) {
  const uint64_t x64 = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (x64 >= a.mL) return;
  const uint32_t x = (uint32_t)x64;
  const uint32_t j = a.plan->vfinal[x];
  if (j >= a.mL) {  // never taken unless a logic error
    raise_error(a.ctrl, ERR_INTERNAL, 11);
    return;
  }
  a.ka[x] = a.key1_stash[j];
  a.va[x] = j;
}

// After the second sort: each position gets its item's gapped position (for
// k_rename) and its later partners, written to the sort buffer that does
// not hold the result.
__global__ void __launch_bounds__(256) k_wide_finish(WideArgs a) {
  const uint64_t y64 = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (y64 >= a.mL) return;
  const uint32_t y = (uint32_t)y64;
  const SortPlan *p = a.plan;
  const uint32_t j = p->vfinal[y];
  const uint32_t lo = (uint32_t)(p->kfinal[y] >> a.W);
  if (j >= a.mL || lo >= a.GL || j < __ldg(a.loff + lo)) {  // never taken unless a logic error
    raise_error(a.ctrl, ERR_INTERNAL, 12);
    return;
  }
  const uint32_t g = __ldg(a.lg + lo);
  const uint64_t at = (uint64_t)__ldg(a.gstart + g) + (j - __ldg(a.loff + lo));
  if (at >= a.m) {  // never taken unless a logic error
    raise_error(a.ctrl, ERR_INTERNAL, 13);
    return;
  }
  const uint32_t ip = (uint32_t)a.act[at];
  const_cast<uint32_t *>(p->vfinal)[y] = ip;
  (p->final_idx ? a.ka : a.kb)[y] = a.sec_stash[j];
}

cudaError_t launch_wide_rekey(const WideArgs &a, cudaStream_t stream) {
  if (a.mL == 0) return cudaSuccess;
  k_wide_rekey<<<(unsigned)(((uint64_t)a.mL + 255) / 256), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wide_finish(const WideArgs &a, cudaStream_t stream) {
  if (a.mL == 0) return cudaSuccess;
  k_wide_finish<<<(unsigned)(((uint64_t)a.mL + 255) / 256), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

// ---- small groups: one tile per block ---------------------------------------

// Tiles whose small groups have at most RF_RANK_GMAX members and whose
// items would make at most RF_RANK_AVG comparisons each on average (sum of
// squared group sizes <= RF_RANK_AVG x items) are ordered by counting
// instead of the in-tile radix sort.
#ifndef GBSA_RF_RANK_GMAX
#define GBSA_RF_RANK_GMAX 64
#endif
#ifndef GBSA_RF_RANK_AVG
#define GBSA_RF_RANK_AVG 16
#endif
constexpr uint32_t RF_RANK_GMAX = GBSA_RF_RANK_GMAX;
constexpr uint32_t RF_RANK_AVG = GBSA_RF_RANK_AVG;

template <int BLOCK, int CAP>
struct RfCfg {
  static constexpr int WARPS = BLOCK / 32;
  static constexpr int ITEMS = CAP / BLOCK;       // slots per thread
  static constexpr int NOMINAL = CAP / 2;         // tile window and largest small group
  static constexpr int MAXG = NOMINAL / 2 + 1;    // groups have >= 2 members
  static constexpr int GPT = (MAXG + BLOCK - 1) / BLOCK;  // groups per thread
  static constexpr int DPT = RADIX / BLOCK;       // digits per thread in the digit scan
  static_assert(ITEMS >= 1 && ITEMS <= 16, "slots per thread");
  static_assert(DPT >= 1 && RADIX % BLOCK == 0, "digits per thread");
};

// Per-slot data of a tile when a round ranks a-tuples (a = 3 or 4): the
// first sort orders the slots by their later partner names, the second by
// (local group, first partner name) and keeps that order among ties.
template <int CAP, bool WIDE>
struct RfWide {
  uint64_t key1[CAP];  // (local group << W) | r2
  uint64_t sec[CAP];   // r3 (a = 3) or (r3 << W) | r4 (a = 4)
  uint32_t ip[CAP];    // gapped position
};
template <int CAP>
struct RfWide<CAP, false> {};

template <int BLOCK, int CAP, bool WIDE>
struct RfSmem {
  using C = RfCfg<BLOCK, CAP>;
  uint64_t keys[CAP + CAP / 16];  // padded (e + e/16) after the last pass
  uint32_t vals[CAP + CAP / 32];  // padded (e + e/32) after the last pass
  RfWide<CAP, WIDE> w;
  union {
    uint32_t gsrc[C::MAXG];             // first position of each local group
    // Not read: keeps the arrays below at the offsets of the layout that
    // measured fastest (the same shape with 3 KB less shared memory ran the
    // refine about 5% slower on GB300).
    uint32_t spacer[C::WARPS][RADIX];
  };
  uint16_t whist[2][C::WARPS][RADIX];   // per pass (double-buffered): counts, then prefixes
  uint32_t dstart[RADIX];
  uint32_t gname[C::MAXG];
  uint32_t ghead[C::MAXG];              // head rank (SA interval start) of the local group
  uint32_t goff[C::MAXG + 1];           // start of the local group in the tile
  uint32_t tmp[2][4 * C::WARPS];        // scan scratch (double-buffered)
  uint32_t flag, all_small, upd_local, upd_base, surv_base, grp_base;
  uint32_t gmax, gsq;  // largest small group, sum of squared small-group sizes
  unsigned long long orv, orv2;
};

// One-barrier exclusive sum over the block: warp scans, warp totals in
// `tmp`, then every thread adds the totals of the warps before it. `tmp`
// must not be rewritten before the next barrier.
template <int BLOCK>
__device__ __forceinline__ uint32_t rf_block_excl_sum(uint32_t v, uint32_t *tmp, uint32_t &total) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_inclusive(v, OpAdd());
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint32_t t = tmp[w];
    before += w < warp ? t : 0u;
    all += t;
  }
  total = all;
  return before + incl - v;
}

// One-barrier fused scans of the rename phase: exclusive max (mx), two
// exclusive sums (s1, s2) and the exclusive suffix minimum (mn, over the
// threads after this one).
template <int BLOCK>
__device__ __forceinline__ void rf_block_scan4(uint32_t mx, uint32_t s1, uint32_t s2, uint32_t mn,
                                               uint32_t *tmp, uint32_t &ex_mx, uint32_t &ex_s1,
                                               uint32_t &ex_s2, uint32_t &sf_mn, uint32_t &tot_s1,
                                               uint32_t &tot_s2) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t imx = mx, is1 = s1, is2 = s2, imn = mn;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t omx = __shfl_up_sync(0xffffffffu, imx, d);
    const uint32_t os1 = __shfl_up_sync(0xffffffffu, is1, d);
    const uint32_t os2 = __shfl_up_sync(0xffffffffu, is2, d);
    const uint32_t omn = __shfl_down_sync(0xffffffffu, imn, d);
    if (lane >= d) {
      imx = omx > imx ? omx : imx;
      is1 += os1;
      is2 += os2;
    }
    if (lane + d < 32) imn = omn < imn ? omn : imn;
  }
  if (lane == 31) {
    tmp[warp] = imx;
    tmp[WARPS + warp] = is1;
    tmp[2 * WARPS + warp] = is2;
  }
  if (lane == 0) tmp[3 * WARPS + warp] = imn;
  __syncthreads();
  uint32_t pmx = 0, ps1 = 0, ps2 = 0, pmn = 0xFFFFFFFFu, t1 = 0, t2 = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint32_t a1 = tmp[WARPS + w], a2 = tmp[2 * WARPS + w];
    t1 += a1;
    t2 += a2;
    if (w < warp) {
      const uint32_t a0 = tmp[w];
      pmx = a0 > pmx ? a0 : pmx;
      ps1 += a1;
      ps2 += a2;
    }
    if (w > warp) {
      const uint32_t a3 = tmp[3 * WARPS + w];
      pmn = a3 < pmn ? a3 : pmn;
    }
  }
  uint32_t emx = __shfl_up_sync(0xffffffffu, imx, 1);
  if (lane == 0) emx = 0;
  uint32_t nmn = __shfl_down_sync(0xffffffffu, imn, 1);
  if (lane == 31) nmn = 0xFFFFFFFFu;
  ex_mx = emx > pmx ? emx : pmx;
  ex_s1 = ps1 + is1 - s1;
  ex_s2 = ps2 + is2 - s2;
  sf_mn = nmn < pmn ? nmn : pmn;
  tot_s1 = t1;
  tot_s2 = t2;
}

// Rank of digit d among this warp's earlier lanes with the same digit, plus
// the warp's running count of d (wh), which the lowest such lane advances.
// Peers are found with match.any: in a refine tile the digits of a warp
// take few distinct values (the members of a group mostly share their
// partner's name), where it measured faster than the radix pass's
// shared-memory peer masks (refine 82.5 -> 74.5 ms at n = 2^28); on the
// radix pass's high-entropy digits it measured slower, so the pass keeps
// the masks.
__device__ __forceinline__ uint32_t rf_rank_digit(uint32_t d, uint16_t *wh, uint32_t lt) {
  const uint32_t peers = __match_any_sync(0xffffffffu, d);
  const uint32_t before = wh[d];
  __syncwarp();
  if ((peers & lt) == 0) wh[d] = (uint16_t)(before + __popc(peers));
  __syncwarp();
  return before + __popc(peers & lt);
}

// Stable LSD radix sort of S.keys/S.vals[0, cnt) in shared memory over the
// 8-bit digits below `nbits` that vary inside the tile. Warp w ranks the
// contiguous chunk [w*C, (w+1)*C) with C = 32 * ceil(cnt / BLOCK), so every
// warp does the same useful work and (warp, slot, lane) is the input order.
// The last pass writes the padded layout read by the rename phase (at
// least one pass always runs; with pad_out false it writes the plain
// layout). Four barriers per pass.
template <int BLOCK, int CAP, bool WIDE>
__device__ void rf_tile_sort(RfSmem<BLOCK, CAP, WIDE> &S, uint32_t cnt,
                             unsigned long long varying, uint32_t nbits, bool pad_out) {
  using C = RfCfg<BLOCK, CAP>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  const uint32_t K = (cnt + BLOCK - 1) / BLOCK;  // slots per lane, <= ITEMS
  const uint32_t chunk = K * 32;
  const uint32_t ndig = (nbits + RADIX_BITS - 1) / RADIX_BITS;
  for (int x = tid; x < C::WARPS * RADIX; x += BLOCK) (&S.whist[0][0][0])[x] = 0;
  __syncthreads();
  uint32_t last = 0;
  for (uint32_t p = 0; p < ndig; ++p)
    if ((varying >> (p * RADIX_BITS)) & 0xFFull) last = p;
  uint32_t buf = 0;
  for (uint32_t p = 0; p <= last; ++p) {
    const bool kept = ((varying >> (p * RADIX_BITS)) & 0xFFull) != 0ull;
    if (!kept && p != last) continue;
    const uint32_t shift = p * RADIX_BITS;
    const bool pad = pad_out && p == last;
    uint64_t key[C::ITEMS];
    uint32_t val[C::ITEMS], pos[C::ITEMS];
    uint16_t *wh = S.whist[buf][warp];
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      if ((uint32_t)k < K) {
        const uint32_t li = warp * chunk + k * 32 + lane;
        const bool valid = li < cnt;
        key[k] = valid ? S.keys[li] : ~0ull;
        val[k] = valid ? S.vals[li] : 0u;
        const uint32_t d = valid ? (uint32_t)(key[k] >> shift) & 0xFFu : 0xFFu;
        pos[k] = rf_rank_digit(d, wh, lt);
      }
    }
    __syncthreads();
    // Thread t owns digits [t*DPT, (t+1)*DPT): per-warp prefixes, then the
    // block scan of the digit totals gives each digit's start in the tile.
    uint32_t dsum = 0, dtot[C::DPT];
#pragma unroll
    for (int i = 0; i < C::DPT; ++i) {
      const uint32_t d = tid * C::DPT + i;
      uint32_t total = 0;
#pragma unroll
      for (int w = 0; w < C::WARPS; ++w) {
        const uint32_t c = S.whist[buf][w][d];
        S.whist[buf][w][d] = (uint16_t)total;
        total += c;
      }
      dtot[i] = total;
      dsum += total;
    }
    uint32_t all;
    uint32_t run = rf_block_excl_sum<BLOCK>(dsum, S.tmp[buf], all);
#pragma unroll
    for (int i = 0; i < C::DPT; ++i) {
      S.dstart[tid * C::DPT + i] = run;
      run += dtot[i];
    }
    __syncthreads();
    uint16_t *nxt = &S.whist[buf ^ 1][0][0];
    for (int x = tid; x < C::WARPS * RADIX; x += BLOCK) nxt[x] = 0;
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t li = warp * chunk + k * 32 + lane;
      if ((uint32_t)k < K && li < cnt) {
        const uint32_t d = (uint32_t)(key[k] >> shift) & 0xFFu;
        const uint32_t q = S.dstart[d] + S.whist[buf][warp][d] + pos[k];
        S.keys[pad ? q + (q >> 4) : q] = key[k];
        S.vals[pad ? q + (q >> 5) : q] = val[k];
      }
    }
    __syncthreads();
    buf ^= 1;
  }
}

// Tiles whose groups all have at most RF_GROUP_MAX members (the pairs left
// by long copied segments, for example) are refined group by group: each
// thread takes its own groups of the tile's table whole -- their active
// entries, partner names, a stable sort of at most four items in
// registers, the subgroups and their names -- so no shared-memory sort or
// item-wise rename runs. One block-wide scan of (survivors, surviving
// groups, changed names) per thread places the outputs. The names are the
// item-wise path's: a subgroup of len items starting at a in its group's
// sorted order has the SA interval [head + a, head + a + len).
constexpr uint32_t RF_GROUP_MAX = 4;

// Exclusive sum over the block of 64-bit values (one barrier), the total in
// `total`; `tmp` holds 2 * WARPS words and is not rewritten before the
// next barrier.
template <int BLOCK>
__device__ __forceinline__ uint64_t rf_block_excl_sum64(uint64_t v, uint32_t *tmp,
                                                        uint64_t &total) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) {
    tmp[2 * warp] = (uint32_t)incl;
    tmp[2 * warp + 1] = (uint32_t)(incl >> 32);
  }
  __syncthreads();
  uint64_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint64_t t = ((uint64_t)tmp[2 * w + 1] << 32) | tmp[2 * w];
    before += w < warp ? t : 0ull;
    all += t;
  }
  total = all;
  return before + incl - v;
}

__device__ __forceinline__ void cswap(uint64_t &x, uint64_t &y) {
  const uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
  x = lo;
  y = hi;
}

template <int BLOCK, int CAP>
__device__ __forceinline__ void refine_tiny_groups(RfSmem<BLOCK, CAP, false> &S,
                                                   const RefineArgs &a,
                                                   const uint32_t (&sz)[RfCfg<BLOCK, CAP>::GPT],
                                                   const uint32_t h) {
  using C = RfCfg<BLOCK, CAP>;
  constexpr int GPT = C::GPT;
  constexpr int M = (int)RF_GROUP_MAX;
  const int tid = threadIdx.x;
  // Entries, then partner names of all of this thread's groups, every load
  // issued before its use, kept in registers as (r2 << 32) | i'.
  static_assert(M == 4, "the sorting network below orders four items");
  uint64_t it[GPT][M];
#pragma unroll
  for (int r = 0; r < GPT; ++r) {
    const uint32_t lg = tid * GPT + r;
    const uint32_t base = sz[r] ? S.gsrc[lg] : 0u;
#pragma unroll
    for (int k = 0; k < M; ++k) it[r][k] = (uint32_t)k < sz[r] ? a.act[base + k] : ~0ull;
  }
#pragma unroll
  for (int r = 0; r < GPT; ++r)
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((uint32_t)k < sz[r]) {
        const uint32_t ip = (uint32_t)it[r][k];
        const uint32_t r2 = __ldg(a.isa + min((uint64_t)ip + h, a.isa_len - 1)) + 1u;
        it[r][k] = ((uint64_t)r2 << 32) | ip;
      }
  uint32_t n_surv = 0, n_grp = 0, n_chg = 0;
#pragma unroll
  for (int r = 0; r < GPT; ++r) {
    const uint32_t z = sz[r];
    if (!z) continue;
    // Sort by (partner name, position): padding (all ones) stays last, and
    // the order among equal names, which names do not depend on, is fixed.
    cswap(it[r][0], it[r][1]);
    cswap(it[r][2], it[r][3]);
    cswap(it[r][0], it[r][2]);
    cswap(it[r][1], it[r][3]);
    cswap(it[r][1], it[r][2]);
    const uint32_t lg = tid * GPT + r;
    const uint32_t head = S.ghead[lg], old = S.gname[lg];
    uint32_t a0 = 0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if ((uint32_t)k < z) {
        const bool end = (uint32_t)k + 1 == z || (it[r][k + 1 < M ? k + 1 : k] >> 32) != (it[r][k] >> 32);
        if (end) {  // subgroup [a0, k]
          const uint32_t len = k + 1 - a0, lo = head + a0;
          const uint32_t name =
              len == 1 || a.naming != NAMES_RETAIN ? lo : (old - lo < len ? old : lo + len / 2);
          if (len > 1) {
            n_surv += len;
            ++n_grp;
          }
          if (name != old) n_chg += len;
          a0 = k + 1;
        }
      }
    }
  }
  // Place the outputs: survivors (21 bits), surviving groups (21 bits) and
  // changed names (22 bits) scanned together.
  const uint64_t mine = (uint64_t)n_surv | ((uint64_t)n_grp << 21) | ((uint64_t)n_chg << 42);
  uint64_t tot;
  // S.tmp[1]: the caller's last scan used S.tmp[0], which some warps may
  // still be reading.
  const uint64_t ex = rf_block_excl_sum64<BLOCK>(mine, S.tmp[1], tot);
  if (tid == 0) {
    const uint32_t tot_surv = (uint32_t)(tot & 0x1FFFFF), tot_grp = (uint32_t)((tot >> 21) & 0x1FFFFF);
    const uint32_t tot_chg = (uint32_t)(tot >> 42);
    const unsigned long long inc = ((unsigned long long)tot_grp << 32) | tot_surv;
    const unsigned long long o =
        inc ? atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctrl->rc.m_s), inc) : 0ull;
    S.surv_base = (uint32_t)o;
    S.grp_base = (uint32_t)(o >> 32);
    S.upd_base = tot_chg ? atomicAdd(&a.ctrl->rc.upd, tot_chg) : 0u;
  }
  __syncthreads();
  uint32_t run_surv = S.surv_base + (uint32_t)(ex & 0x1FFFFF);
  uint32_t run_grp = S.grp_base + (uint32_t)((ex >> 21) & 0x1FFFFF);
  uint32_t run_chg = S.upd_base + (uint32_t)(ex >> 42);
#pragma unroll
  for (int r = 0; r < GPT; ++r) {
    const uint32_t z = sz[r];
    if (!z) continue;
    const uint32_t lg = tid * GPT + r;
    const uint32_t head = S.ghead[lg], old = S.gname[lg];
    // Bit k of E: item k ends its subgroup (the last item, or the next item
    // has another partner name). Item x then belongs to the subgroup
    // [a0, e]: e the first end at or after x, a0 one past the last end
    // before it.
    uint32_t E = 0;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((uint32_t)k < z &&
          ((uint32_t)k + 1 == z || (it[r][k + 1 < M ? k + 1 : k] >> 32) != (it[r][k] >> 32)))
        E |= 1u << k;
#pragma unroll
    for (int x = 0; x < M; ++x) {
      if ((uint32_t)x >= z) continue;
      const uint32_t e = (uint32_t)x + __ffs(E >> x) - 1;
      const uint32_t below = E & ((1u << x) - 1u);
      const uint32_t a0 = below ? 32u - __clz(below) : 0u;
      const uint32_t len = e + 1 - a0, lo = head + a0;
      const uint32_t name =
          len == 1 || a.naming != NAMES_RETAIN ? lo : (old - lo < len ? old : lo + len / 2);
      const uint32_t ip = (uint32_t)it[r][x];
      if (name >= a.N || ip >= a.isa_len) {  // never taken unless a logic error
        raise_error(a.ctrl, ERR_INTERNAL, name >= a.N ? 15 : 16);
        return;
      }
      if (len > 1 && (uint32_t)x == a0) {  // a surviving subgroup starts here
        a.gstart_out[run_grp] = run_surv;
        a.gname_out[run_grp] = name;
        a.ghead_out[run_grp] = lo;
      }
      if (name != old) a.upd[run_chg++] = ((uint64_t)name << 32) | ip;
      if (len == 1) {
        a.sa[name] = local_index(ip, a.seg_off, a.S);
      } else {
        a.act_out[run_surv++] = ((uint64_t)run_grp << 32) | ip;
        if ((uint32_t)x == e) ++run_grp;
      }
    }
  }
}

// One refine tile (whole groups whose starts fall in the tile's window).
// Every thread of the block calls it; all returns are block-uniform.
template <int BLOCK, int CAP, bool WIDE>
__device__ __forceinline__ void refine_tile(RfSmem<BLOCK, CAP, WIDE> &S, const RefineArgs &a,
                                            const uint32_t tile, const uint32_t h) {
  using C = RfCfg<BLOCK, CAP>;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.orv = 0ull;
    S.orv2 = 0ull;
    S.upd_local = 0u;
    S.gmax = 0u;
    S.gsq = 0u;
    S.flag = has_error(a.ctrl) ? 1u : 0u;
  }
  __syncthreads();
  if (S.flag) return;
  const uint32_t g0 = __ldg(a.tfirst + tile), g1 = __ldg(a.tfirst + tile + 1);
  const uint32_t ng = g1 - g0;
  if (ng > (uint32_t)C::MAXG) {  // never taken unless a logic error
    if (tid == 0) raise_error(a.ctrl, ERR_INTERNAL, 8);
    return;
  }
  if (ng == 0) return;

  // Local group table: source position, name, head rank, size (0 for a
  // large group), then exclusive offsets inside the tile.
  uint32_t sz[C::GPT];
  uint32_t mysum = 0, mybig = 0, mymax = 0, mysq = 0;
#pragma unroll
  for (int r = 0; r < C::GPT; ++r) {
    const uint32_t lg = tid * C::GPT + r;
    sz[r] = 0;
    if (lg < ng) {
      const uint32_t g = g0 + lg;
      const uint32_t s = __ldg(a.gstart + g), e = __ldg(a.gstart + g + 1);
      S.gsrc[lg] = s;
      S.gname[lg] = __ldg(a.gname + g);
      S.ghead[lg] = __ldg(a.ghead + g);
      const uint32_t size = e - s;
      if (size <= (uint32_t)C::NOMINAL)
        sz[r] = size;
      else
        mybig = 1;
      mysum += sz[r];
      mysq += sz[r] * sz[r];
      mymax = sz[r] > mymax ? sz[r] : mymax;
    }
  }
  {
    const uint32_t wsq = __reduce_add_sync(0xffffffffu, mysq);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, mymax);
    if ((tid & 31) == 0 && wsq) {
      atomicAdd(&S.gsq, wsq);
      atomicMax(&S.gmax, wmax);
    }
  }
  uint32_t nitems;
  uint32_t run = rf_block_excl_sum<BLOCK>(mysum, S.tmp[0], nitems);
  if (nitems > (uint32_t)CAP) {  // never taken unless a logic error
    if (tid == 0) raise_error(a.ctrl, ERR_INTERNAL, 9);
    return;
  }
  if (nitems == 0) return;
  if constexpr (!WIDE && CAP <= 1024) {
    // Block-uniform (S.gmax is complete after the scan's barrier): every
    // group has at most 4 members. That path takes each group whole from
    // its source, so it needs neither the tile offsets below nor their
    // barriers.
    if (S.gmax <= RF_GROUP_MAX) {
      refine_tiny_groups<BLOCK, CAP>(S, a, sz, h);
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < C::GPT; ++r) {
    const uint32_t lg = tid * C::GPT + r;
    if (lg < ng) S.goff[lg] = run;
    run += sz[r];
  }
  const int any_big = __syncthreads_or(mybig);
  if (tid == 0) {
    S.goff[ng] = nitems;
    S.all_small = any_big ? 0u : 1u;
  }
  __syncthreads();
  const uint32_t cnt = nitems;
  const uint32_t K = (cnt + BLOCK - 1) / BLOCK;

  // Load (g, i') and gather the partner names; all loads of a thread are
  // issued before their uses.
  uint64_t ent[C::ITEMS];
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const uint32_t q = k * BLOCK + tid;
    ent[k] = 0ull;
    if ((uint32_t)k < K && q < cnt) {
      uint32_t src;
      if (S.all_small) {
        src = S.gsrc[0] + q;
      } else {
        uint32_t lo = 0, hi = ng - 1;  // last local group with goff <= q
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (S.goff[mid] <= q)
            lo = mid;
          else
            hi = mid - 1;
        }
        src = S.gsrc[lo] + (q - S.goff[lo]);
      }
      ent[k] = a.act[src];
    }
  }
  uint32_t r2v[C::ITEMS];
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const uint32_t q = k * BLOCK + tid;
    r2v[k] = 0;
    if ((uint32_t)k < K && q < cnt) {
      const uint64_t at = min((uint64_t)(uint32_t)ent[k] + h, a.isa_len - 1);
      r2v[k] = __ldg(a.isa + at) + 1u;
    }
  }
  // a = 3, 4 (Prefix Quadrupling): the names of i' + 2h and i' + 3h as well,
  // 0 once an earlier one is the end sentinel (ties on a non-zero name
  // imply the later offsets stay inside the text; the rest never decide).
  uint64_t secv[WIDE ? C::ITEMS : 1];
  if constexpr (WIDE) {
    uint32_t r3v[C::ITEMS], r4v[C::ITEMS];
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t q = k * BLOCK + tid;
      r3v[k] = r4v[k] = 0;
      if ((uint32_t)k < K && q < cnt) {
        const uint64_t ip = (uint32_t)ent[k];
        r3v[k] = __ldg(a.isa + min(ip + (uint64_t)2 * h, a.isa_len - 1)) + 1u;
        if (a.mult == 4) r4v[k] = __ldg(a.isa + min(ip + (uint64_t)3 * h, a.isa_len - 1)) + 1u;
      }
    }
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t r3 = r2v[k] ? r3v[k] : 0u;
      const uint32_t r4 = r3 ? r4v[k] : 0u;
      secv[k] = a.mult == 4 ? (((uint64_t)r3 << a.W) | r4) : (uint64_t)r3;
    }
  }
  unsigned long long orv = 0ull, orv2 = 0ull;
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const uint32_t q = k * BLOCK + tid;
    if ((uint32_t)k < K && q < cnt) {
      const uint32_t lgq = (uint32_t)(ent[k] >> 32) - g0;
      const uint64_t key = ((uint64_t)lgq << a.W) | r2v[k];
      if constexpr (WIDE) {
        S.w.key1[q] = key;
        S.w.sec[q] = secv[k];
        S.w.ip[q] = (uint32_t)ent[k];
        S.keys[q] = secv[k];
        S.vals[q] = q;
      } else {
        S.keys[q] = key;
        S.vals[q] = (uint32_t)ent[k];
      }
    }
  }
  __syncthreads();
  // Tiles of small groups only (the pairs left by long repeats, for
  // example): each item's place is its group's start plus the number of
  // members with a smaller partner name, or an equal one earlier in the
  // list, which is the stable sort's order, at about (sum of squared group
  // sizes) / items comparisons per item instead of the radix passes.
  if constexpr (!WIDE) {
    if (S.gmax <= RF_RANK_GMAX && S.gsq <= RF_RANK_AVG * cnt) {
      uint32_t dst[C::ITEMS];
#pragma unroll
      for (int k = 0; k < C::ITEMS; ++k) {
        const uint32_t q = k * BLOCK + tid;
        dst[k] = 0;
        if ((uint32_t)k < K && q < cnt) {
          const uint32_t lgq = (uint32_t)(ent[k] >> 32) - g0;
          const uint32_t lo = S.goff[lgq], hi = S.goff[lgq + 1];
          // Members share the group bits, so whole keys compare as names.
          const uint64_t kq = ((uint64_t)lgq << a.W) | r2v[k];
          uint32_t before = 0;
          for (uint32_t x = lo; x < hi; ++x) {
            const uint64_t o = S.keys[x];
            before += (o < kq || (o == kq && x < q)) ? 1u : 0u;
          }
          dst[k] = lo + before;
        }
      }
      __syncthreads();  // every read of the input order is done
#pragma unroll
      for (int k = 0; k < C::ITEMS; ++k) {
        const uint32_t q = k * BLOCK + tid;
        if ((uint32_t)k < K && q < cnt) {
          const uint32_t lgq = (uint32_t)(ent[k] >> 32) - g0;
          const uint32_t e = dst[k];
          S.keys[e + (e >> 4)] = ((uint64_t)lgq << a.W) | r2v[k];
          S.vals[e + (e >> 5)] = (uint32_t)ent[k];
        }
      }
      __syncthreads();
      goto renamed_order;
    }
  }
  {
  // Bits that vary inside the tile: OR of (key ^ first key). Every key
  // shares the first key's local group 0 bits only when ng == 1, so the
  // reference key is the tile's first key.
  if constexpr (WIDE) {
    const uint64_t key0 = S.w.key1[0], sec0 = S.w.sec[0];
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t q = k * BLOCK + tid;
      if ((uint32_t)k < K && q < cnt) {
        orv |= S.w.key1[q] ^ key0;
        orv2 |= S.w.sec[q] ^ sec0;
      }
    }
  } else {
    const uint64_t key0 = S.keys[0];
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t q = k * BLOCK + tid;
      if ((uint32_t)k < K && q < cnt) orv |= S.keys[q] ^ key0;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    orv |= __shfl_xor_sync(0xffffffffu, orv, d);
    if constexpr (WIDE) orv2 |= __shfl_xor_sync(0xffffffffu, orv2, d);
  }
  if ((tid & 31) == 0 && orv) atomicOr(&S.orv, orv);
  if (WIDE && (tid & 31) == 0 && orv2) atomicOr(&S.orv2, orv2);
  __syncthreads();
  const uint32_t gbits = ng > 1 ? 32u - __clz(ng - 1) : 0u;
  if constexpr (WIDE) {
    // LSD over the tuple: the later partners first, then (group, r2); both
    // sorts are stable, so ties on (group, r2) keep the first sort's order.
    rf_tile_sort<BLOCK, CAP, WIDE>(S, cnt, S.orv2, a.mult == 4 ? 2 * a.W : a.W, false);
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t q = k * BLOCK + tid;
      if ((uint32_t)k < K && q < cnt) S.keys[q] = S.w.key1[S.vals[q]];
    }
    __syncthreads();
  }
  rf_tile_sort<BLOCK, CAP, WIDE>(S, cnt, S.orv, a.W + gbits, true);
  }
renamed_order:

  // Rename in blocked layout: items tid*K .. tid*K+K-1 of the sorted tile.
  const uint32_t l0 = tid * K;
  bool f[C::ITEMS + 1];
  {
    uint64_t prev = 0ull, prev2 = 0ull;
    if (l0 > 0 && l0 - 1 < cnt) {
      const uint32_t e = l0 - 1;
      prev = S.keys[e + (e >> 4)];
      if constexpr (WIDE) prev2 = S.w.sec[S.vals[e + (e >> 5)]];
    }
#pragma unroll
    for (int k = 0; k <= C::ITEMS; ++k) {
      const uint32_t j = l0 + k;
      f[k] = true;
      if ((uint32_t)k <= K && j < cnt) {
        const uint64_t kcur = S.keys[j + (j >> 4)];
        f[k] = (j == 0) || kcur != prev;
        prev = kcur;
        if constexpr (WIDE) {
          const uint64_t scur = S.w.sec[S.vals[j + (j >> 5)]];
          f[k] = f[k] || scur != prev2;
          prev2 = scur;
        }
      }
    }
  }
  // Subgroup bounds: start = last head at or before j (max-scan), end =
  // first head after j (suffix min-scan); both inside the tile, since tiles
  // hold whole groups.
  uint32_t th_head = 0, th_first = 0xFFFFFFFFu, th_surv = 0, th_hs = 0;
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const uint32_t j = l0 + k;
    if ((uint32_t)k < K && j < cnt) {
      const bool uniq = f[k] && f[k + 1];
      if (f[k]) {
        th_head = j;
        if (th_first == 0xFFFFFFFFu) th_first = j;
      }
      if (!uniq) {
        ++th_surv;
        if (f[k]) ++th_hs;
      }
    }
  }
  uint32_t ex_head, ex_surv, ex_hs, next_head, tot_surv, tot_hs;
  rf_block_scan4<BLOCK>(th_head, th_surv, th_hs, th_first, S.tmp[1], ex_head, ex_surv, ex_hs,
                        next_head, tot_surv, tot_hs);
  if (next_head > cnt) next_head = cnt;
  uint32_t rend[C::ITEMS];
  {
    uint32_t e = next_head;
#pragma unroll
    for (int k = C::ITEMS - 1; k >= 0; --k) {
      const uint32_t j = l0 + k;
      rend[k] = e;
      if ((uint32_t)k < K && j < cnt && f[k]) e = j;
    }
  }
  // New name of item j (see NamingRule): its subgroup's SA interval is
  // [ghead + (start - goff), ghead + (end - goff)).
  auto name_of = [&](uint32_t lgq, uint32_t start, uint32_t end) -> uint32_t {
    const uint32_t lo = S.ghead[lgq] + (start - S.goff[lgq]);
    if (a.naming != NAMES_RETAIN) return lo;
    const uint32_t len = end - start, old = S.gname[lgq];
    return old - lo < len ? old : lo + len / 2;
  };
  // Changed names are queued in any order: a shared-memory atomic gives
  // each thread its slots, one global atomic the tile's.
  uint32_t th_chg = 0;
  {
    uint32_t rh = ex_head;
#pragma unroll
    for (int k = 0; k < C::ITEMS; ++k) {
      const uint32_t j = l0 + k;
      if ((uint32_t)k < K && j < cnt) {
        if (f[k]) rh = j;
        const uint32_t lgq = (uint32_t)(S.keys[j + (j >> 4)] >> a.W);
        if (name_of(lgq, rh, rend[k]) != S.gname[lgq]) ++th_chg;
      }
    }
  }
  const uint32_t my_chg = th_chg ? atomicAdd(&S.upd_local, th_chg) : 0u;
  __syncthreads();

  // Output space: the next active list only needs each group contiguous, so
  // one 64-bit atomic reserves this tile's survivors (low word) and groups
  // (high word) together, keeping group starts increasing with the group
  // ordinal. Queued updates take one more atomic.
  if (tid == 0) {
    const unsigned long long inc = ((unsigned long long)tot_hs << 32) | tot_surv;
    const unsigned long long old =
        (tot_surv | tot_hs) ? atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctrl->rc.m_s), inc)
                            : 0ull;
    S.surv_base = (uint32_t)old;
    S.grp_base = (uint32_t)(old >> 32);
    S.upd_base = S.upd_local ? atomicAdd(&a.ctrl->rc.upd, S.upd_local) : 0u;
  }
  __syncthreads();
  uint32_t run_head = ex_head;
  uint32_t run_surv = S.surv_base + ex_surv;
  uint32_t run_hs = S.grp_base + ex_hs;
  uint32_t run_chg = S.upd_base + my_chg;
#pragma unroll
  for (int k = 0; k < C::ITEMS; ++k) {
    const uint32_t j = l0 + k;
    if ((uint32_t)k < K && j < cnt) {
      if (f[k]) run_head = j;
      const uint64_t kk = S.keys[j + (j >> 4)];
      uint32_t ip = S.vals[j + (j >> 5)];
      if constexpr (WIDE) ip = S.w.ip[ip];
      const uint32_t lgq = (uint32_t)(kk >> a.W);
      const uint32_t name = name_of(lgq, run_head, rend[k]);
      if (name >= a.N || ip >= a.isa_len) {  // never taken unless a logic error
        raise_error(a.ctrl, ERR_INTERNAL, 10);
        continue;
      }
      if (name != S.gname[lgq]) a.upd[run_chg++] = ((uint64_t)name << 32) | ip;
      if (f[k] && f[k + 1]) {
        a.sa[name] = local_index(ip, a.seg_off, a.S);
      } else {
        if (f[k]) {
          a.gstart_out[run_hs] = run_surv;
          a.gname_out[run_hs] = name;
          a.ghead_out[run_hs] = S.ghead[lgq] + (run_head - S.goff[lgq]);
          ++run_hs;
        }
        a.act_out[run_surv] = ((uint64_t)(run_hs - 1) << 32) | ip;
        ++run_surv;
      }
    }
  }
}

// Up to 8 slots per thread: 64 registers (4 blocks of 256 or 8 of 128 per
// SM); 16 slots: 128 registers (such tiles fit 2 blocks per SM anyway).
// Blocks take tiles blockIdx.x, + gridDim.x, ... (tiles share nothing, so
// any grid works); in device-driven rounds the tile count and h come from
// the round state.
template <int BLOCK, int CAP, bool WIDE, bool PERSIST>
__global__ void __launch_bounds__(BLOCK, (CAP / BLOCK > 8 ? 512 : 1024) / BLOCK)
    k_refine(RefineArgs a) {
  using Sm = RfSmem<BLOCK, CAP, WIDE>;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Sm &S = *reinterpret_cast<Sm *>(smem_raw);
  if constexpr (!PERSIST) {  // one tile per block (host-driven rounds)
    refine_tile<BLOCK, CAP, WIDE>(S, a, blockIdx.x, a.h);
  } else {
    uint32_t tiles = a.tiles, h = a.h;
    if (a.rs) {
      if (!a.rs->live) return;
      tiles = a.rs->tiles;
      h = a.rs->h;
    }
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      refine_tile<BLOCK, CAP, WIDE>(S, a, tile, h);
      __syncthreads();  // the next tile reuses the shared buffers
    }
  }
}

template <int BLOCK, int CAP, bool WIDE, bool PERSIST>
cudaError_t launch_refine_p(const RefineArgs &a, uint32_t grid, cudaStream_t stream) {
  const int smem = (int)sizeof(RfSmem<BLOCK, CAP, WIDE>);
  cudaError_t e = ensure_smem_attributes(
      reinterpret_cast<const void *>(&k_refine<BLOCK, CAP, WIDE, PERSIST>), smem, true);
  if (e != cudaSuccess) return e;
  k_refine<BLOCK, CAP, WIDE, PERSIST><<<grid, BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}

// The one-tile-per-block instance unless the round state or a grid cap
// asks for the looping one (its loop costs the single-tile form registers).
template <int BLOCK, int CAP, bool WIDE>
cudaError_t launch_refine_t(const RefineArgs &a, cudaStream_t stream) {
  if (!a.rs && !a.grid_cap) return launch_refine_p<BLOCK, CAP, WIDE, false>(a, a.tiles, stream);
  const uint32_t grid = a.grid_cap && a.tiles > a.grid_cap ? a.grid_cap : a.tiles;
  return launch_refine_p<BLOCK, CAP, WIDE, true>(a, grid, stream);
}

template <bool WIDE>
cudaError_t launch_refine_w(const RefineArgs &a, cudaStream_t stream) {
  switch (a.shape) {
    case 0: return launch_refine_t<128, 1024, WIDE>(a, stream);
    case 1: return launch_refine_t<256, 2048, WIDE>(a, stream);
    case 2: return launch_refine_t<256, 4096, WIDE>(a, stream);
    case 3: return launch_refine_t<256, 1024, WIDE>(a, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_refine(const RefineArgs &a, cudaStream_t stream) {
  if (a.tiles == 0) return cudaSuccess;
  if (a.mult == 2) return launch_refine_w<false>(a, stream);
  if (a.mult == 3 || a.mult == 4) return launch_refine_w<true>(a, stream);
  return cudaErrorInvalidValue;
}

// ---- ISA writes of new names ------------------------------------------------
// One block per 2048-entry chunk, 8 independent entries per thread; blocks
// start in chunk order, so after position bucketing the ISA being written
// stays a narrow window.

constexpr int WB_ITEMS = 8;
constexpr int WB_CHUNK = 256 * WB_ITEMS;

// Blocks take chunks blockIdx.x, + gridDim.x, ...; with one block per chunk
// they start in chunk order. In device-driven rounds (rs) the kernels read
// from the position-bucketed copy when the round state says the round
// bucketed its entries.
__global__ void __launch_bounds__(256) k_apply_names(const uint64_t *__restrict__ act,
                                                    const uint32_t *lo_p, const uint32_t *count_p,
                                                    const uint32_t *__restrict__ gname,
                                                    const uint32_t *__restrict__ gold,
                                                    uint32_t *isa, uint64_t isa_len,
                                                    uint32_t translated,
                                                    const uint64_t *__restrict__ bucketed,
                                                    const uint32_t *zero,
                                                    const uint32_t *bucketed_count,
                                                    const RoundState *rs) {
  if (rs) {
    if (!rs->live || rs->mL == 0) return;
    if (rs->bucket_surv) {
      act = bucketed;
      lo_p = zero;
      count_p = bucketed_count;
      translated = 1;
    }
  }
  const uint64_t lo = *lo_p, n = *count_p;
  if (translated) {  // (name << 32) | i', every one a change
    for (uint64_t c0 = (uint64_t)blockIdx.x * WB_CHUNK; c0 < n;
         c0 += (uint64_t)gridDim.x * WB_CHUNK) {
      uint64_t e[WB_ITEMS];
#pragma unroll
      for (int k = 0; k < WB_ITEMS; ++k) {
        const uint64_t x = c0 + (uint64_t)k * 256 + threadIdx.x;
        e[k] = x < n ? act[lo + x] : ~0ull;
      }
#pragma unroll
      for (int k = 0; k < WB_ITEMS; ++k) {
        const uint32_t ip = (uint32_t)e[k];
        if (e[k] != ~0ull && ip < isa_len) isa[ip] = (uint32_t)(e[k] >> 32);
      }
    }
    return;
  }
  for (uint64_t c0 = (uint64_t)blockIdx.x * WB_CHUNK; c0 < n;
       c0 += (uint64_t)gridDim.x * WB_CHUNK) {
    uint64_t e[WB_ITEMS];
#pragma unroll
    for (int k = 0; k < WB_ITEMS; ++k) {
      const uint64_t x = c0 + (uint64_t)k * 256 + threadIdx.x;
      e[k] = x < n ? act[lo + x] : ~0ull;
    }
#pragma unroll
    for (int k = 0; k < WB_ITEMS; ++k) {
      if (e[k] == ~0ull) continue;
      const uint32_t g = (uint32_t)(e[k] >> 32), ip = (uint32_t)e[k];
      const uint32_t name = __ldg(gname + g);
      if (name != __ldg(gold + g) && ip < isa_len) isa[ip] = name;
    }
  }
}

cudaError_t launch_apply_names(const uint64_t *act, const uint32_t *lo, const uint32_t *count,
                               uint32_t max_count, const uint32_t *gname, const uint32_t *gold,
                               uint32_t *isa, uint64_t isa_len, cudaStream_t stream,
                               uint32_t translated, const uint64_t *bucketed,
                               const uint32_t *zero, const uint32_t *bucketed_count,
                               const RoundState *rs, uint32_t grid_cap) {
  uint64_t blocks = ((uint64_t)max_count + WB_CHUNK - 1) / WB_CHUNK;
  if (blocks == 0) return cudaSuccess;
  if (grid_cap && blocks > grid_cap) blocks = grid_cap;
  k_apply_names<<<(unsigned)blocks, 256, 0, stream>>>(act, lo, count, gname, gold, isa, isa_len,
                                                      translated, bucketed, zero, bucketed_count,
                                                      rs);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_scatter_updates(const uint64_t *__restrict__ upd,
                                                        uint32_t max_upd, uint32_t *isa,
                                                        uint64_t isa_len, Ctrl *ctrl,
                                                        const uint64_t *__restrict__ bucketed,
                                                        const RoundState *rs) {
  if (rs) {
    if (!rs->live) return;
    if (rs->bucket_upd) upd = bucketed;
  }
  const uint64_t n = min(ctrl->rc.upd, max_upd);
  for (uint64_t c0 = (uint64_t)blockIdx.x * WB_CHUNK; c0 < n;
       c0 += (uint64_t)gridDim.x * WB_CHUNK) {
    uint64_t u[WB_ITEMS];
#pragma unroll
    for (int k = 0; k < WB_ITEMS; ++k) {
      const uint64_t x = c0 + (uint64_t)k * 256 + threadIdx.x;
      u[k] = x < n ? upd[x] : ~0ull;
    }
#pragma unroll
    for (int k = 0; k < WB_ITEMS; ++k) {
      const uint32_t ip = (uint32_t)u[k];
      if (u[k] != ~0ull && ip < isa_len) isa[ip] = (uint32_t)(u[k] >> 32);
    }
  }
}

cudaError_t launch_scatter_updates(const uint64_t *upd, uint32_t max_upd, uint32_t *isa,
                                   uint64_t isa_len, Ctrl *ctrl, cudaStream_t stream,
                                   const uint64_t *bucketed, const RoundState *rs,
                                   uint32_t grid_cap) {
  uint64_t blocks = ((uint64_t)max_upd + WB_CHUNK - 1) / WB_CHUNK;
  if (blocks == 0) return cudaSuccess;
  if (grid_cap && blocks > grid_cap) blocks = grid_cap;
  k_scatter_updates<<<(unsigned)blocks, 256, 0, stream>>>(upd, max_upd, isa, isa_len, ctrl,
                                                          bucketed, rs);
  return cudaGetLastError();
}

}  // namespace gbsa
