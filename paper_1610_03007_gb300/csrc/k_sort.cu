// Step A2 — stable LSD radix sort of (64-bit key, 32-bit value) pairs: the
// "sort triples by name pair" step of prefix doubling (Section 2.1,
// Algorithm 1; Algorithm 5 sorts only the undiscarded items).
//
// One-sweep structure (Adinets & Merrill, "Onesweep: A Faster Least
// Significant Digit Radix Sort for GPUs", 2022), written from that
// description:
//   1. k_digit_histogram: one read of all keys builds the 256-bin histogram
//      of every digit position at once.
//   2. k_sort_plan (one block): exclusive digit offsets per pass; a digit
//      position whose keys all share one value is skipped; the source and
//      destination buffers of the remaining passes ping-pong A <-> B.
//   3. k_onesweep per kept pass: each tile of 256 x 8..16 items ranks its items by
//      digit (peers of equal digit by shared-memory masks or match.any, so
//      the local order is stable), publishes its per-digit counts, finds its per-digit
//      global offsets by decoupled look-back over the preceding tiles, stages
//      the tile in shared memory in digit order and writes each digit run
//      with consecutive addresses.
//
// Bound: HBM. Per pass: 12 bytes read + 12 bytes written per item; the
// histogram reads 8 bytes per item once per sort.
#include "launch.h"

namespace gbsa {

// ---- 1. histogram of every digit position --------------------------------

constexpr int DH_BLOCK = 256;

__global__ void __launch_bounds__(DH_BLOCK)
k_digit_histogram(const uint64_t *__restrict__ keys, uint32_t m, DigitSpec spec,
                  uint32_t *__restrict__ hist, const RoundState *rs) {
  __shared__ uint32_t s_hist[MAX_PASSES][RADIX];
  if (rs) {  // device-driven rounds: the large groups' items and digits
    if (!rs->live) return;
    m = rs->mL;
    spec = rs->spec;
  }
  for (int x = threadIdx.x; x < MAX_PASSES * RADIX; x += DH_BLOCK) (&s_hist[0][0])[x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t P = spec.P;
  const uint64_t stride = (uint64_t)gridDim.x * DH_BLOCK;
  // Every lane of a warp runs the same number of iterations so the votes
  // below see the whole warp; lanes past the end carry no item.
  const uint64_t warp_base = (uint64_t)blockIdx.x * DH_BLOCK + (threadIdx.x & ~31u);
  for (uint64_t w0 = warp_base; w0 < m; w0 += stride) {
    const uint64_t j = w0 + lane;
    const bool valid = j < m;
    const uint64_t key = valid ? keys[j] : 0ull;
    const uint32_t nvalid = __popc(__ballot_sync(0xffffffffu, valid));
    for (uint32_t p = 0; p < P; ++p) {
      const uint32_t d = digit_of(key, spec.shift[p], spec.bits[p]);
      const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
      // Runs of equal digits are common (sorted group ids): one atomic per warp.
      if (__all_sync(0xffffffffu, !valid || d == d0)) {
        if (lane == 0) atomicAdd(&s_hist[p][d0], nvalid);
      } else if (valid) {
        atomicAdd(&s_hist[p][d], 1u);
      }
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < P * RADIX; x += DH_BLOCK) {
    uint32_t v = (&s_hist[0][0])[x];
    if (v) atomicAdd(&hist[x], v);
  }
}

cudaError_t launch_digit_histogram(const uint64_t *keys, uint32_t m, const DigitSpec &spec,
                                   uint32_t *hist, int num_sms, cudaStream_t stream,
                                   const RoundState *rs) {
  if (m == 0 || (spec.P == 0 && !rs)) return cudaSuccess;
  uint64_t want = ((uint64_t)m + DH_BLOCK - 1) / DH_BLOCK;
  uint64_t cap = (uint64_t)num_sms * 8;
  unsigned grid = (unsigned)(want > cap ? cap : want);
  k_digit_histogram<<<grid, DH_BLOCK, 0, stream>>>(keys, m, spec, hist, rs);
  return cudaGetLastError();
}

// ---- 2. plan ---------------------------------------------------------------

// Passes whose digits a 32-key warp is expected to spread over at most this
// many values rank with match.any (repeated Zipf bytes: about 20; uniform
// DNA or bytes: 28 to 30, where the masks measured faster).
constexpr float MATCH_RANK_MAX_DISTINCT = 24.f;

__global__ void __launch_bounds__(RADIX)
k_sort_plan(const uint32_t *__restrict__ hist, uint32_t *__restrict__ digit_base, DigitSpec spec,
            uint32_t m, uint64_t *ka, uint64_t *kb, uint32_t *va, uint32_t *vb,
            SortPlan *plan, Ctrl *ctrl, const RoundState *rs, uint32_t keep_first) {
  __shared__ uint32_t s_tmp[RADIX / 32 + 1];
  if (rs) {  // device-driven rounds
    if (!rs->live) return;
    m = rs->mL;
    spec = rs->spec;
  }
  __shared__ uint32_t s_active[MAX_PASSES];
  __shared__ float s_e[RADIX / 32];
  __shared__ uint32_t s_match;
  const uint32_t d = threadIdx.x;
  if (d == 0) s_match = 0u;
  for (uint32_t p = 0; p < spec.P; ++p) {
    const uint32_t c = hist[p * RADIX + d];
    uint32_t total;
    const uint32_t excl = block_exclusive<RADIX>(c, OpAdd(), 0u, s_tmp, total);
    digit_base[p * RADIX + d] = excl;
    // A digit position is constant iff one bin holds every key.
    const int constant = __syncthreads_or(c == m);
    if (d == 0) s_active[p] = constant && !(keep_first && p == 0) ? 0u : 1u;
    // Expected distinct digits among 32 keys drawn from this histogram:
    // sum over d of 1 - (1 - p_d)^32. Few (a skewed alphabet) -> the pass
    // ranks with match.any, else with the shared-memory masks.
    float q = m ? 1.f - (float)c / (float)m : 1.f;
    q *= q;
    q *= q;
    q *= q;
    q *= q;
    q *= q;
    float e = 1.f - q;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((d & 31) == 0) s_e[d >> 5] = e;
    __syncthreads();
    if (d == 0) {
      float all = 0.f;
      for (int w = 0; w < RADIX / 32; ++w) all += s_e[w];
      if (all <= MATCH_RANK_MAX_DISTINCT) s_match |= 1u << p;
    }
    __syncthreads();
  }
  __syncthreads();
  if (d == 0) {
    uint32_t cur = 0, kept = 0, mask = 0;
    uint64_t *k[2] = {ka, kb};
    uint32_t *v[2] = {va, vb};
    for (uint32_t p = 0; p < MAX_PASSES; ++p) {
      const uint32_t act = p < spec.P ? s_active[p] : 0u;
      plan->active[p] = act;
      plan->ksrc[p] = k[cur];
      plan->vsrc[p] = v[cur];
      plan->kdst[p] = k[cur ^ 1];
      plan->vdst[p] = v[cur ^ 1];
      if (act) {
        cur ^= 1;
        ++kept;
        mask |= 1u << p;
      }
    }
    plan->n_active = kept;
    plan->match_mask = s_match;
    plan->final_idx = cur;
    plan->kfinal = k[cur];
    plan->vfinal = v[cur];
    ctrl->passes = kept;
    ctrl->pass_mask = mask;
  }
}

cudaError_t launch_sort_plan(const uint32_t *hist, uint32_t *digit_base, const DigitSpec &spec,
                             uint32_t m, uint64_t *ka, uint64_t *kb, uint32_t *va,
                             uint32_t *vb, SortPlan *plan, Ctrl *ctrl, cudaStream_t stream,
                             const RoundState *rs, bool keep_first) {
  k_sort_plan<<<1, RADIX, 0, stream>>>(hist, digit_base, spec, m, ka, kb, va, vb, plan, ctrl, rs,
                                       keep_first ? 1u : 0u);
  return cudaGetLastError();
}

// ---- 3. one-sweep pass -----------------------------------------------------

constexpr int OS_BLOCK = 256;  // == RADIX: thread d owns digit d in the look-back
constexpr int OS_WARPS = OS_BLOCK / 32;
static_assert(OS_BLOCK == RADIX, "one thread per digit");
#ifndef GBSA_LB_WINDOW
#define GBSA_LB_WINDOW 4
#endif
// Predecessors read per look-back round trip (4 independent 8-byte loads
// per digit thread).
constexpr int LB_WINDOW = GBSA_LB_WINDOW;

template <int OS_ITEMS>
struct OsSmem {
  static constexpr int OS_TILE = OS_BLOCK * OS_ITEMS;
  uint64_t keys[OS_TILE];           // tile in input order, then in digit order
  uint32_t vals[OS_TILE];
  uint32_t match[OS_WARPS][RADIX];  // per-warp peer masks (zero between uses)
  uint16_t whist[OS_WARPS][RADIX];  // per-warp counts, then each warp's first slot per digit
  uint32_t goff[RADIX];             // global index of a run = goff + local index
  uint32_t tmp[OS_WARPS + 1];
  uint32_t tile;
  uint32_t bail;
  uint64_t bar;                     // completion of the tile's bulk copies
};

// Index j of round 0's keys over one text (PassArgs.text): the tail
// position n-1-j for j < tails, else position j - tails (k_pack.cu's layout).
__device__ __forceinline__ uint32_t text_position(uint64_t j, uint32_t tails, uint64_t n) {
  return (uint32_t)(j < tails ? n - 1 - j : j - tails);
}

// The keys of one tile built from the text (the first pass of round 0): the
// dense codes of the characters the tile's keys cover are packed MSB-first
// into 32-bit words in shared memory (the key buffer, unused until the
// scatter), and each key is the cb bits at its position's bit offset: three
// word reads and a funnel shift. Tail keys (tile 0 only) read their few
// characters directly. Items past the end read as all ones.
template <int OS_ITEMS>
__device__ __forceinline__ void text_keys(OsSmem<OS_ITEMS> &S, const PassArgs &a, uint64_t base,
                                          uint32_t count, uint64_t n,
                                          uint64_t (&key)[OS_ITEMS]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t *s_code = reinterpret_cast<uint8_t *>(S.vals);
  uint32_t *words = reinterpret_cast<uint32_t *>(S.keys);
  const uint32_t b = a.b, cpw = 32 / b, t = a.tails;
  s_code[tid] = a.code[tid];
  __syncthreads();
  // Non-tail indices [jl, jh) hold positions [jl - t, jh - t); their keys
  // read characters [jl - t, jh - t + c0 - 1), all inside the text.
  const uint64_t jl = base > t ? base : (uint64_t)t, jh = base + count;
  uint64_t w0 = 0;
  if (jl < jh) {
    w0 = (jl - t) / cpw;
    const uint64_t c_end = jh - t + a.c0 - 1;
    const uint32_t nw = (uint32_t)((c_end + cpw - 1) / cpw - w0) + 2;
    // A word's cpw (>= 4) characters start at a multiple of 4: 4-byte loads
    // when the text is 4-byte aligned, bytes at the end of the text.
    const bool v4 = (reinterpret_cast<uintptr_t>(a.text) & 3u) == 0;
    for (uint32_t x = tid; x < nw; x += OS_BLOCK) {
      const uint64_t c = (w0 + x) * cpw;
      uint32_t w = 0;
      if (v4 && c + cpw <= n) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.text + c);
        for (uint32_t q = 0; q < cpw / 4; ++q) {
          const uint32_t v = __ldg(src + q);
#pragma unroll
          for (int k = 0; k < 4; ++k) w = (w << b) | s_code[(v >> (8 * k)) & 0xFFu];
        }
      } else {
        for (uint32_t q = 0; q < cpw; ++q)
          w = (w << b) | (c + q < n ? (uint32_t)s_code[__ldg(a.text + c + q)] : 0u);
      }
      words[x] = w;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < OS_ITEMS; ++k) {
    const uint32_t li = warp * (32 * OS_ITEMS) + k * 32 + lane;
    const uint64_t j = base + li;
    if (li >= count) {
      key[k] = ~0ull;
    } else if (j >= t) {
      const uint64_t o = (j - t - w0 * cpw) * b;  // bit offset in the window
      const uint32_t w = (uint32_t)(o >> 5), r = (uint32_t)(o & 31);
      const uint32_t w0v = words[w], w1v = words[w + 1], w2v = words[w + 2];
      // the 64 bits from bit r of w0v:w1v:w2v, as two funnel shifts
      const uint64_t x =
          ((uint64_t)__funnelshift_l(w1v, w0v, r) << 32) | __funnelshift_l(w2v, w1v, r);
      key[k] = a.cb >= 64 ? x : x >> (64 - a.cb);
    } else {  // tail: j + 1 characters left, zero-padded
      const uint64_t p = n - 1 - j;
      uint64_t kk = 0;
      for (uint32_t q = 0; q <= (uint32_t)j; ++q)
        kk |= (uint64_t)s_code[__ldg(a.text + p + q)] << (a.cb - b * (q + 1));
      key[k] = kk;
    }
  }
}

// OS_ITEMS keys per thread (8, 12 or 16; chosen per build): 16 fits three
// blocks per SM (~62 KB of shared memory each), 12 four, 8 five; registers
// are capped to match.
//
// FROM_TEXT: the first pass of round 0 over one text builds its keys from
// the text (text_keys) and its values are the positions, so the packed keys
// are never written and read back.
template <int OS_ITEMS, bool PERSIST, bool FROM_TEXT>
__global__ void __launch_bounds__(OS_BLOCK, OS_ITEMS >= 16 ? 3 : (OS_ITEMS >= 12 ? 4 : 5))
    k_onesweep(PassArgs a) {
  constexpr int OS_TILE = OS_BLOCK * OS_ITEMS;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  OsSmem<OS_ITEMS> &S = *reinterpret_cast<OsSmem<OS_ITEMS> *>(smem_raw);
  if (!a.plan->active[a.p]) return;
  // Sizes and digit: from the arguments, or in device-driven rounds from
  // the round state (the pass's launch epoch is then an offset).
  uint32_t m = a.m, shift = a.shift, bits = a.bits, epoch = a.epoch;
  if (a.rs) {
    if (!a.rs->live) return;
    m = a.rs->mL;
    shift = a.rs->spec.shift[a.p];
    bits = a.rs->spec.bits[a.p];
    epoch = a.rs->epoch + a.epoch;
  }
  const uint32_t tiles = (uint32_t)(((uint64_t)m + OS_TILE - 1) / OS_TILE);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) mbar_init(&S.bar, 1);
  const uint64_t *__restrict__ ksrc = a.plan->ksrc[a.p];
  const uint32_t *__restrict__ vsrc = a.plan->vsrc[a.p];
  uint64_t *__restrict__ kdst = a.plan->kdst[a.p];
  uint32_t *__restrict__ vdst = a.plan->vdst[a.p];
  const uint32_t dmax = (1u << bits) - 1u;
  uint32_t phase = 0;  // parity of the tile-load barrier's next phase
  // Tiles are taken from the launch's counter until it passes the last one
  // (a grid smaller than the tile count makes the blocks persistent).
  for (;;) {
    if (tid == 0) {
      S.tile = atomicAdd(a.tile_ctr, 1u);
      S.bail = has_error(a.ctrl) ? 1u : 0u;
    }
    for (int x = tid; x < OS_WARPS * RADIX; x += OS_BLOCK) {
      (&S.whist[0][0])[x] = 0;
      (&S.match[0][0])[x] = 0u;
    }
    __syncthreads();
    if (S.bail || S.tile >= tiles) return;
    const uint32_t tile = S.tile;
    const uint64_t base = (uint64_t)tile * OS_TILE;
    const uint32_t count = (uint32_t)min((uint64_t)OS_TILE, (uint64_t)m - base);

    uint64_t key[OS_ITEMS];
    uint32_t pos[OS_ITEMS];
    if constexpr (FROM_TEXT) {
      text_keys<OS_ITEMS>(S, a, base, count, m, key);
    } else {
      // Load the tile: one bulk copy each for keys and values (TMA, 16-byte
      // granules), plain loads for a ragged remainder or unaligned arrays. A
      // block's earlier tile wrote these buffers through ordinary stores, so
      // the copy is ordered after them by a proxy fence.
      const uint64_t *kp = ksrc + base;
      const uint32_t *vp = vsrc + base;
      const bool aligned = ((((uintptr_t)kp) | ((uintptr_t)vp)) & 15u) == 0;
      const uint32_t kbytes = aligned ? (count * 8u) & ~15u : 0u;
      const uint32_t vbytes = aligned ? (count * 4u) & ~15u : 0u;
      if (tid == 0 && (kbytes | vbytes)) {
        fence_proxy_async_shared();
        mbar_expect_tx(&S.bar, kbytes + vbytes);
        if (kbytes) bulk_g2s(S.keys, kp, kbytes, &S.bar);
        if (vbytes) bulk_g2s(S.vals, vp, vbytes, &S.bar);
      }
      for (uint32_t e = kbytes / 8u + tid; e < count; e += OS_BLOCK) S.keys[e] = kp[e];
      for (uint32_t e = vbytes / 4u + tid; e < count; e += OS_BLOCK) S.vals[e] = vp[e];
      if (kbytes | vbytes) {
        if (!mbar_wait_bounded(&S.bar, phase, a.ctrl, a.spin_limit)) S.bail = 1;
        phase ^= 1u;
      }
      __syncthreads();
      if (S.bail) return;

      // Warp-striped items: item k of lane l at warp*32*ITEMS + k*32 + l, so
      // the order (warp, k, lane) is the input order inside the tile. Items
      // past the end read as all ones: they take the largest digit and come
      // last in the tile.
#pragma unroll
      for (int k = 0; k < OS_ITEMS; ++k) {
        const uint32_t li = warp * (32 * OS_ITEMS) + k * 32 + lane;
        key[k] = li < count ? S.keys[li] : ~0ull;
      }
    }
    const uint32_t d = tid;  // thread d owns digit d and its status word
    uint64_t *st = a.status + (uint64_t)tile * RADIX + d;

    // Rank within the tile: stable, by per-warp peers and counts (peers by
    // match.any on the plan's low-entropy passes, else by the masks).
    uint16_t *wh = S.whist[warp];
    uint32_t *mt = S.match[warp];
    const uint32_t lt = lanemask_lt();
    if ((a.plan->match_mask >> a.p) & 1u) {
#pragma unroll
      for (int k = 0; k < OS_ITEMS; ++k)
        pos[k] = warp_rank_digit_match(digit_of(key[k], shift, bits), wh, lt);
    } else {
#pragma unroll
      for (int k = 0; k < OS_ITEMS; ++k)
        pos[k] = warp_rank_digit(digit_of(key[k], shift, bits), mt, wh, lane, lt);
    }
    __syncthreads();

    // Thread d: counts of digit d per warp -> per-warp exclusive prefixes;
    // their sum is the tile's count of digit d, published now (taking the
    // counts from the ranking instead of by one shared-memory atomic per key
    // before it measured 6 % faster on DNA: the atomics collide on banks).
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) {
      const uint32_t c = S.whist[w][d];
      S.whist[w][d] = (uint16_t)total;
      total += c;
    }
    const uint32_t mine = total;
    if (a.inject && tile == 0) {
      // Test hook: this tile never publishes, so the next tile's wait expires.
      if (d == 0) S.bail = 1;
    } else {
      status_store(st, status_word(epoch, tile == 0 ? ST_INC : ST_AGG, mine));
    }
    uint32_t tile_total;
    const uint32_t start = block_exclusive<OS_BLOCK>(total, OpAdd(), 0u, S.tmp, tile_total);
    // Each warp's first slot per digit = run start + warp prefix (< 2^16:
    // a tile holds at most 4096 keys), so placing a key takes one
    // digit-indexed load.
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) S.whist[w][d] = (uint16_t)(S.whist[w][d] + start);
    __syncthreads();

    // Permute the tile into digit order in place (every key of the input
    // order is in registers since the ranking), values after every read of
    // their input order. This needs no global offsets, so it runs before
    // the look-back: the predecessors get that much longer to publish.
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
      const uint32_t li = warp * (32 * OS_ITEMS) + k * 32 + lane;
      const uint32_t dk = li < count ? digit_of(key[k], shift, bits) : dmax;
      pos[k] += S.whist[warp][dk];
      S.keys[pos[k]] = key[k];
    }
    uint32_t val[OS_ITEMS];
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
      const uint32_t li = warp * (32 * OS_ITEMS) + k * 32 + lane;
      if constexpr (FROM_TEXT)
        val[k] = li < count ? text_position(base + li, a.tails, m) : 0u;
      else
        val[k] = li < count ? S.vals[li] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) S.vals[pos[k]] = val[k];

    // Look back over the predecessors.
    if (!S.bail) {
      if (tile == 0) {
        S.goff[d] = a.digit_base[d] - start;
      } else {
        uint32_t excl = 0;
        if (look_back_w<LB_WINDOW>(a.status, RADIX, d, tile, epoch, OpAdd(), excl, a.ctrl,
                                   a.spin_limit)) {
          status_store(st, status_word(epoch, ST_INC, excl + mine));
          S.goff[d] = a.digit_base[d] + excl - start;
        } else {
          S.bail = 1;
        }
      }
    }
    __syncthreads();
    if (S.bail) return;

    // Write each digit run with consecutive addresses.
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
      const uint32_t q = k * OS_BLOCK + tid;
      if (q < count) {
        const uint64_t kk = S.keys[q];
        const uint32_t g = S.goff[digit_of(kk, shift, bits)] + q;
        if (g < m) {
          kdst[g] = kk;
          vdst[g] = S.vals[q];
        } else {  // never taken unless the histogram and the pass disagree
          raise_error(a.ctrl, ERR_INTERNAL, 2);
        }
      }
    }
    if constexpr (!PERSIST) return;  // one tile per block: no second claim
    __syncthreads();  // the next tile reuses the shared buffers
  }
}

template <int OS_ITEMS>
cudaError_t launch_onesweep_t(const PassArgs &a, cudaStream_t stream) {
  const int smem = (int)sizeof(OsSmem<OS_ITEMS>);
  const uint64_t tile = (uint64_t)OS_BLOCK * OS_ITEMS;
  const uint64_t tiles = ((uint64_t)a.m + tile - 1) / tile;
  if (a.text) {  // the first pass of round 0 over one text (never persistent)
    if (a.p != 0 || a.rs || a.b == 0 || 32 % a.b != 0 || a.cb == 0 || a.cb > 64)
      return cudaErrorInvalidValue;
    const void *fn = reinterpret_cast<const void *>(&k_onesweep<OS_ITEMS, false, true>);
    cudaError_t e = ensure_smem_attributes(fn, smem, true);
    if (e != cudaSuccess) return e;
    k_onesweep<OS_ITEMS, false, true><<<(unsigned)tiles, OS_BLOCK, smem, stream>>>(a);
    return cudaGetLastError();
  }
  // One tile per block unless the grid is capped (persistent blocks loop).
  const bool persist = a.grid_cap && tiles > a.grid_cap;
  const void *fn = persist ? reinterpret_cast<const void *>(&k_onesweep<OS_ITEMS, true, false>)
                           : reinterpret_cast<const void *>(&k_onesweep<OS_ITEMS, false, false>);
  cudaError_t e = ensure_smem_attributes(fn, smem, true);
  if (e != cudaSuccess) return e;
  if (persist)
    k_onesweep<OS_ITEMS, true, false><<<a.grid_cap, OS_BLOCK, smem, stream>>>(a);
  else
    k_onesweep<OS_ITEMS, false, false><<<(unsigned)tiles, OS_BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_onesweep(const PassArgs &a, cudaStream_t stream) {
  if (a.m == 0) return cudaSuccess;
  switch (a.items) {
    case 8: return launch_onesweep_t<8>(a, stream);
    case 12: return launch_onesweep_t<12>(a, stream);
    case 16: return launch_onesweep_t<16>(a, stream);
  }
  return cudaErrorInvalidValue;
}

// ---- copy-back for the standalone sort ------------------------------------

// When the last kept pass left the result in buffer B, copy it to A (the
// caller's arrays). The decision is read from the device plan.
__global__ void k_copy_back(const SortPlan *__restrict__ plan, uint64_t *__restrict__ ka,
                            uint32_t *__restrict__ va, uint32_t m) {
  if (plan->final_idx == 0) return;
  const uint64_t *kb = plan->kfinal;
  const uint32_t *vb = plan->vfinal;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (uint64_t)gridDim.x * blockDim.x) {
    ka[j] = kb[j];
    va[j] = vb[j];
  }
}

cudaError_t launch_copy_back(const SortPlan *plan, uint64_t *ka, uint32_t *va, uint32_t m,
                             int num_sms, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  uint64_t want = ((uint64_t)m + 255) / 256, cap = (uint64_t)num_sms * 8;
  k_copy_back<<<(unsigned)(want > cap ? cap : want), 256, 0, stream>>>(plan, ka, va, m);
  return cudaGetLastError();
}

}  // namespace gbsa
