// Step A1 — initial keys (Section 2.1, Algorithm 1: the initial name pairs
// (T[i], T[i+1]); here c0 characters per key instead of 2).
//
// key = (text id << c0*b) | the dense codes of T[i .. i+c0), first
// character most significant, zero-padded past the end of the text.
//
// Padding with code 0 lets a short suffix near the end tie with a longer
// suffix whose next characters have code 0. Such a tail suffix (fewer than
// c0 characters left) is smaller than every longer suffix with the same key,
// and among tails with equal keys the shorter is smaller. So keys are laid
// out tail-first within each text: the c0-1 last positions in descending
// order, then the others ascending. The stable sort keeps that order inside
// runs of equal keys, and the round-0 rename gives every tail a group of
// its own.
//
// vals hold gapped positions: text s occupies [off_s + s, off_s + s + len_s)
// and the slot right after it is an end sentinel of the ISA.
//
// Bound: HBM, N bytes read (+ L1-cached overlap of c0-1 bytes per key),
// 12 N bytes written; the digit histograms of the following sort are
// accumulated in shared memory on the way.
#include "launch.h"

namespace gbsa {

constexpr int PACK_BLOCK = 256;
// Keys of at least this many characters take the sliding fast path (for
// short keys the per-key loads are already few, and the warp-strided stores
// of the general path coalesce better: measured 2.89 vs 3.35 ms for 8-char
// keys at 2^28; 33.9 vs 27.8 ms for 32-char keys at 2^31).
constexpr uint32_t PACK_SLIDE_MIN = 16;

// Digit histograms of one key (warp-aggregated when a warp shares a digit).
// With top_only, only the most significant digit's (the others follow from
// it, k_pack_hist_fixup).
__device__ __forceinline__ void pack_hist(uint32_t (*s_hist)[RADIX], const DigitSpec &spec,
                                          uint64_t key, bool valid, int lane, bool top_only) {
  const uint32_t nvalid = __popc(__ballot_sync(0xffffffffu, valid));
  for (uint32_t p = top_only ? spec.P - 1 : 0; p < spec.P; ++p) {
    const uint32_t d = digit_of(key, spec.shift[p], spec.bits[p]);
    const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
    if (__all_sync(0xffffffffu, !valid || d == d0)) {
      if (lane == 0 && nvalid) atomicAdd(&s_hist[p][d0], nvalid);
    } else if (valid) {
      atomicAdd(&s_hist[p][d], 1u);
    }
  }
}

// One block packs PACK_BLOCK * ITEMS consecutive keys. The 256-bin histograms of
// every radix digit of the keys (the one-sweep sort's upfront histogram)
// are accumulated here as well, so the sort needs no separate read of the
// keys.
//
// Fast path (keys of PACK_SLIDE_MIN or more characters, the block's keys
// all in one text's non-tail range, where index j holds position j - t and
// every key has c0 characters): the text
// window is staged once in shared memory as dense codes, and each thread
// builds ITEMS consecutive keys by sliding, one character shifted in
// per key. Otherwise the text of the block's first and last key is found
// once, and each key is assembled from its own characters.
//
// ITEMS keys per thread: 16 where the sliding path applies (longer slides
// amortise the c0 - 1 characters each thread reads before its first key:
// 12.2 -> 10.5 ms for 24-character keys at 2^31), 8 otherwise (the
// per-key path's stores coalesce better with more blocks: 1.96 vs 2.31 ms
// for 8-character keys at 2^28).
template <int ITEMS>
__global__ void __launch_bounds__(PACK_BLOCK) k_pack(PackArgs a) {
  constexpr int PACK_SPAN = PACK_BLOCK * ITEMS;
  __shared__ uint8_t s_code[RADIX];
  __shared__ uint32_t s_hist[MAX_PASSES][RADIX];
  __shared__ uint32_t s_seg[2];
  __shared__ uint8_t s_txt[PACK_SPAN + 64];
  // Fast path: the block's keys, key x at x + x / ITEMS (the k-th keys
  // of a warp's threads fall in distinct banks), written out with
  // consecutive addresses.
  __shared__ uint64_t s_keys[PACK_SPAN + PACK_SPAN / ITEMS];
  const int tid = threadIdx.x, lane = tid & 31;
  s_code[tid] = a.code[tid];
  for (int x = tid; x < MAX_PASSES * RADIX; x += PACK_BLOCK) (&s_hist[0][0])[x] = 0;
  const uint64_t j0 = (uint64_t)blockIdx.x * PACK_SPAN;
  const uint64_t jl = min(j0 + PACK_SPAN, (uint64_t)a.N) - 1;
  if (tid < 2) s_seg[tid] = a.S > 1 ? segment_of(a.seg_off, a.S, (uint32_t)(tid == 0 ? j0 : jl)) : 0u;
  __syncthreads();
  const uint32_t s_lo = s_seg[0], s_hi = s_seg[1];

  // Fast-path test (block-uniform).
  bool fast = false;
  uint32_t f_off = 0, f_t = 0;
  if (s_lo == s_hi && a.c0 >= PACK_SLIDE_MIN && a.c0 <= 64) {
    f_off = __ldg(a.seg_off + s_lo);
    const uint32_t len = __ldg(a.seg_off + s_lo + 1) - f_off;
    f_t = len < a.c0 - 1 ? len : a.c0 - 1;
    fast = len >= a.c0 && j0 >= (uint64_t)f_off + f_t;
  }
  if (fast) {
    const uint64_t pos0 = j0 - f_t;                    // text position of index j0
    const uint32_t span = (uint32_t)(jl - j0 + 1);
    const uint32_t need = span + a.c0 - 1;             // characters of the window
    for (uint32_t x = tid; x < need; x += PACK_BLOCK) s_txt[x] = s_code[__ldg(a.text + pos0 + x)];
    __syncthreads();
    const uint64_t mask = a.cb >= 64 ? ~0ull : ((1ull << a.cb) - 1ull);
    const uint64_t segbits = a.S > 1 ? (uint64_t)s_lo << a.cb : 0ull;
    const uint32_t x0 = (uint32_t)tid * ITEMS;
    uint64_t key = 0;
    if (x0 < span)
      for (uint32_t q = 0; q + 1 < a.c0; ++q) key = (key << a.b) | s_txt[x0 + q];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t x = x0 + k;
      const bool valid = x < span;
      uint64_t out = 0;
      if (valid) {
        key = ((key << a.b) | s_txt[x + a.c0 - 1]) & mask;
        out = key | segbits;
        s_keys[x + x / ITEMS] = out;
      }
      pack_hist(s_hist, a.spec, out, valid, lane, a.top_only != 0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t x = (uint32_t)k * PACK_BLOCK + tid;
      if (x < span) {
        a.keys[j0 + x] = s_keys[x + x / ITEMS];
        a.vals[j0 + x] = (uint32_t)(pos0 + x) + s_lo;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint64_t j64 = j0 + (uint64_t)k * PACK_BLOCK + tid;
      const bool valid = j64 < a.N;
      uint64_t key = 0;
      if (valid) {
        const uint32_t j = (uint32_t)j64;
        uint32_t s = s_lo;
        if (s_hi != s_lo) {  // the last s in [s_lo, s_hi] with seg_off[s] <= j
          uint32_t lo = s_lo, hi = s_hi;
          while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (__ldg(a.seg_off + mid) <= j)
              lo = mid;
            else
              hi = mid - 1;
          }
          s = lo;
        }
        const uint32_t off = __ldg(a.seg_off + s);
        const uint32_t len = __ldg(a.seg_off + s + 1) - off;
        const uint32_t rel = j - off;
        const uint32_t t = len < a.c0 - 1 ? len : a.c0 - 1;  // tail positions of this text
        const uint32_t irel = rel < t ? len - 1 - rel : rel - t;
        const uint32_t avail = len - irel;
        const uint32_t take = avail < a.c0 ? avail : a.c0;
        const uint8_t *p = a.text + off + irel;
        for (uint32_t q = 0; q < take; ++q)
          key |= (uint64_t)s_code[__ldg(p + q)] << (a.cb - a.b * (q + 1));
        if (a.S > 1) key |= (uint64_t)s << a.cb;
        a.keys[j] = key;
        a.vals[j] = off + irel + s;
      }
      pack_hist(s_hist, a.spec, key, valid, lane, a.top_only != 0);
    }
  }
  __syncthreads();
  for (uint32_t x = a.top_only ? (a.spec.P - 1) * RADIX + tid : tid; x < a.spec.P * RADIX;
       x += PACK_BLOCK) {
    const uint32_t v = (&s_hist[0][0])[x];
    if (v) atomicAdd(&a.hist[x], v);
  }
}

// The digit histograms of a single text's keys from the top digit's alone,
// when every digit covers g = 8 / b whole characters (b divides 8 and c0 * b
// is a multiple of 8): digit p of the key at position i is the g-character
// gram at i + q_p, q_p = (c0 * b - 8 (p + 1)) / b, with code 0 past the end
// of the text. Over i in [0, n) those grams are the grams at [q_p, n + q_p):
// the top digit's histogram (q = 0, grams at [0, n)) minus the grams at
// [0, q_p) plus q_p all-padding grams (digit 0). One block; q_p < 64.
__global__ void __launch_bounds__(RADIX) k_pack_hist_fixup(PackArgs a) {
  __shared__ uint8_t s_code[RADIX];
  __shared__ uint32_t s_gram[64];
  const uint32_t d = threadIdx.x;
  s_code[d] = a.code[d];
  const uint32_t P = a.spec.P, g = 8 / a.b;
  const uint32_t top = a.hist[(P - 1) * RADIX + d];
  __syncthreads();
  // grams at positions 0 .. 63 (all q_p are below c0 <= 64)
  if (d < 64) {
    uint32_t v = 0;
    for (uint32_t c = 0; c < g; ++c) {
      const uint64_t x = (uint64_t)d + c;
      v = (v << a.b) | (x < a.N ? s_code[a.text[x]] : 0u);
    }
    s_gram[d] = v;
  }
  __syncthreads();
  for (uint32_t p = 0; p + 1 < P; ++p) {
    const uint32_t qp = (a.cb - 8 * (p + 1)) / a.b;
    uint32_t below = 0;
    for (uint32_t x = 0; x < qp; ++x) below += s_gram[x] == d ? 1u : 0u;
    a.hist[p * RADIX + d] = top - below + (d == 0 ? qp : 0u);
  }
}

// The top digit's histogram alone (keys == NULL, top_only): the g-character
// gram (g = 8 / B) at every position p in [0, n), code 0 past the end, is
// the top digit of the key of p whatever index holds it, so no key is
// formed. Each thread takes 16 consecutive positions from one 16-byte load
// (plus the next g - 1 characters from its neighbour lane) and slides the
// gram through them in registers; per-warp counters in shared memory.
constexpr int GRAM_PER_THREAD = 16;
template <int B>
__global__ void __launch_bounds__(PACK_BLOCK) k_gram_hist(PackArgs a) {
  constexpr uint32_t G = 8 / B;
  __shared__ uint8_t s_code[RADIX];
  __shared__ uint32_t s_hist[PACK_BLOCK / 32][RADIX];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_code[tid] = a.code[tid];
  for (int w = 0; w < PACK_BLOCK / 32; ++w) s_hist[w][tid] = 0u;
  __syncthreads();
  const uint64_t n = a.N;
  const bool vec = (reinterpret_cast<uintptr_t>(a.text) & 15u) == 0;
  const uint64_t step = (uint64_t)gridDim.x * PACK_BLOCK * GRAM_PER_THREAD;
  // Whole warps iterate together (the shuffle below needs every lane).
  for (uint64_t p0 = ((uint64_t)blockIdx.x * PACK_BLOCK + (tid & ~31)) * GRAM_PER_THREAD; p0 < n;
       p0 += step) {
    const uint64_t p = p0 + (uint64_t)lane * GRAM_PER_THREAD;
    uint32_t w[6];  // characters p .. p + 23 (zero bytes past the end)
    if (vec && p + 16 <= n) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.text + p));
      w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t x = 0;
        for (int c = 3; c >= 0; --c) {
          const uint64_t i = p + 4 * q + c;
          x = (x << 8) | (i < n ? (uint32_t)__ldg(a.text + i) : 0u);
        }
        w[q] = x;
      }
    }
    w[4] = __shfl_down_sync(0xffffffffu, w[0], 1);
    w[5] = __shfl_down_sync(0xffffffffu, w[1], 1);
    if (lane == 31) {  // the next lane's characters are the next chunk's
#pragma unroll
      for (int q = 4; q < 6; ++q) {
        uint32_t x = 0;
        for (int c = 3; c >= 0; --c) {
          const uint64_t i = p + 4 * q + c;
          x = (x << 8) | (i < n ? (uint32_t)__ldg(a.text + i) : 0u);
        }
        w[q] = x;
      }
    }
    if (p >= n) continue;
    uint32_t gram = 0;
#pragma unroll
    for (uint32_t c = 0; c + 1 < G; ++c) gram = (gram << B) | s_code[(w[c >> 2] >> (8 * (c & 3))) & 0xFFu];
#pragma unroll
    for (uint32_t i = 0; i < GRAM_PER_THREAD; ++i) {
      const uint32_t c = i + G - 1;  // the gram's last character
      gram = ((gram << B) | s_code[(w[c >> 2] >> (8 * (c & 3))) & 0xFFu]) & 0xFFu;
      if (p + i < n) atomicAdd(&s_hist[warp][gram], 1u);
    }
  }
  __syncthreads();
  uint32_t v = 0;
  for (int w = 0; w < PACK_BLOCK / 32; ++w) v += s_hist[w][tid];
  if (v) atomicAdd(&a.hist[(a.spec.P - 1) * RADIX + tid], v);
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream) {
  if (a.N == 0) return cudaSuccess;
  if (!a.keys) {  // histograms only: the first radix pass forms the keys
    if (!a.top_only) return cudaErrorInvalidValue;
    const uint64_t span = (uint64_t)PACK_BLOCK * GRAM_PER_THREAD;
    const uint64_t want = ((uint64_t)a.N + span - 1) / span;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    switch (a.b) {
      case 1: k_gram_hist<1><<<grid, PACK_BLOCK, 0, stream>>>(a); break;
      case 2: k_gram_hist<2><<<grid, PACK_BLOCK, 0, stream>>>(a); break;
      case 4: k_gram_hist<4><<<grid, PACK_BLOCK, 0, stream>>>(a); break;
      case 8: k_gram_hist<8><<<grid, PACK_BLOCK, 0, stream>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pack_hist_fixup<<<1, RADIX, 0, stream>>>(a);
    return cudaGetLastError();
  }
  if (a.c0 >= PACK_SLIDE_MIN) {
    const uint64_t span = PACK_BLOCK * 16;
    k_pack<16><<<(unsigned)((a.N + span - 1) / span), PACK_BLOCK, 0, stream>>>(a);
  } else {
    const uint64_t span = PACK_BLOCK * 8;
    k_pack<8><<<(unsigned)((a.N + span - 1) / span), PACK_BLOCK, 0, stream>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !a.top_only) return e;
  k_pack_hist_fixup<<<1, RADIX, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace gbsa
