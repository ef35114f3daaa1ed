// DC7 (Section 2.2, Algorithms 8-10): the suffix array by recursion on the
// difference cover D7 = {0, 1, 3} modulo 7, 3/7 of the positions.
//
// One level, on a text t of n integers in [1, K] padded with 16 zeros:
//   1. Samples: for each a in D7 the positions i = a mod 7 with i <= n, so
//      that every class ends with a window reaching past the text (such
//      windows are unique: their first zero sits at a different offset, and
//      only position n has an all-zero window). They are sorted by their
//      7-character windows: one radix sort of the packed window when
//      7 bits(K) <= 64, else stable sorts of chunks of it, last chunk first.
//   2. Names: a flag where a window differs from its predecessor, inclusive
//      sums (names 1-based), scattered to the recursion text R = T_0 T_1 T_3
//      (the names of the class-0 samples in text order, then class 1, then
//      class 3).
//   3. If names repeat, the next level gives SA_R and rank(R[k]) = its
//      position in SA_R + 1; otherwise the names are the ranks.
//   4. The seven classes S_j (positions i = j mod 7, i < n) in suffix order.
//      With l_j the smallest offset that reaches a sample ((j + l_j) mod 7 in
//      D7), S_j is the samples of class (j + l_j) mod 7 in rank order, moved
//      back by l_j, then stably sorted by the l_j characters in front of
//      them (nothing to sort for j in D7). The one position of class 4 or 5
//      whose sample would lie past n is put first; its own characters
//      (which reach the end of the text) place it.
//   5. Merge of the seven. Every element carries its position, its next six
//      characters and the ranks of the three samples among its next seven
//      positions (0 past n). Suffixes of classes a and b compare by their
//      first l(a, b) characters, then by the ranks at offset l(a, b), the
//      smallest offset that takes both into D7 (the lookup of the paper's
//      CompareDC7). A tree of merge-path merges: (S0 S1) (S2 S3) (S4 S5),
//      then (S01 S23) (S45 S6), then the two halves into SA.
//
// Level 0 reads the 8-bit text as t[i] = T[i] + 1 (K = 256), so 0 is the
// end of text, smaller than every character (Section 2's order).
//
// Bound: HBM. Per level: the sample sort (about 3/7 n keys, one to four
// sorts of 12 bytes per key and pass), the class lists and their short
// character sorts, and three merge passes over 40-byte elements.
#include "dcx.cuh"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {
namespace {

constexpr uint32_t D7_MASK = 0x0Bu;  // {0, 1, 3}
constexpr uint32_t PAD7 = 16;        // zeros after every level's text

__host__ __device__ __forceinline__ bool in_d7(uint32_t r) { return (D7_MASK >> r) & 1u; }

// Smallest offset l >= 0 with (a + l) mod 7 in D7.
__host__ __device__ __forceinline__ uint32_t l_first(uint32_t a) {
  uint32_t l = 0;
  while (!in_d7((a + l) % 7)) ++l;
  return l;
}

// Smallest offset l >= 0 taking both a and b into D7 (exists: D7 is a
// difference cover modulo 7).
__device__ __forceinline__ uint32_t l_pair(uint32_t a, uint32_t b) {
  uint32_t l = 0;
  while (l < 7 && !(in_d7((a + l) % 7) && in_d7((b + l) % 7))) ++l;
  return l;
}

// Which of the three samples an element's rank slot holds: D7 = {0, 1, 3}.
__device__ __forceinline__ uint32_t d7_slot(uint32_t r) { return r == 0 ? 0u : (r == 1 ? 1u : 2u); }

// Samples i = a mod 7 with i <= n.
__host__ __device__ __forceinline__ uint32_t class_samples(uint32_t n, uint32_t a) {
  return n >= a ? (n - a) / 7 + 1 : 0u;
}

// Positions i = j mod 7 with i < n.
__host__ __device__ __forceinline__ uint32_t class_size(uint32_t n, uint32_t j) {
  return n > j ? (n - 1 - j) / 7 + 1 : 0u;
}

__device__ __forceinline__ uint32_t dc7_sample_pos(uint32_t k, uint32_t c0, uint32_t c1) {
  return k < c0 ? 7u * k : (k < c0 + c1 ? 7u * (k - c0) + 1u : 7u * (k - c0 - c1) + 3u);
}

// Index of position p in the recursion text, or ~0 if p is not a sample.
__device__ __forceinline__ uint32_t dc7_sample_idx(uint64_t p, uint32_t n, uint32_t c0,
                                                   uint32_t c1) {
  if (p > n) return ~0u;
  const uint32_t a = (uint32_t)(p % 7), q = (uint32_t)(p / 7);
  if (a == 0) return q;
  if (a == 1) return c0 + q;
  if (a == 3) return c0 + c1 + q;
  return ~0u;
}

// t[p + lo .. p + hi) packed with b bits each, the first character highest.
__device__ __forceinline__ uint64_t pack_chars(const uint32_t *t, uint64_t p, uint32_t lo,
                                               uint32_t hi, uint32_t b) {
  uint64_t key = 0;
  for (uint32_t c = lo; c < hi; ++c) key = (key << b) | t[p + c];
  return key;
}

__global__ void k_dc7_text0(const uint8_t *__restrict__ T, uint64_t n, uint32_t *__restrict__ t) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + PAD7;
       i += (uint64_t)gridDim.x * blockDim.x)
    t[i] = i < n ? (uint32_t)T[i] + 1u : 0u;
}

// Sample k of the recursion text: its window chunk [lo, hi) and position.
__global__ void k_dc7_keys(const uint32_t *__restrict__ t, uint32_t m, uint32_t c0, uint32_t c1,
                           uint32_t b, uint32_t lo, uint32_t hi, uint64_t *__restrict__ keys,
                           uint32_t *__restrict__ vals) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = dc7_sample_pos((uint32_t)k, c0, c1);
    keys[k] = pack_chars(t, p, lo, hi, b);
    vals[k] = p;
  }
}

// keys[k] = chunk [lo, hi) of the characters at position vals[k].
__global__ void k_dc7_rekey(const uint32_t *__restrict__ t, uint32_t m, uint32_t b, uint32_t lo,
                            uint32_t hi, const uint32_t *__restrict__ vals,
                            uint64_t *__restrict__ keys) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x)
    keys[k] = pack_chars(t, vals[k], lo, hi, b);
}

// flags[k] = 1 where the window of vals[k] differs from its predecessor's:
// from the sorted keys when they hold whole windows (keys != NULL), else
// from the text.
__global__ void k_dc7_flags(const uint32_t *__restrict__ t, uint32_t m,
                            const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                            uint32_t *__restrict__ flags) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f = 1;
    if (k > 0) {
      if (keys) {
        f = keys[k] != keys[k - 1] ? 1u : 0u;
      } else {
        const uint32_t p = vals[k], q = vals[k - 1];
        f = 0;
        for (int c = 0; c < 7; ++c) f |= t[p + c] != t[q + c] ? 1u : 0u;
      }
    }
    flags[k] = f;
  }
}

__global__ void k_dc7_scatter_names(uint32_t m, uint32_t n, uint32_t c0, uint32_t c1,
                                    const uint32_t *__restrict__ vals,
                                    const uint32_t *__restrict__ names, uint32_t *__restrict__ R) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = dc7_sample_idx(vals[k], n, c0, c1);
    if (x < m) R[x] = names[k];
  }
}

// All names unique: SA_R[name - 1] = k.
__global__ void k_dc7_sa_from_names(uint32_t m, const uint32_t *__restrict__ R,
                                    uint32_t *__restrict__ saR) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = R[k];
    if (r >= 1 && r <= m) saR[r - 1] = (uint32_t)k;
  }
}

// After the recursion: rank(SA_R[k]) = k + 1 (into R).
__global__ void k_dc7_ranks(uint32_t m, const uint32_t *__restrict__ saR, uint32_t *__restrict__ R) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = saR[k];
    if (s < m) R[s] = (uint32_t)k + 1u;
  }
}

// ---- merge -------------------------------------------------------------------

// A merge element: its position, the ranks of the samples at the offsets
// l with (pos + l) mod 7 = 0, 1, 3 (0 past n), and its next six characters.
// Padded to three 16-byte words, moved with vector loads and stores.
struct __align__(16) Elt7 {
  uint32_t pos;
  uint32_t r[3];
  uint32_t c[6];
  uint32_t pad[2];
};
static_assert(sizeof(Elt7) == 48, "Elt7 layout");
constexpr uint32_t ELT7_WORDS = sizeof(Elt7) / 16;

// dst[0, count) = src[0, count) by 16-byte words, the block's threads
// striding through them.
__device__ __forceinline__ void copy_elts(Elt7 *dst, const Elt7 *src, uint32_t count) {
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
  uint4 *d4 = reinterpret_cast<uint4 *>(dst);
  for (uint32_t x = threadIdx.x; x < count * ELT7_WORDS; x += blockDim.x) d4[x] = s4[x];
}

// One element per thread, staged in shared memory and written out in
// 16-byte words by consecutive threads.
__global__ void __launch_bounds__(DC_BLOCK) k_dc7_elts(const uint32_t *__restrict__ t,
                                                       const uint32_t *__restrict__ R,
                                                       uint32_t n, uint32_t c0, uint32_t c1,
                                                       const uint32_t *__restrict__ cls,
                                                       Elt7 *__restrict__ E) {
  __shared__ Elt7 buf[DC_BLOCK];
  const uint32_t m = c0 + c1 + class_samples(n, 3);
  const uint64_t base = (uint64_t)blockIdx.x * DC_BLOCK;
  const uint64_t x = base + threadIdx.x;
  Elt7 e{};
  if (x < n) {
    const uint32_t i = cls[x];
    e.pos = i;
    if (i < n) {  // else a class list is incomplete (never taken)
      const uint32_t j = i % 7;
#pragma unroll
      for (uint32_t d = 0; d < 3; ++d) {
        const uint32_t target = d == 0 ? 0u : (d == 1 ? 1u : 3u);
        const uint64_t p = (uint64_t)i + (target + 7 - j) % 7;
        const uint32_t k = dc7_sample_idx(p, n, c0, c1);
        e.r[d] = k < m ? R[k] : 0u;
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) e.c[c] = t[(uint64_t)i + c];
    }
  }
  buf[threadIdx.x] = e;
  __syncthreads();
  const uint32_t cnt = (uint32_t)min((uint64_t)DC_BLOCK, n > base ? n - base : 0);
  const uint4 *b4 = reinterpret_cast<const uint4 *>(buf);
  uint4 *o4 = reinterpret_cast<uint4 *>(E + base);
  for (uint32_t w = threadIdx.x; w < cnt * ELT7_WORDS; w += DC_BLOCK) o4[w] = b4[w];
}

// The lookup table of CompareDC7 for classes a, b: l = l(a, b) in bits
// 0-2, the rank slot of a at offset l in bits 3-4, that of b in bits 5-6.
__device__ __forceinline__ uint32_t cmp7_entry(uint32_t a, uint32_t b) {
  const uint32_t l = l_pair(a, b);
  return l | (d7_slot((a + l) % 7) << 3) | (d7_slot((b + l) % 7) << 5);
}

// Does suffix x come before suffix y (the comparison of CompareDC7)? lut
// holds cmp7_entry for the 49 class pairs.
__device__ __forceinline__ bool less7(const Elt7 &x, const Elt7 &y, const uint8_t *lut) {
  const uint32_t e = lut[(x.pos % 7) * 7 + y.pos % 7];
  const uint32_t l = e & 7u;
  for (uint32_t k = 0; k < l; ++k)
    if (x.c[k] != y.c[k]) return x.c[k] < y.c[k];
  return x.r[(e >> 3) & 3u] < y.r[(e >> 5) & 3u];
}

constexpr int MG7_ITEMS = 2;
constexpr int MG7_TILE = DC_BLOCK * MG7_ITEMS;

__device__ __forceinline__ void load_lut(uint8_t *lut) {
  for (uint32_t x = threadIdx.x; x < 49; x += blockDim.x) lut[x] = (uint8_t)cmp7_entry(x / 7, x % 7);
}

// Merge path: split[b] = elements of A among the first min(b * tile, na + nb)
// merged ones, for b = 0 .. blocks; one thread per block boundary, so that
// the merge blocks start at once.
__global__ void __launch_bounds__(DC_BLOCK) k_dc7_splits(const Elt7 *ea, uint32_t na,
                                                         const Elt7 *eb, uint32_t nb,
                                                         uint32_t blocks, uint32_t *split) {
  __shared__ uint8_t lut[49];
  load_lut(lut);
  __syncthreads();
  const uint64_t bidx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bidx > blocks) return;
  const uint32_t d = (uint32_t)min(bidx * MG7_TILE, (uint64_t)na + nb);
  uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (less7(ea[mid], eb[d - 1 - mid], lut))
      lo = mid + 1;
    else
      hi = mid;
  }
  split[bidx] = lo;
}

// out_e (POS = false) or out_pos (POS = true) = merge of A and B, block b
// covering outputs [b * tile, (b + 1) * tile) from the precomputed splits.
template <bool POS>
__global__ void __launch_bounds__(DC_BLOCK) k_dc7_merge(const Elt7 *ea, uint32_t na,
                                                        const Elt7 *eb, uint32_t nb,
                                                        const uint32_t *__restrict__ split,
                                                        Elt7 *out_e, uint32_t *out_pos) {
  __shared__ Elt7 e[MG7_TILE];  // A slice, then B slice
  __shared__ uint16_t pick[MG7_TILE];
  __shared__ uint8_t lut[49];
  load_lut(lut);
  const uint32_t total = na + nb;
  const uint32_t d0 = blockIdx.x * MG7_TILE;
  const uint32_t d1 = min(d0 + (uint32_t)MG7_TILE, total);
  const uint32_t a0 = split[blockIdx.x], a1 = split[blockIdx.x + 1];
  const uint32_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t sa = a1 - a0, sb = b1 - b0, len = d1 - d0;
  if (a1 < a0 || sa > len || sb > len || a1 > na) return;  // never taken unless unsorted
  copy_elts(e, ea + a0, sa);
  copy_elts(e + sa, eb + b0, sb);
  __syncthreads();
  const uint32_t dt = min((uint32_t)threadIdx.x * MG7_ITEMS, len);
  uint32_t lo = dt > sb ? dt - sb : 0u, hi = dt < sa ? dt : sa;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (less7(e[mid], e[sa + dt - 1 - mid], lut))
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t i = lo, j = dt - lo;
#pragma unroll
  for (int k = 0; k < MG7_ITEMS; ++k) {
    if (dt + k < len) {
      const bool take_a = j >= sb || (i < sa && less7(e[i], e[sa + j], lut));
      pick[dt + k] = (uint16_t)(take_a ? i++ : sa + j++);
    }
  }
  __syncthreads();
  if (POS) {
    for (uint32_t x = threadIdx.x; x < len; x += DC_BLOCK) out_pos[d0 + x] = e[pick[x]].pos;
  } else {
    uint4 *o4 = reinterpret_cast<uint4 *>(out_e + d0);
    const uint4 *e4 = reinterpret_cast<const uint4 *>(e);
    for (uint32_t x = threadIdx.x; x < len * ELT7_WORDS; x += DC_BLOCK)
      o4[x] = e4[pick[x / ELT7_WORDS] * ELT7_WORDS + x % ELT7_WORDS];
  }
}

// ---- class lists -------------------------------------------------------------

// One word written by the device (a class's first entry).
__global__ void k_dc7_set(uint32_t *p, uint32_t v) { *p = v; }

// Class j from the ranked samples: flags[r] = 1 where the sample of rank r
// is of class s = (j + l) mod 7 and p - l is a position of the text.
__global__ void k_dc7_class_flags(uint32_t m, const uint32_t *__restrict__ saR, uint32_t n,
                                  uint32_t c0, uint32_t c1, uint32_t s, uint32_t l,
                                  uint32_t *__restrict__ flags) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = saR[r];
    uint32_t f = 0;
    if (k < m) {
      const uint32_t p = dc7_sample_pos(k, c0, c1);
      f = (p % 7 == s && p >= l && p - l < n) ? 1u : 0u;
    }
    flags[r] = f;
  }
}

// After the inclusive scan of those flags (incl): the flagged samples, moved
// back by l, to out[front + incl[r] - 1].
__global__ void k_dc7_class_scatter(uint32_t m, const uint32_t *__restrict__ saR, uint32_t c0,
                                    uint32_t c1, uint32_t l, const uint32_t *__restrict__ incl,
                                    uint32_t front, uint32_t cnt, uint32_t *__restrict__ out) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t before = r ? incl[r - 1] : 0u;
    if (incl[r] == before) continue;
    const uint32_t at = front + before;
    const uint32_t k = saR[r];
    if (at < cnt && k < m) out[at] = dc7_sample_pos(k, c0, c1) - l;
  }
}

}  // namespace
}  // namespace gbsa

namespace gbsa {
namespace {

struct Dc7 : DcxRun {
  uint32_t *trace = nullptr;  // level 0's recursion text, if wanted

  // Stable sort of (keys, vals)[0, m) by the characters t[v + lo0 .. v + hi0)
  // of each value v: one radix sort per chunk of at most 64 bits, the last
  // chunk first. With first_built the caller has put the last chunk's keys
  // in keys already.
  sa_status sort_chars(const uint32_t *t, uint64_t *keys, uint32_t *vals, uint32_t m, uint32_t b,
                       uint32_t lo0, uint32_t hi0, bool first_built) {
    const uint32_t per = std::max<uint32_t>(1, 64 / b);
    uint32_t hi = hi0;
    bool built = first_built;
    sa_status s;
    while (hi > lo0) {
      const uint32_t lo = hi - std::min(per, hi - lo0);
      if (!built) {
        k_dc7_rekey<<<grid(m), DC_BLOCK, 0, st>>>(t, m, b, lo, hi, vals, keys);
        if ((s = ok()) != SA_OK) return s;
      }
      built = false;
      if ((s = sort(keys, vals, m, (hi - lo) * b)) != SA_OK) return s;
      hi = lo;
    }
    return SA_OK;
  }

  // split: at least total / tile + 2 words of scratch.
  sa_status merge(const Elt7 *a, uint32_t na, const Elt7 *b, uint32_t nb, Elt7 *out_e,
                  uint32_t *out_pos, uint32_t *split) {
    const uint64_t total = (uint64_t)na + nb;
    if (total == 0) return SA_OK;
    const unsigned blocks = (unsigned)((total + MG7_TILE - 1) / MG7_TILE);
    k_dc7_splits<<<(blocks + DC_BLOCK) / DC_BLOCK, DC_BLOCK, 0, st>>>(a, na, b, nb, blocks,
                                                                     split);
    if (out_pos)
      k_dc7_merge<true><<<blocks, DC_BLOCK, 0, st>>>(a, na, b, nb, split, nullptr, out_pos);
    else
      k_dc7_merge<false><<<blocks, DC_BLOCK, 0, st>>>(a, na, b, nb, split, out_e, nullptr);
    return ok();
  }

  // Suffix array of t[0, n) (values in [1, K], t[n .. n + 15] = 0) into sa.
  sa_status level(const uint32_t *t, uint32_t n, uint64_t K, uint32_t *sa, int depth) {
    if (n == 0) return SA_OK;
    if (depth > 96) return SA_ERR_INTERNAL;
    const uint32_t c0 = class_samples(n, 0), c1 = class_samples(n, 1), c3 = class_samples(n, 3);
    const uint32_t m = c0 + c1 + c3;
    const uint32_t b = bits_for_value(K);
    Scope sc(this);
    uint32_t *R, *saR, *tmp, *sums, *gotd;
    const uint64_t tiles = ((uint64_t)m + SC_TILE - 1) / SC_TILE;
    sa_status s;
    if ((s = sc.get(&R, (uint64_t)m + PAD7)) != SA_OK) return s;
    if ((s = sc.get(&saR, m)) != SA_OK) return s;
    if ((s = sc.get(&tmp, m)) != SA_OK) return s;
    if ((s = sc.get(&sums, tiles)) != SA_OK) return s;
    if ((s = sc.get(&gotd, 8)) != SA_OK) return s;

    // 1-2. Sort the samples by their windows and name them.
    uint32_t count = 0;
    {
      Scope s1(this);
      uint64_t *keys;
      uint32_t *vals;
      if ((s = s1.get(&keys, m)) != SA_OK) return s;
      if ((s = s1.get(&vals, m)) != SA_OK) return s;
      const uint32_t per = std::max<uint32_t>(1, 64 / b);
      const uint32_t lo = 7 - std::min<uint32_t>(per, 7);
      k_dc7_keys<<<grid(m), DC_BLOCK, 0, st>>>(t, m, c0, c1, b, lo, 7, keys, vals);
      if ((s = ok()) != SA_OK) return s;
      if ((s = sort_chars(t, keys, vals, m, b, 0, 7, true)) != SA_OK) return s;
      k_dc7_flags<<<grid(m), DC_BLOCK, 0, st>>>(t, m, per >= 7 ? keys : nullptr, vals, tmp);
      if ((s = ok()) != SA_OK || (s = scan(tmp, tmp, m, sums)) != SA_OK) return s;
      if (cudaMemsetAsync(R, 0, ((size_t)m + PAD7) * 4, st) != cudaSuccess) return SA_ERR_CUDA;
      k_dc7_scatter_names<<<grid(m), DC_BLOCK, 0, st>>>(m, n, c0, c1, vals, tmp, R);
      if ((s = ok()) != SA_OK) return s;
      if (cudaMemcpyAsync(&count, tmp + m - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return SA_ERR_CUDA;
      if (depth == 0 && trace &&
          cudaMemcpyAsync(trace, R, (size_t)m * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SA_ERR_CUDA;
    }
    if (count == 0 || count > m) return SA_ERR_INTERNAL;

    // 3. Ranks of the samples (R) and the samples in rank order (saR).
    if (count < m) {
      if ((s = level(R, m, count, saR, depth + 1)) != SA_OK) return s;
      k_dc7_ranks<<<grid(m), DC_BLOCK, 0, st>>>(m, saR, R);
    } else {
      k_dc7_sa_from_names<<<grid(m), DC_BLOCK, 0, st>>>(m, R, saR);
    }
    if ((s = ok()) != SA_OK) return s;

    // 4. The seven classes in suffix order, one after the other in cls.
    uint32_t size[7], off[8], front[7];
    off[0] = 0;
    for (uint32_t j = 0; j < 7; ++j) {
      size[j] = class_size(n, j);
      off[j + 1] = off[j] + size[j];
      // The class's last position, if the sample it would use lies past n.
      front[j] = size[j] && j + 7 * (size[j] - 1) + l_first(j) > n ? 1u : 0u;
    }
    if (off[7] != n) return SA_ERR_INTERNAL;
    uint32_t *cls;
    uint64_t *ckeys;
    if ((s = sc.get(&cls, n)) != SA_OK) return s;
    if ((s = sc.get(&ckeys, size[0])) != SA_OK) return s;  // class 0 is the largest
    if (cudaMemsetAsync(gotd, 0, 8 * 4, st) != cudaSuccess) return SA_ERR_CUDA;
    for (uint32_t j = 0; j < 7; ++j) {
      if (size[j] == 0) continue;
      const uint32_t l = l_first(j), cs = (j + l) % 7;
      uint32_t *out = cls + off[j];
      if (front[j]) k_dc7_set<<<1, 1, 0, st>>>(out, j + 7 * (size[j] - 1));
      k_dc7_class_flags<<<grid(m), DC_BLOCK, 0, st>>>(m, saR, n, c0, c1, cs, l, tmp);
      if ((s = ok()) != SA_OK || (s = scan(tmp, tmp, m, sums)) != SA_OK) return s;
      k_dc7_class_scatter<<<grid(m), DC_BLOCK, 0, st>>>(m, saR, c0, c1, l, tmp, front[j],
                                                        size[j], out);
      if ((s = ok()) != SA_OK) return s;
      if (cudaMemcpyAsync(gotd + j, tmp + m - 1, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SA_ERR_CUDA;
      if (l > 0 && (s = sort_chars(t, ckeys, out, size[j], b, 0, l, false)) != SA_OK) return s;
    }
    uint32_t got[8];
    if (cudaMemcpyAsync(got, gotd, 8 * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SA_ERR_CUDA;
    for (uint32_t j = 0; j < 7; ++j)
      if (size[j] && got[j] + front[j] != size[j]) return SA_ERR_INTERNAL;

    // 5. Elements and the merge tree.
    Elt7 *E, *E2;
    uint32_t *sp;
    if ((s = sc.get(&E, n)) != SA_OK || (s = sc.get(&E2, n)) != SA_OK) return s;
    if ((s = sc.get(&sp, (uint64_t)n / MG7_TILE + 2)) != SA_OK) return s;
    k_dc7_elts<<<(unsigned)(((uint64_t)n + DC_BLOCK - 1) / DC_BLOCK), DC_BLOCK, 0, st>>>(
        t, R, n, c0, c1, cls, E);
    if ((s = ok()) != SA_OK) return s;
    if ((s = merge(E + off[0], size[0], E + off[1], size[1], E2 + off[0], nullptr, sp)) != SA_OK ||
        (s = merge(E + off[2], size[2], E + off[3], size[3], E2 + off[2], nullptr, sp)) != SA_OK ||
        (s = merge(E + off[4], size[4], E + off[5], size[5], E2 + off[4], nullptr, sp)) != SA_OK)
      return s;
    if (size[6] && cudaMemcpyAsync(E2 + off[6], E + off[6], (size_t)size[6] * sizeof(Elt7),
                                   cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SA_ERR_CUDA;
    if ((s = merge(E2 + off[0], off[2] - off[0], E2 + off[2], off[4] - off[2], E + off[0],
                   nullptr, sp)) != SA_OK ||
        (s = merge(E2 + off[4], off[6] - off[4], E2 + off[6], off[7] - off[6], E + off[4],
                   nullptr, sp)) != SA_OK)
      return s;
    return merge(E, off[4], E + off[4], off[7] - off[4], nullptr, sa, sp);
  }
};

}  // namespace
}  // namespace gbsa

GBSA_API sa_status sa_build_dc7(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                                uint32_t *trace_names, gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  if (n == 0) return SA_OK;
  gbsa::Dc7 d;
  d.st = (cudaStream_t)stream;
  d.trace = trace_names;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SA_ERR_CUDA;
  sa_status s;
  {
    gbsa::Dc7::Scope sc(&d);
    uint32_t *t;
    if ((s = sc.get(&t, n + gbsa::PAD7)) != SA_OK) return s;
    gbsa::k_dc7_text0<<<d.grid(n + gbsa::PAD7), gbsa::DC_BLOCK, 0, d.st>>>(text, n, t);
    if ((s = gbsa::Dc7::ok()) != SA_OK) return s;
    s = d.level(t, (uint32_t)n, 256, sa_out, 0);
  }
  if (s == SA_OK && cudaStreamSynchronize(d.st) != cudaSuccess) return SA_ERR_CUDA;
  return s;
}
