// DC3 (the skew algorithm of Karkkainen and Sanders, CPM 2003; the paper's
// Section 2.2, Algorithm 7, gives its distributed form): the suffix array
// by recursion on the difference cover D3 = {1, 2}.
//
// One level, on a text t of n integers in [1, K] padded with three zeros:
//   1. The sample positions i mod 3 != 0 (plus the dummy position n when
//      n mod 3 = 1, whose triple is all zeros) are sorted by their triples
//      (t[i], t[i+1], t[i+2]): one radix sort of a packed 64-bit key when
//      3 bits(K) <= 64, else two stable sorts (t[i+2], then (t[i], t[i+1])).
//   2. Names: a flag where a triple differs from its predecessor, inclusive
//      prefix sums (names 1-based), scattered to the recursion text R =
//      [names of positions 1 mod 3 | names of positions 2 mod 3].
//   3. If names repeat, the suffix array of R comes from the next level, and
//      rank12[SA_R[k]] = k + 1; otherwise SA_R[name - 1] = k directly.
//   4. The positions 0 mod 3, taken in the order of their right neighbour's
//      rank (from SA_R) and stably sorted by t[i], give S0 in suffix order.
//   5. S12 (from SA_R, the dummy dropped) and S0 are merged with the skew
//      comparison: for i = 1 mod 3 compare (t[i], rank(i+1)); for
//      i = 2 mod 3 compare (t[i], t[i+1], rank(i+2)).
// The merge is merge path: the elements of both inputs are first written out
// in order with their comparison data (character pair, neighbours' ranks);
// each block finds its output range's split by a binary search over those
// arrays, stages both input slices in shared memory, and each thread merges
// 4 outputs.
//
// Level 0 reads the 8-bit text as t[i] = T[i] + 1 (K = 256), so 0 is the
// end of text, smaller than every character (Section 2's order).
//
// Bound: HBM. Per level about 12 n bytes of sort input per pass (as the
// radix sort of the prefix-doubling path), a few random 4-byte reads per
// sample (names, ranks) and per merged element (its comparison data).
#include "dcx.cuh"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {
namespace {

__device__ __forceinline__ uint32_t sample_pos(uint64_t k, uint32_t n0) {
  return k < n0 ? (uint32_t)(3 * k + 1) : (uint32_t)(3 * (k - n0) + 2);
}

// Index of sample position p in the recursion text.
__device__ __forceinline__ uint32_t sample_idx(uint32_t p, uint32_t n0) {
  return p % 3 == 1 ? p / 3 : p / 3 + n0;
}

__global__ void k_dc3_text0(const uint8_t *__restrict__ T, uint64_t n, uint32_t *__restrict__ t) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + 3;
       i += (uint64_t)gridDim.x * blockDim.x)
    t[i] = i < n ? (uint32_t)T[i] + 1u : 0u;
}

// Sample keys. mode 0: the packed triple; mode 1: t[p+2] only.
__global__ void k_dc3_keys12(const uint32_t *__restrict__ t, uint32_t n02, uint32_t n0,
                             uint32_t b, int mode, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n02;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = sample_pos(k, n0);
    keys[k] = mode == 0 ? ((uint64_t)t[p] << (2 * b)) | ((uint64_t)t[p + 1] << b) | t[p + 2]
                        : (uint64_t)t[p + 2];
    vals[k] = p;
  }
}

// keys[k] from the position vals[k]: mode 0: (t[p] << b) | t[p+1]; mode 1: t[p].
__global__ void k_dc3_rekey(const uint32_t *__restrict__ t, uint32_t m, uint32_t b, int mode,
                            const uint32_t *__restrict__ vals, uint64_t *__restrict__ keys) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = vals[k];
    keys[k] = mode == 0 ? ((uint64_t)t[p] << b) | t[p + 1] : (uint64_t)t[p];
  }
}

// flags[k] = 1 where the triple of vals[k] differs from its predecessor's:
// the sorted keys hold the whole triple (two_stage = 0) or its first two
// names, the third then read from t.
__global__ void k_dc3_flags(const uint32_t *__restrict__ t, uint32_t m,
                            const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                            int two_stage, uint32_t *__restrict__ flags) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f = 1;
    if (k > 0) {
      f = keys[k] != keys[k - 1] ? 1u : 0u;
      if (!f && two_stage) f = t[vals[k] + 2] != t[vals[k - 1] + 2] ? 1u : 0u;
    }
    flags[k] = f;
  }
}

// ---- names, ranks, S0 --------------------------------------------------------

__global__ void k_dc3_scatter_names(uint32_t m, uint32_t n0, const uint32_t *__restrict__ vals,
                                    const uint32_t *__restrict__ names_sorted,
                                    uint32_t *__restrict__ R) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x)
    R[sample_idx(vals[k], n0)] = names_sorted[k];
}

// All names unique: SA_R[name - 1] = k.
__global__ void k_dc3_sa_from_names(uint32_t m, const uint32_t *__restrict__ R,
                                    uint32_t *__restrict__ sa12) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = R[k];
    if (r >= 1 && r <= m) sa12[r - 1] = (uint32_t)k;
  }
}

// After the recursion: rank12[SA_R[k]] = k + 1 (into R).
__global__ void k_dc3_ranks(uint32_t m, const uint32_t *__restrict__ sa12, uint32_t *__restrict__ R) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = sa12[k];
    if (s < m) R[s] = (uint32_t)k + 1u;
  }
}

__global__ void k_dc3_s0_flags(uint32_t m, uint32_t n0, const uint32_t *__restrict__ sa12,
                               uint32_t *__restrict__ flags) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x)
    flags[k] = sa12[k] < n0 ? 1u : 0u;
}

// S0 in the order of the right neighbour's rank: position 3 sa12[k].
__global__ void k_dc3_s0_scatter(uint32_t m, uint32_t n0, const uint32_t *__restrict__ sa12,
                                 const uint32_t *__restrict__ incl, uint32_t *__restrict__ s0) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = sa12[k];
    if (s < n0) {
      const uint32_t at = incl[k] - 1u;
      if (at < n0) s0[at] = 3u * s;
    }
  }
}

// ---- merge of S12 and S0 ---------------------------------------------------

constexpr int MG_ITEMS = 4;
constexpr int MG_TILE = DC_BLOCK * MG_ITEMS;

// A merge element: its position, t[p], t[p+1] and the ranks of the sample
// positions p+1 and p+2 (0 where the position is not a sample); padded to
// two 16-byte words, moved with vector loads and stores.
struct __align__(16) Elt {
  uint32_t pos, c0, c1, r1, r2, pad[3];
};
static_assert(sizeof(Elt) == 32, "Elt layout");
constexpr uint32_t ELT_WORDS = sizeof(Elt) / 16;

struct MergeArgs {
  const uint32_t *t;     // the level's text (padded with three zeros)
  const uint32_t *R;     // ranks of the sample positions (padded with three zeros)
  const uint32_t *sa12;  // suffix array of the recursion text
  const uint32_t *s0;    // positions 0 mod 3 in suffix order
  uint32_t n, n0, skip;  // skip: 1 if SA_R starts with the dummy position
  uint32_t na, nb;       // |S12| (dummy dropped), |S0|
  Elt *ea, *eb;          // the two inputs' elements, in order (built by k_dc3_elts)
  uint32_t *split;       // merge path: S12 elements before each block's first output
  uint32_t *sa;          // out: n positions
};

__device__ __forceinline__ Elt make_elt(const MergeArgs &a, uint32_t p) {
  Elt e{};
  e.pos = p;
  e.c0 = a.t[p];
  e.c1 = a.t[p + 1];
  e.r1 = (p + 1) % 3 ? a.R[sample_idx(p + 1, a.n0)] : 0u;
  e.r2 = (p + 2) % 3 ? a.R[sample_idx(p + 2, a.n0)] : 0u;
  return e;
}

// The elements of both inputs with their comparison data, in order: the
// gathers happen once, in parallel, and the merge reads contiguous arrays.
// One element per thread, staged in shared memory and written out in
// 16-byte words by consecutive threads.
__global__ void __launch_bounds__(DC_BLOCK) k_dc3_elts(MergeArgs a) {
  __shared__ Elt buf[DC_BLOCK];
  const uint64_t total = (uint64_t)a.na + a.nb;
  const uint64_t base = (uint64_t)blockIdx.x * DC_BLOCK;
  const uint64_t k = base + threadIdx.x;
  Elt e{};
  if (k < a.na) {
    const uint32_t s = a.sa12[a.skip + k];
    e = make_elt(a, s < a.n0 ? 3u * s + 1u : 3u * (s - a.n0) + 2u);
  } else if (k < total) {
    e = make_elt(a, a.s0[k - a.na]);
  }
  buf[threadIdx.x] = e;
  __syncthreads();
  const uint32_t cnt = (uint32_t)min((uint64_t)DC_BLOCK, total > base ? total - base : 0);
  const uint4 *b4 = reinterpret_cast<const uint4 *>(buf);
  for (uint32_t w = threadIdx.x; w < cnt * ELT_WORDS; w += DC_BLOCK) {
    const uint64_t x = base + w / ELT_WORDS;
    uint4 *dst = reinterpret_cast<uint4 *>(x < a.na ? a.ea + x : a.eb + (x - a.na));
    dst[w % ELT_WORDS] = b4[w];
  }
}

__device__ __forceinline__ Elt elt_a(const MergeArgs &a, uint32_t k) { return a.ea[k]; }
__device__ __forceinline__ Elt elt_b(const MergeArgs &a, uint32_t k) { return a.eb[k]; }

// Does the sample suffix x come before the suffix y = 0 mod 3?
__device__ __forceinline__ bool before(const Elt &x, const Elt &y) {
  if (x.pos % 3 == 1) return x.c0 < y.c0 || (x.c0 == y.c0 && x.r1 <= y.r1);
  if (x.c0 != y.c0) return x.c0 < y.c0;
  if (x.c1 != y.c1) return x.c1 < y.c1;
  return x.r2 <= y.r2;
}

// Number of S12 elements among the first d merged ones (merge path).
__device__ uint32_t merge_split(const MergeArgs &a, uint32_t d) {
  uint32_t lo = d > a.nb ? d - a.nb : 0u, hi = d < a.na ? d : a.na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (before(elt_a(a, mid), elt_b(a, d - 1 - mid)))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// split[b] = merge_split(b * tile) for b = 0 .. blocks (the last one the
// whole output), one thread per block boundary, so that the merge blocks
// start at once.
__global__ void __launch_bounds__(DC_BLOCK) k_dc3_splits(MergeArgs a, uint32_t blocks) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b > blocks) return;
  a.split[b] = merge_split(a, (uint32_t)min(b * MG_TILE, (uint64_t)a.n));
}

// dst[0, count) = src[0, count) by 16-byte words over the block's threads.
__device__ __forceinline__ void copy_elts(Elt *dst, const Elt *src, uint32_t count) {
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
  uint4 *d4 = reinterpret_cast<uint4 *>(dst);
  for (uint32_t x = threadIdx.x; x < count * ELT_WORDS; x += DC_BLOCK) d4[x] = s4[x];
}

__global__ void __launch_bounds__(DC_BLOCK) k_dc3_merge(MergeArgs a) {
  __shared__ Elt e[MG_TILE];  // S12 slice, then S0 slice
  __shared__ uint32_t out[MG_TILE];
  const uint32_t d0 = blockIdx.x * MG_TILE;
  const uint32_t d1 = min(d0 + (uint32_t)MG_TILE, a.n);
  const uint32_t a0 = a.split[blockIdx.x], a1 = a.split[blockIdx.x + 1];
  const uint32_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t na = a1 - a0, nb = b1 - b0, len = d1 - d0;
  if (a1 < a0 || a1 > a.na || na > len || nb > len) return;  // never taken unless unsorted
  copy_elts(e, a.ea + a0, na);
  copy_elts(e + na, a.eb + b0, nb);
  __syncthreads();
  const uint32_t dt = min((uint32_t)threadIdx.x * MG_ITEMS, len);
  uint32_t lo = dt > nb ? dt - nb : 0u, hi = dt < na ? dt : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (before(e[mid], e[na + dt - 1 - mid]))
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t i = lo, j = dt - lo;
#pragma unroll
  for (int k = 0; k < MG_ITEMS; ++k) {
    if (dt + k < len) {
      const bool take_a = j >= nb || (i < na && before(e[i], e[na + j]));
      out[dt + k] = take_a ? e[i++].pos : e[na + j++].pos;
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < len; x += DC_BLOCK) a.sa[d0 + x] = out[x];
}

}  // namespace
}  // namespace gbsa

namespace gbsa {
namespace {

struct Dc3 : DcxRun {
  uint32_t *trace = nullptr;  // level 0's recursion text, if wanted

  // Suffix array of t[0, n) (values in [1, K], t[n..n+2] = 0) into sa.
  sa_status level(const uint32_t *t, uint32_t n, uint64_t K, uint32_t *sa, int depth) {
    if (n == 0) return SA_OK;
    if (depth > 96) return SA_ERR_INTERNAL;
    const uint32_t n0 = (n + 2) / 3, n1 = (n + 1) / 3, n2 = n / 3, n02 = n0 + n2;
    const uint32_t b = bits_for_value(K);
    Scope sc(this);
    uint32_t *R, *sa12, *tmp, *sums;
    const uint64_t tiles = ((uint64_t)std::max(n02, n0) + SC_TILE - 1) / SC_TILE;
    sa_status s;
    if ((s = sc.get(&R, (uint64_t)n02 + 3)) != SA_OK) return s;
    if ((s = sc.get(&sa12, n02)) != SA_OK) return s;
    if ((s = sc.get(&tmp, std::max(n02, n0))) != SA_OK) return s;
    if ((s = sc.get(&sums, tiles)) != SA_OK) return s;

    // 1-2. Sort the samples by their triples and name them.
    uint32_t count = 0;
    {
      Scope s1(this);
      uint64_t *keys;
      uint32_t *vals;
      if ((s = s1.get(&keys, n02)) != SA_OK) return s;
      if ((s = s1.get(&vals, n02)) != SA_OK) return s;
      if (3 * b <= 64) {
        k_dc3_keys12<<<grid(n02), DC_BLOCK, 0, st>>>(t, n02, n0, b, 0, keys, vals);
        if ((s = ok()) != SA_OK || (s = sort(keys, vals, n02, 3 * b)) != SA_OK) return s;
      } else {
        k_dc3_keys12<<<grid(n02), DC_BLOCK, 0, st>>>(t, n02, n0, b, 1, keys, vals);
        if ((s = ok()) != SA_OK || (s = sort(keys, vals, n02, b)) != SA_OK) return s;
        k_dc3_rekey<<<grid(n02), DC_BLOCK, 0, st>>>(t, n02, b, 0, vals, keys);
        if ((s = ok()) != SA_OK || (s = sort(keys, vals, n02, 2 * b)) != SA_OK) return s;
      }
      k_dc3_flags<<<grid(n02), DC_BLOCK, 0, st>>>(t, n02, keys, vals, 3 * b > 64 ? 1 : 0, tmp);
      if ((s = ok()) != SA_OK || (s = scan(tmp, tmp, n02, sums)) != SA_OK) return s;
      if (cudaMemsetAsync(R, 0, ((size_t)n02 + 3) * 4, st) != cudaSuccess) return SA_ERR_CUDA;
      k_dc3_scatter_names<<<grid(n02), DC_BLOCK, 0, st>>>(n02, n0, vals, tmp, R);
      if ((s = ok()) != SA_OK) return s;
      if (cudaMemcpyAsync(&count, tmp + n02 - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return SA_ERR_CUDA;
      if (depth == 0 && trace &&
          cudaMemcpyAsync(trace, R, (size_t)n02 * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SA_ERR_CUDA;
    }
    if (count == 0 || count > n02) return SA_ERR_INTERNAL;

    // 3. Ranks of the samples.
    if (count < n02) {
      if ((s = level(R, n02, count, sa12, depth + 1)) != SA_OK) return s;
      k_dc3_ranks<<<grid(n02), DC_BLOCK, 0, st>>>(n02, sa12, R);
    } else {
      k_dc3_sa_from_names<<<grid(n02), DC_BLOCK, 0, st>>>(n02, R, sa12);
    }
    if ((s = ok()) != SA_OK) return s;

    // 4. S0: positions 0 mod 3 in the order of their right neighbour's rank,
    // then stably by their character.
    uint64_t *keys0;
    uint32_t *s0;
    if ((s = sc.get(&keys0, n0)) != SA_OK) return s;
    if ((s = sc.get(&s0, n0)) != SA_OK) return s;
    k_dc3_s0_flags<<<grid(n02), DC_BLOCK, 0, st>>>(n02, n0, sa12, tmp);
    if ((s = ok()) != SA_OK || (s = scan(tmp, tmp, n02, sums)) != SA_OK) return s;
    k_dc3_s0_scatter<<<grid(n02), DC_BLOCK, 0, st>>>(n02, n0, sa12, tmp, s0);
    k_dc3_rekey<<<grid(n0), DC_BLOCK, 0, st>>>(t, n0, b, 1, s0, keys0);
    if ((s = ok()) != SA_OK || (s = sort(keys0, s0, n0, b)) != SA_OK) return s;

    // 5. Merge.
    MergeArgs ma{};
    ma.t = t;
    ma.R = R;
    ma.sa12 = sa12;
    ma.s0 = s0;
    ma.n = n;
    ma.n0 = n0;
    ma.skip = n0 - n1;
    ma.na = n02 - ma.skip;
    ma.nb = n0;
    ma.sa = sa;
    const uint32_t blocks = (uint32_t)(((uint64_t)n + MG_TILE - 1) / MG_TILE);
    if ((s = sc.get(&ma.ea, ma.na)) != SA_OK || (s = sc.get(&ma.eb, ma.nb)) != SA_OK ||
        (s = sc.get(&ma.split, (uint64_t)blocks + 1)) != SA_OK)
      return s;
    k_dc3_elts<<<(unsigned)(((uint64_t)ma.na + ma.nb + DC_BLOCK - 1) / DC_BLOCK), DC_BLOCK, 0,
                 st>>>(ma);
    k_dc3_splits<<<(blocks + DC_BLOCK) / DC_BLOCK, DC_BLOCK, 0, st>>>(ma, blocks);
    k_dc3_merge<<<blocks, DC_BLOCK, 0, st>>>(ma);
    return ok();
  }
};

}  // namespace
}  // namespace gbsa

GBSA_API sa_status sa_build_dc3(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                                uint32_t *trace_names, gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  if (n == 0) return SA_OK;
  gbsa::Dc3 d;
  d.st = (cudaStream_t)stream;
  d.trace = trace_names;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SA_ERR_CUDA;
  sa_status s;
  {
    gbsa::Dc3::Scope sc(&d);
    uint32_t *t;
    if ((s = sc.get(&t, n + 3)) != SA_OK) return s;
    gbsa::k_dc3_text0<<<d.grid(n + 3), gbsa::DC_BLOCK, 0, d.st>>>(text, n, t);
    if ((s = gbsa::Dc3::ok()) != SA_OK) return s;
    s = d.level(t, (uint32_t)n, 256, sa_out, 0);
  }
  if (s == SA_OK && cudaStreamSynchronize(d.st) != cudaSuccess) return SA_ERR_CUDA;
  return s;
}
