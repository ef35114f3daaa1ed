// LCP array from the suffix array: a direct consumer of SA named as future
// work at the end of the paper (Section 3). lcp[0] = 0 and, for j >= 1,
// lcp[j] is the longest common prefix of the suffixes SA[j-1] and SA[j]
// (Section 2's suffix order).
//
// Permuted form of Kasai et al.'s linear-time algorithm (Kasai, Lee,
// Arimura, Arikawa, Park, CPM 2001; permuted LCP of Karkkainen, Manzini and
// Puglisi, CPM 2009): with Phi[SA[j]] = SA[j-1], the permuted array
// PLCP[i] = lcp(i, Phi[i]) satisfies PLCP[i] >= PLCP[i-1] - 1, so a scan in
// text order extends each value from the previous one minus one.
//
//   k_lcp_phi:    Phi[SA[j]] = SA[j-1] (j >= 1); Phi[SA[0]] = n (none).
//                 From 2^20 characters on, the writes are first grouped by
//                 position (k_lcp_entries builds (Phi value, SA[j]) pairs,
//                 the position bucketing of the ISA writes partitions them
//                 into 256 position ranges, k_lcp_apply writes them range
//                 by range), so the Phi being written stays in L2 instead of
//                 each 4-byte write costing a sector read and write.
//   k_lcp_plcp:   the text is cut into chunks of LCP_CHUNK positions, one
//                 thread per chunk scanning it in order; a chunk's first
//                 value is extended from 0, every later one from the
//                 previous minus one. Characters are compared 8 at a time
//                 (two funnel-shifted aligned 32-bit windows per suffix).
//   k_lcp_gather: lcp[j] = PLCP[SA[j]].
// Work: 2n character comparisons plus, per chunk, the first value's LCP.
// Bound: HBM / latency. Algorithmic bytes per position: 8 (Phi: read SA,
// random write) + 10 (PLCP: read Phi, write PLCP, one sequential and one
// random text byte) + 12 (gather: read SA, random read of PLCP, write).
#include <algorithm>

#include "../../include/gbsa.h"
#include "launch.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {

constexpr uint32_t LCP_CHUNK = 256;

__global__ void __launch_bounds__(256) k_lcp_phi(const uint32_t *__restrict__ sa, uint64_t n,
                                                 uint32_t *__restrict__ phi) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const uint32_t s = sa[j];
    if (s < n) phi[s] = j ? sa[j - 1] : (uint32_t)n;
  }
}

// Position-bucketed Phi writes: e[j] = (Phi value << 32) | SA[j].
__global__ void __launch_bounds__(256) k_lcp_entries(const uint32_t *__restrict__ sa, uint64_t n,
                                                     uint64_t *__restrict__ e) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
    e[j] = ((uint64_t)(j ? sa[j - 1] : (uint32_t)n) << 32) | sa[j];
}

__global__ void k_lcp_set_count(uint32_t *count, uint32_t n) { *count = n; }

// Phi[low] = high for the bucketed entries; blocks take consecutive chunks
// of LCP_APPLY entries in launch order, so the positions written stay in a
// narrow window.
constexpr int LCP_APPLY_ITEMS = 8;
constexpr uint32_t LCP_APPLY = 256 * LCP_APPLY_ITEMS;

__global__ void __launch_bounds__(256) k_lcp_apply(const uint64_t *__restrict__ e, uint64_t n,
                                                   uint32_t *__restrict__ phi) {
  const uint64_t c0 = (uint64_t)blockIdx.x * LCP_APPLY;
  uint64_t u[LCP_APPLY_ITEMS];
#pragma unroll
  for (int k = 0; k < LCP_APPLY_ITEMS; ++k) {
    const uint64_t x = c0 + (uint64_t)k * 256 + threadIdx.x;
    u[k] = x < n ? e[x] : ~0ull;
  }
#pragma unroll
  for (int k = 0; k < LCP_APPLY_ITEMS; ++k) {
    const uint32_t s = (uint32_t)u[k];
    if (u[k] != ~0ull && s < n) phi[s] = (uint32_t)(u[k] >> 32);
  }
}

// Bytes [x, x + 8) of T as two little-endian words; T 4-byte aligned and
// x + 12 <= n (the three aligned words read lie inside the text).
__device__ __forceinline__ void load8(const uint8_t *T, uint64_t x, uint32_t &lo, uint32_t &hi) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(T + (x & ~3ull));
  const uint32_t sh = (uint32_t)(x & 3u) * 8u;
  const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
  lo = __funnelshift_r(w0, w1, sh);
  hi = __funnelshift_r(w1, w2, sh);
}

// lcp(i, p) given that the first h characters are known equal.
__device__ __forceinline__ uint64_t lcp_extend(const uint8_t *T, uint64_t n, uint64_t i,
                                               uint64_t p, uint64_t h, bool words) {
  const uint64_t lim = n - (i > p ? i : p);  // the shorter suffix's length
  while (h < lim) {
    if (words && h + 12 <= lim) {
      uint32_t a0, a1, b0, b1;
      load8(T, i + h, a0, a1);
      load8(T, p + h, b0, b1);
      const uint32_t x0 = a0 ^ b0, x1 = a1 ^ b1;
      if (x0) return h + (uint32_t)(__ffs(x0) - 1) / 8u;
      if (x1) return h + 4 + (uint32_t)(__ffs(x1) - 1) / 8u;
      h += 8;
    } else {
      if (T[i + h] != T[p + h]) return h;
      ++h;
    }
  }
  return h;
}

__global__ void __launch_bounds__(256) k_lcp_plcp(const uint8_t *__restrict__ T, uint64_t n,
                                                  const uint32_t *__restrict__ phi,
                                                  uint32_t *__restrict__ plcp) {
  const bool words = (((uintptr_t)T) & 3u) == 0;
  const uint64_t chunks = (n + LCP_CHUNK - 1) / LCP_CHUNK;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += stride) {
    const uint64_t i0 = c * LCP_CHUNK, i1 = min(n, i0 + LCP_CHUNK);
    uint64_t h = 0;
    for (uint64_t i = i0; i < i1; ++i) {
      const uint32_t p = phi[i];
      if (p >= n) {  // the smallest suffix (or not a suffix array): nothing before it
        h = 0;
        plcp[i] = 0;
        continue;
      }
      h = lcp_extend(T, n, i, p, h, words);
      plcp[i] = (uint32_t)h;
      if (h) --h;
    }
  }
}

__global__ void __launch_bounds__(256) k_lcp_gather(const uint32_t *__restrict__ sa, uint64_t n,
                                                    const uint32_t *__restrict__ plcp,
                                                    uint32_t *__restrict__ lcp) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const uint32_t s = sa[j];
    lcp[j] = (j == 0 || s >= n) ? 0u : plcp[s];
  }
}

}  // namespace gbsa

namespace {

int lcp_sm_count() { return gbsa::device_sm_count(); }

unsigned grid_for(uint64_t units, int per_sm) {
  const uint64_t want = (units + 255) / 256, cap = (uint64_t)lcp_sm_count() * per_sm;
  return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr uint64_t LCP_BUCKET_MIN = 1ull << 20;  // bucket the Phi writes from this size on

// Phi (4n) | entries (8n; PLCP reuses its first half) | bucketed entries
// (8n) | bucket counts | the entry count.
struct LcpLayout {
  size_t phi, ent, ent2, counts, count, total;
};

LcpLayout lcp_layout(uint64_t n) {
  LcpLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o += align256(b);
    return r;
  };
  L.phi = take((size_t)n * 4);
  L.ent = take((size_t)n * 8);
  L.ent2 = take((size_t)n * 8);
  L.counts = take((size_t)gbsa::BUCKET_BLOCKS_MAX * 256 * 4);
  L.count = take(4);
  L.total = o;
  return L;
}

}  // namespace

GBSA_API size_t sa_lcp_workspace_bytes(uint64_t n) { return lcp_layout(n).total; }

GBSA_API sa_status sa_lcp(const uint8_t *text, uint64_t n, const uint32_t *sa, uint32_t *lcp_out,
                          void *workspace, size_t ws_bytes, gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa || !lcp_out)) return SA_ERR_INVALID_ARG;
  if (n == 0) return SA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = sa_lcp_workspace_bytes(n);
  void *ws = workspace;
  if (ws) {
    if (ws_bytes < need || ((uintptr_t)ws & 255)) return SA_ERR_INVALID_ARG;
  } else if (cudaMallocAsync(&ws, need, st) != cudaSuccess) {
    return SA_ERR_OOM;
  }
  const LcpLayout L = lcp_layout(n);
  uint8_t *base = static_cast<uint8_t *>(ws);
  uint32_t *phi = reinterpret_cast<uint32_t *>(base + L.phi);
  uint32_t *plcp = reinterpret_cast<uint32_t *>(base + L.ent);
  const uint64_t chunks = (n + gbsa::LCP_CHUNK - 1) / gbsa::LCP_CHUNK;
  cudaError_t e = cudaSuccess;
  if (n >= LCP_BUCKET_MIN) {
    uint64_t *ent = reinterpret_cast<uint64_t *>(base + L.ent);
    uint32_t *count = reinterpret_cast<uint32_t *>(base + L.count);
    gbsa::k_lcp_entries<<<grid_for(n, 8), 256, 0, st>>>(sa, n, ent);
    gbsa::k_lcp_set_count<<<1, 1, 0, st>>>(count, (uint32_t)n);
    gbsa::BucketArgs ba{};
    ba.in = ent;
    ba.lo = nullptr;
    ba.count = count;
    ba.max_count = (uint32_t)n;
    uint32_t bits = 0;
    while (bits < 64 && (n >> bits)) ++bits;
    ba.shift = bits > 8 ? bits - 8 : 0;
    ba.blocks = std::min<uint32_t>(gbsa::BUCKET_BLOCKS_MAX, 4u * (uint32_t)lcp_sm_count());
    ba.counts = reinterpret_cast<uint32_t *>(base + L.counts);
    ba.out = reinterpret_cast<uint64_t *>(base + L.ent2);
    if ((e = gbsa::launch_bucket_count(ba, st)) == cudaSuccess &&
        (e = gbsa::launch_bucket_offsets(ba, st)) == cudaSuccess &&
        (e = gbsa::launch_bucket_scatter(ba, st)) == cudaSuccess) {
      gbsa::k_lcp_apply<<<(unsigned)((n + gbsa::LCP_APPLY - 1) / gbsa::LCP_APPLY), 256, 0, st>>>(
          ba.out, n, phi);
    }
  } else {
    gbsa::k_lcp_phi<<<grid_for(n, 8), 256, 0, st>>>(sa, n, phi);
  }
  gbsa::k_lcp_plcp<<<grid_for(chunks, 8), 256, 0, st>>>(text, n, phi, plcp);
  gbsa::k_lcp_gather<<<grid_for(n, 8), 256, 0, st>>>(sa, n, plcp, lcp_out);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (!workspace) {
    const cudaError_t f = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = f;
  }
  return e == cudaSuccess ? SA_OK : SA_ERR_CUDA;
}
