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

int lcp_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  return sms;
}

unsigned grid_for(uint64_t units, int per_sm) {
  const uint64_t want = (units + 255) / 256, cap = (uint64_t)lcp_sm_count() * per_sm;
  return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

GBSA_API size_t sa_lcp_workspace_bytes(uint64_t n) { return 2 * align256((size_t)n * 4); }

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
  uint32_t *phi = static_cast<uint32_t *>(ws);
  uint32_t *plcp = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(ws) + align256(n * 4));
  const uint64_t chunks = (n + gbsa::LCP_CHUNK - 1) / gbsa::LCP_CHUNK;
  gbsa::k_lcp_phi<<<grid_for(n, 8), 256, 0, st>>>(sa, n, phi);
  gbsa::k_lcp_plcp<<<grid_for(chunks, 8), 256, 0, st>>>(text, n, phi, plcp);
  gbsa::k_lcp_gather<<<grid_for(n, 8), 256, 0, st>>>(sa, n, plcp, lcp_out);
  cudaError_t e = cudaGetLastError();
  if (!workspace) {
    const cudaError_t f = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = f;
  }
  return e == cudaSuccess ? SA_OK : SA_ERR_CUDA;
}
