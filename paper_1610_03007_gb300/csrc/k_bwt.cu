// Burrows-Wheeler transform from the suffix array: the direct consumer of
// SA named as future work at the end of the paper (Section 3), and the
// identity BWT[r] = T[SA[r] - 1] of the definition (Section 2: SA orders
// the suffixes; the BWT lists the character preceding each one).
//
// Rows of T$ (n + 1 of them): row 0 is the suffix $ alone, preceded by
// T[n - 1]; row r >= 1 is the suffix SA[r - 1], preceded by T[SA[r - 1] - 1],
// except the row whose suffix is T itself, which holds $ (stored as 0) and
// whose index is the primary index.
//
// k_bwt: one grid-stride pass over groups of eight rows; SA read and BWT
// written with consecutive addresses, one random byte read of T per row,
// eight of them in flight per thread.
// Bound: HBM. Algorithmic bytes per row: 4 (SA) + 1 (T, random) + 1 (BWT).
#include "../../include/gbsa.h"
#include "launch.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {

// Eight rows per thread: their SA entries, then eight independent text
// reads, then (when BWT is 8-byte aligned and the group is whole) one
// 8-byte store.
__global__ void __launch_bounds__(256) k_bwt(const uint8_t *__restrict__ T, uint64_t n,
                                             const uint32_t *__restrict__ sa,
                                             uint8_t *__restrict__ bwt,
                                             unsigned long long *primary) {
  const uint64_t groups = (n + 1 + 7) / 8;
  const bool packed = (((uintptr_t)bwt) & 7u) == 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
    const uint64_t r0 = 8 * g;
    uint32_t sv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint64_t r = r0 + i;
      sv[i] = (r >= 1 && r <= n) ? sa[r - 1] : 0u;
    }
    uint8_t c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint64_t r = r0 + i;
      c[i] = 0;
      if (r == 0) {
        if (n > 0)
          c[i] = T[n - 1];
        else
          *primary = 0;  // T$ = $: the only row is the text itself
      } else if (r <= n) {
        if (sv[i] == 0)
          *primary = r;
        else if (sv[i] <= n)  // an entry beyond n (not a suffix array) reads nothing
          c[i] = T[sv[i] - 1];
      }
    }
    if (packed && r0 + 7 <= n) {
      uint64_t w = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) w |= (uint64_t)c[i] << (8 * i);
      *reinterpret_cast<uint64_t *>(bwt + r0) = w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (r0 + i <= n) bwt[r0 + i] = c[i];
    }
  }
}

}  // namespace gbsa

namespace {

int sm_count_cached() { return gbsa::device_sm_count(); }

}  // namespace

GBSA_API sa_status sa_bwt(const uint8_t *text, uint64_t n, const uint32_t *sa, uint8_t *bwt_out,
                          uint64_t *primary_out, gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (!bwt_out || !primary_out || (n > 0 && (!text || !sa))) return SA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t groups = (n + 1 + 7) / 8;
  const uint64_t want = (groups + 255) / 256, cap = (uint64_t)sm_count_cached() * 8;
  gbsa::k_bwt<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(
      text, n, sa, bwt_out, reinterpret_cast<unsigned long long *>(primary_out));
  return cudaGetLastError() == cudaSuccess ? SA_OK : SA_ERR_CUDA;
}
