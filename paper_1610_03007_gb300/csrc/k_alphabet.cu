// Step A0 — alphabet of the input: a histogram of the 256 byte values, from
// which the host derives sigma, an order-preserving dense code and the bits
// per character b = ceil(log2 sigma). It generalises the character pairs of
// the initial triples (Section 2.1, Algorithm 1): the initial names are
// built from as many dense codes as fit one 64-bit key.
//
// Bound: HBM read of n bytes; 16-byte vector loads, per-warp privatised
// shared-memory counters, one global atomic per bin and block.
#include "launch.h"

namespace gbsa {

constexpr int HIST_BLOCK = 512;
constexpr int HIST_COPIES = HIST_BLOCK / 32;  // one private histogram per warp

__global__ void __launch_bounds__(HIST_BLOCK)
k_byte_histogram(const uint8_t *__restrict__ text, uint64_t n, uint32_t *__restrict__ hist) {
  __shared__ uint32_t s_hist[HIST_COPIES][RADIX];
  for (int x = threadIdx.x; x < HIST_COPIES * RADIX; x += HIST_BLOCK) (&s_hist[0][0])[x] = 0;
  __syncthreads();
  uint32_t *mine = s_hist[threadIdx.x >> 5];
  // Aligned body with 16-byte loads, then the ragged head and tail bytes.
  const uintptr_t addr = (uintptr_t)text;
  uint64_t head = (16 - (addr & 15)) & 15;
  if (head > n) head = n;
  const uint64_t body = (n - head) / 16;
  const uint4 *vec = (const uint4 *)(text + head);
  const uint64_t stride = (uint64_t)gridDim.x * HIST_BLOCK;
  for (uint64_t v = (uint64_t)blockIdx.x * HIST_BLOCK + threadIdx.x; v < body; v += stride) {
    uint4 q = __ldg(vec + v);
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int s = 0; s < 32; s += 8) atomicAdd(&mine[(w[k] >> s) & 255u], 1u);
    }
  }
  const uint64_t tail0 = head + body * 16;
  const uint64_t gtid = (uint64_t)blockIdx.x * HIST_BLOCK + threadIdx.x;
  if (gtid < head) atomicAdd(&mine[text[gtid]], 1u);
  if (gtid < n - tail0) atomicAdd(&mine[text[tail0 + gtid]], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += HIST_BLOCK) {
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < HIST_COPIES; ++c) s += s_hist[c][d];
    if (s) atomicAdd(&hist[d], s);
  }
}

cudaError_t launch_byte_histogram(const uint8_t *text, uint64_t n, uint32_t *hist, int num_sms,
                                  cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  uint64_t want = (n / 16 + HIST_BLOCK - 1) / HIST_BLOCK;
  uint64_t cap = (uint64_t)num_sms * 4;
  unsigned grid = (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
  k_byte_histogram<<<grid, HIST_BLOCK, 0, stream>>>(text, n, hist);
  return cudaGetLastError();
}

}  // namespace gbsa
