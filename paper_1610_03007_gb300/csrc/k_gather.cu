// Step A5 — partner names through the inverse suffix array (Section 2.1,
// Algorithm 4: the name of suffix i + 2^k, or the sentinel past the end).
//
// For every active item (g, i'): r2 = ISA[i' + h] + 1, where the slot after
// each text holds 0xFFFFFFFF so the sentinel becomes 0 and sorts below every
// real name (the paper's literal sentinel 0 would collide with the real name
// 0). An active item always has i' + h <= the end slot of its text, because
// a suffix with at most h characters already has a unique name. The sort key
// is (g << W) | r2 with g the group ordinal (rounds keep groups in order)
// and W = bits of the largest r2.
//
// Also the output fix-ups of the batched build (gapped positions -> local
// indices).
//
// Bound: HBM; 8 bytes read + 4 bytes gathered (one 32-byte sector each when
// the ISA exceeds L2) + 12 bytes written per item.
#include "launch.h"

namespace gbsa {

constexpr int GA_BLOCK = 256;

__global__ void __launch_bounds__(GA_BLOCK)
k_gather(const uint64_t *__restrict__ act, uint32_t m, uint32_t h, uint32_t W,
         const uint32_t *__restrict__ isa, uint64_t isa_last, uint64_t *__restrict__ keys,
         uint32_t *__restrict__ vals) {
  const uint64_t j = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x;
  if (j >= m) return;
  const uint64_t a = act[j];
  const uint32_t ip = (uint32_t)a;
  const uint32_t g = (uint32_t)(a >> 32);
  // ip + h never passes the end slot of its text; the clamp only keeps a
  // logic error from reading outside the array.
  const uint64_t at = min((uint64_t)ip + h, isa_last);
  const uint32_t r2 = __ldg(isa + at) + 1u;
  keys[j] = ((uint64_t)g << W) | r2;
  vals[j] = ip;
}

cudaError_t launch_gather(const uint64_t *act, uint32_t m, uint32_t h, uint32_t W,
                          const uint32_t *isa, uint64_t isa_len, uint64_t *keys, uint32_t *vals,
                          cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  const uint64_t grid = ((uint64_t)m + GA_BLOCK - 1) / GA_BLOCK;
  k_gather<<<(unsigned)grid, GA_BLOCK, 0, stream>>>(act, m, h, W, isa, isa_len - 1, keys, vals);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(GA_BLOCK)
k_sa_to_local(uint32_t *sa, uint32_t N, const uint32_t *__restrict__ seg_off, uint32_t S) {
  const uint64_t r = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x;
  if (r >= N) return;
  const uint32_t s = segment_of(seg_off, S, (uint32_t)r);
  sa[r] -= __ldg(seg_off + s) + s;
}

cudaError_t launch_sa_to_local(uint32_t *sa, uint32_t N, const uint32_t *seg_off, uint32_t S,
                               cudaStream_t stream) {
  if (N == 0 || S <= 1) return cudaSuccess;
  const uint64_t grid = ((uint64_t)N + GA_BLOCK - 1) / GA_BLOCK;
  k_sa_to_local<<<(unsigned)grid, GA_BLOCK, 0, stream>>>(sa, N, seg_off, S);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(GA_BLOCK)
k_isa_to_local(const uint32_t *__restrict__ isa, uint32_t *__restrict__ out, uint32_t N,
               const uint32_t *__restrict__ seg_off, uint32_t S) {
  const uint64_t p = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x;
  if (p >= N) return;
  const uint32_t s = S > 1 ? segment_of(seg_off, S, (uint32_t)p) : 0u;
  const uint32_t off = __ldg(seg_off + s);
  out[p] = isa[p + s] - off;
}

cudaError_t launch_isa_to_local(const uint32_t *isa, uint32_t *isa_out, uint32_t N,
                                const uint32_t *seg_off, uint32_t S, cudaStream_t stream) {
  if (N == 0) return cudaSuccess;
  const uint64_t grid = ((uint64_t)N + GA_BLOCK - 1) / GA_BLOCK;
  k_isa_to_local<<<(unsigned)grid, GA_BLOCK, 0, stream>>>(isa, isa_out, N, seg_off, S);
  return cudaGetLastError();
}

}  // namespace gbsa
