// Output (step A7): the build works on gapped positions (text s occupies
// [off_s + s, off_s + s + len_s), the slot after it is an end sentinel of
// the ISA). SA is written with local indices by the renaming kernels; the
// optional ISA output is gathered here into per-text local ranks.
//
// Bound: HBM; 8 bytes per character.
#include "launch.h"

namespace gbsa {

constexpr int GA_BLOCK = 256;

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
