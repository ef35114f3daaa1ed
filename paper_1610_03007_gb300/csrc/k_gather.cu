// Output (step A7): the build works on gapped positions (text s occupies
// [off_s + s, off_s + s + len_s), the slot after it is an end sentinel of
// the ISA). SA is written with local indices by the renaming kernels; the
// optional ISA output is gathered here into per-text local ranks.
//
// Bound: HBM; 8 bytes per character.
#include "launch.h"
#include "segcopy.h"

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

// Copies by the SMs instead of a copy engine: small readbacks of the
// control block into pinned host memory, and the text and SA of small
// requests between pinned host buffers and the device. A copy engine runs
// the copies of all streams in order, so a small copy waits behind the
// large copies of concurrent builds; kernel stores and loads to pinned host
// memory (mapped into the device's address space) do not.
__global__ void __launch_bounds__(GA_BLOCK)
k_copy_words(uint32_t *__restrict__ dst, const uint32_t *__restrict__ src, uint64_t words) {
  for (uint64_t i = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * GA_BLOCK)
    dst[i] = src[i];
}

__global__ void __launch_bounds__(GA_BLOCK)
k_copy_bytes(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * GA_BLOCK)
    dst[i] = src[i];
}

cudaError_t launch_copy_words(uint32_t *dst, const uint32_t *src, uint64_t words,
                              cudaStream_t stream) {
  if (words == 0) return cudaSuccess;
  const uint64_t want = (words + GA_BLOCK - 1) / GA_BLOCK, cap = (uint64_t)device_sm_count() * 4;
  k_copy_words<<<(unsigned)(want < cap ? want : cap), GA_BLOCK, 0, stream>>>(dst, src, words);
  return cudaGetLastError();
}

cudaError_t launch_copy_bytes(uint8_t *dst, const uint8_t *src, uint64_t n, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = (n + GA_BLOCK - 1) / GA_BLOCK, cap = (uint64_t)device_sm_count() * 4;
  k_copy_bytes<<<(unsigned)(want < cap ? want : cap), GA_BLOCK, 0, stream>>>(dst, src, n);
  return cudaGetLastError();
}

// The host copies of a merged batch of small requests in one launch: block
// row y copies segment y between the batch's flat device buffer and that
// request's pinned host buffer.
template <typename T, bool TO_FLAT>
__global__ void __launch_bounds__(GA_BLOCK) k_copy_segments(T *__restrict__ flat, SegCopy t) {
  const uint32_t s = blockIdx.y;
  const uint64_t base = t.off[s], len = t.off[s + 1] - base;
  T *ext = static_cast<T *>(t.ext[s]);
  for (uint64_t i = (uint64_t)blockIdx.x * GA_BLOCK + threadIdx.x; i < len;
       i += (uint64_t)gridDim.x * GA_BLOCK) {
    if (TO_FLAT)
      flat[base + i] = ext[i];
    else
      ext[i] = flat[base + i];
  }
}

cudaError_t launch_copy_segments(void *flat, const SegCopy &t, uint32_t elem_bytes, bool to_flat,
                                 cudaStream_t stream) {
  if (t.count == 0 || t.count > SegCopy::MAX || (elem_bytes != 1 && elem_bytes != 4))
    return cudaErrorInvalidValue;
  uint64_t longest = 0;
  for (uint32_t s = 0; s < t.count; ++s) {
    if (t.off[s + 1] < t.off[s]) return cudaErrorInvalidValue;
    const uint64_t len = t.off[s + 1] - t.off[s];
    if (len && !t.ext[s]) return cudaErrorInvalidValue;
    if (len > longest) longest = len;
  }
  if (longest == 0) return cudaSuccess;
  // About four blocks per SM over the whole batch.
  const uint64_t want = (longest + GA_BLOCK - 1) / GA_BLOCK;
  uint64_t cap = (uint64_t)device_sm_count() * 4 / t.count;
  if (cap == 0) cap = 1;
  const dim3 grid((unsigned)(want < cap ? want : cap), t.count);
  if (elem_bytes == 1) {
    if (to_flat)
      k_copy_segments<uint8_t, true><<<grid, GA_BLOCK, 0, stream>>>((uint8_t *)flat, t);
    else
      k_copy_segments<uint8_t, false><<<grid, GA_BLOCK, 0, stream>>>((uint8_t *)flat, t);
  } else {
    if (to_flat)
      k_copy_segments<uint32_t, true><<<grid, GA_BLOCK, 0, stream>>>((uint32_t *)flat, t);
    else
      k_copy_segments<uint32_t, false><<<grid, GA_BLOCK, 0, stream>>>((uint32_t *)flat, t);
  }
  return cudaGetLastError();
}

}  // namespace gbsa
