// The library's private stream-ordered memory pool (defined in engine.cu):
// never trimmed, so repeated calls reuse its memory; free with cudaFreeAsync.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace gbsa {
cudaError_t library_pool_alloc(void **p, size_t bytes, cudaStream_t st);
}  // namespace gbsa
