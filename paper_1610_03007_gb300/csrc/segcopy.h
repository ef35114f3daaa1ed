// Host copies of a merged batch of small requests (k_gather.cu): the texts
// of up to MAX requests into one flat device buffer, and their SAs back, each
// in one kernel launch through the device mapping of pinned host memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbsa {

// Passed by value as a kernel parameter: segment s is
// flat[off[s] .. off[s+1]) (in elements) and ext[s] its own buffer (the
// device address of pinned host memory; unused when the segment is empty).
struct SegCopy {
  static constexpr uint32_t MAX = 64;
  void *ext[MAX];
  uint64_t off[MAX + 1];
  uint32_t count;  // 1 .. MAX
};

// to_flat: ext[s] -> flat segments (the texts in); else flat -> ext[s] (the
// SAs out). elem_bytes is 1 (bytes) or 4 (words). cudaErrorInvalidValue for
// a malformed table (count outside 1 .. MAX, decreasing offsets, a missing
// buffer of a non-empty segment).
cudaError_t launch_copy_segments(void *flat, const SegCopy &t, uint32_t elem_bytes, bool to_flat,
                                 cudaStream_t stream);

}  // namespace gbsa
