// Step A1 — initial keys (Section 2.1, Algorithm 1: the initial name pairs
// (T[i], T[i+1]); here c0 characters per key instead of 2).
//
// key = (text id << c0*b) | the dense codes of T[i .. i+c0), first
// character most significant, zero-padded past the end of the text.
//
// Padding with code 0 lets a short suffix near the end tie with a longer
// suffix whose next characters have code 0. Such a tail suffix (fewer than
// c0 characters left) is smaller than every longer suffix with the same key,
// and among tails with equal keys the shorter is smaller. So keys are laid
// out tail-first within each text: the c0-1 last positions in descending
// order, then the others ascending. The stable sort keeps that order inside
// runs of equal keys, and the round-0 rename gives every tail a group of
// its own.
//
// vals hold gapped positions: text s occupies [off_s + s, off_s + s + len_s)
// and the slot right after it is an end sentinel of the ISA.
//
// Bound: HBM, N bytes read (+ L1-cached overlap of c0-1 bytes per key),
// 12 N bytes written.
#include "launch.h"

namespace gbsa {

constexpr int PACK_BLOCK = 256;

__global__ void __launch_bounds__(PACK_BLOCK) k_pack(PackArgs a) {
  __shared__ uint8_t s_code[RADIX];
  s_code[threadIdx.x] = a.code[threadIdx.x];
  __syncthreads();
  const uint64_t j64 = (uint64_t)blockIdx.x * PACK_BLOCK + threadIdx.x;
  if (j64 >= a.N) return;
  const uint32_t j = (uint32_t)j64;
  const uint32_t s = a.S > 1 ? segment_of(a.seg_off, a.S, j) : 0u;
  const uint32_t off = __ldg(a.seg_off + s);
  const uint32_t len = __ldg(a.seg_off + s + 1) - off;
  const uint32_t rel = j - off;
  const uint32_t t = len < a.c0 - 1 ? len : a.c0 - 1;  // tail positions of this text
  const uint32_t irel = rel < t ? len - 1 - rel : rel - t;
  const uint32_t avail = len - irel;
  const uint32_t take = avail < a.c0 ? avail : a.c0;
  const uint8_t *p = a.text + off + irel;
  uint64_t key = 0;
  for (uint32_t q = 0; q < take; ++q)
    key |= (uint64_t)s_code[__ldg(p + q)] << (a.cb - a.b * (q + 1));
  if (a.S > 1) key |= (uint64_t)s << a.cb;
  a.keys[j] = key;
  a.vals[j] = off + irel + s;
}

cudaError_t launch_pack(const PackArgs &a, cudaStream_t stream) {
  if (a.N == 0) return cudaSuccess;
  uint64_t grid = ((uint64_t)a.N + PACK_BLOCK - 1) / PACK_BLOCK;
  k_pack<<<(unsigned)grid, PACK_BLOCK, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace gbsa
