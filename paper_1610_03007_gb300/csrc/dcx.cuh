// Building blocks shared by the difference-cover suffix sorters (DC3 and
// DC7, Section 2.2): a three-phase inclusive scan of u32, stream-ordered
// per-level allocations from the library's pool, and the stable radix sort
// of (key, value) pairs. Each including file gets its own copy (anonymous
// namespace).
#pragma once

#include <algorithm>
#include <vector>

#include "../../include/gbsa.h"
#include "launch.h"
#include "pool.h"

namespace gbsa {
namespace {

constexpr int DC_BLOCK = 256;

// ---- inclusive scan of u32 (three phases; in place allowed) ---------------

constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = DC_BLOCK * SC_ITEMS;

__device__ __forceinline__ uint32_t block_incl_sum(uint32_t v, uint32_t *tmp, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < DC_BLOCK / 32; ++w) {
    const uint32_t s = tmp[w];
    before += w < warp ? s : 0u;
    all += s;
  }
  __syncthreads();
  total = all;
  return before + x;
}

__global__ void __launch_bounds__(DC_BLOCK) k_scan_sums(const uint32_t *__restrict__ in,
                                                        uint64_t m, uint32_t *__restrict__ sums) {
  __shared__ uint32_t tmp[DC_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_ITEMS;
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < m) v += in[base + k];
  uint32_t total;
  block_incl_sum(v, tmp, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive prefix sums of `count` tile sums, in place.
__global__ void __launch_bounds__(DC_BLOCK) k_scan_top(uint32_t *sums, uint32_t count) {
  __shared__ uint32_t tmp[DC_BLOCK / 32];
  const uint32_t per = (count + DC_BLOCK - 1) / DC_BLOCK;
  const uint32_t lo = threadIdx.x * per, hi = min(count, lo + per);
  uint32_t v = 0;
  for (uint32_t i = lo; i < hi; ++i) v += sums[i];
  uint32_t total;
  uint32_t run = block_incl_sum(v, tmp, total) - v;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t s = sums[i];
    sums[i] = run;
    run += s;
  }
}

__global__ void __launch_bounds__(DC_BLOCK) k_scan_apply(const uint32_t *in, uint64_t m,
                                                         const uint32_t *__restrict__ sums,
                                                         uint32_t *out) {
  __shared__ uint32_t tmp[DC_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_ITEMS;
  uint32_t v[SC_ITEMS], s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    v[k] = base + k < m ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_incl_sum(s, tmp, total) - s + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    run += v[k];
    if (base + k < m) out[base + k] = run;
  }
}

uint32_t bits_for_value(uint64_t v) {  // bits to hold 0..v
  uint32_t b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

struct DcxRun {
  cudaStream_t st = nullptr;
  int sms = 1;

  // Stream-ordered allocations of one level, freed when it returns.
  struct Scope {
    DcxRun *d;
    std::vector<void *> ptrs;
    explicit Scope(DcxRun *dd) : d(dd) {}
    ~Scope() {
      for (void *p : ptrs) cudaFreeAsync(p, d->st);
    }
    template <class T>
    sa_status get(T **p, uint64_t count) {
      void *q = nullptr;
      if (library_pool_alloc(&q, (size_t)std::max<uint64_t>(count, 1) * sizeof(T), d->st) !=
          cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_OOM;
      }
      ptrs.push_back(q);
      *p = static_cast<T *>(q);
      return SA_OK;
    }
  };

  unsigned grid(uint64_t m) const {
    const uint64_t want = (m + DC_BLOCK - 1) / DC_BLOCK, cap = (uint64_t)sms * 16;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
  }

  static sa_status ok() { return cudaGetLastError() == cudaSuccess ? SA_OK : SA_ERR_CUDA; }

  // Inclusive prefix sums of in[0, m) into out (may alias in).
  sa_status scan(const uint32_t *in, uint32_t *out, uint64_t m, uint32_t *sums) {
    const uint64_t tiles = (m + SC_TILE - 1) / SC_TILE;
    k_scan_sums<<<(unsigned)tiles, DC_BLOCK, 0, st>>>(in, m, sums);
    k_scan_top<<<1, DC_BLOCK, 0, st>>>(sums, (uint32_t)tiles);
    k_scan_apply<<<(unsigned)tiles, DC_BLOCK, 0, st>>>(in, m, sums, out);
    return ok();
  }

  sa_status sort(uint64_t *keys, uint32_t *vals, uint32_t m, uint32_t bits) {
    return sa_sort_pairs(keys, vals, m, 0, std::min<uint32_t>(64, std::max<uint32_t>(1, bits)),
                         nullptr, 0, (gbsa_stream_t)st);
  }
};

}  // namespace
}  // namespace gbsa
