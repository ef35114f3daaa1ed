// Position bucketing for the ISA writes of Algorithm 5 (new names written
// back through the inverse suffix array, Section 2.1).
//
// The names written back after a rename (round 0: every survivor) or a
// refine (the queued changes) arrive in group order, so their positions i'
// are random: each 4-byte ISA write then dirties its own 32-byte sector, and
// with the ISA several times larger than L2 most sectors are written back
// (and first read) once per name. When many names change, the entries
// ((x << 32) | i') are first partitioned into 256 buckets by i' >> shift,
// one bucket spanning 2^shift positions (8 MB of ISA at n = 2^28), and the
// ISA writes then run in bucket order (blocks launched in array order), so
// the window of ISA being written stays a few buckets wide and in L2.
//
// A radix partition with fixed block ranges (no atomics outside shared
// memory): block b of k_bucket_count owns entries [b*R, (b+1)*R) and
// counts them per bucket; k_bucket_offsets (one block) turns the counts
// into each block's start in each bucket (bucket-major, block-minor);
// k_bucket_scatter re-reads its range in 4096-entry chunks, ranks every
// entry in its bucket with shared-memory atomics, stages the chunk grouped
// by bucket and writes each bucket's run at its block's running offset.
// Order inside a bucket is arbitrary: the ISA writes of one pass commute,
// since every position is written at most once.
//
// A translating partition (BucketArgs.gname set, for the rename's
// survivors) drops the entries whose group kept its parent's name and
// writes the others as (name << 32) | i', reading the group names while the
// entries are still in group order; the ISA writes after it need no
// lookups.
//
// Bound: HBM. Per entry 8 bytes read by the count, 8 read and 8 written by
// the scatter.
#include "launch.h"

namespace gbsa {

namespace {

constexpr int BK_ITEMS = 16;
constexpr int BK_CHUNK = 256 * BK_ITEMS;

struct Range {
  uint64_t lo, n, per;  // first entry, entries, entries per block (a chunk multiple)
};

__device__ __forceinline__ Range entry_range(const BucketArgs &a) {
  Range r;
  r.lo = a.lo ? *a.lo : 0u;
  const uint32_t c = *a.count;
  r.n = c < a.max_count ? c : a.max_count;
  const uint64_t per = (r.n + gridDim.x - 1) / gridDim.x;
  r.per = (per + BK_CHUNK - 1) / BK_CHUNK * BK_CHUNK;
  return r;
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t e, uint32_t shift) {
  return min((uint32_t)e >> shift, (uint32_t)RADIX - 1u);
}

// Translating partition: the entry (g << 32) | i' of a renamed survivor
// becomes (gname[g] << 32) | i', or is dropped (false) when its group kept
// its parent's name. Plain partition: the entry as it is.
__device__ __forceinline__ bool translate(const BucketArgs &a, uint64_t &e) {
  if (!a.gname) return true;
  const uint32_t g = (uint32_t)(e >> 32);
  const uint32_t name = __ldg(a.gname + g);
  if (name == __ldg(a.gold + g)) return false;
  e = ((uint64_t)name << 32) | (uint32_t)e;
  return true;
}

}  // namespace

__global__ void __launch_bounds__(256, 4) k_bucket_count(BucketArgs a) {
  __shared__ uint32_t bins[RADIX];
  const uint32_t t = threadIdx.x;
  bins[t] = 0u;
  __syncthreads();
  const Range r = entry_range(a);
  const uint64_t b0 = (uint64_t)blockIdx.x * r.per;
  const uint64_t b1 = min(b0 + r.per, r.n);
  for (uint64_t c0 = b0; c0 < b1; c0 += BK_CHUNK) {
    uint64_t e[BK_ITEMS];
#pragma unroll
    for (int k = 0; k < BK_ITEMS; ++k) {
      const uint64_t x = c0 + (uint64_t)k * 256 + t;
      e[k] = x < b1 ? a.in[r.lo + x] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < BK_ITEMS; ++k)
      if (c0 + (uint64_t)k * 256 + t < b1 && translate(a, e[k]))
        atomicAdd(&bins[bucket_of(e[k], a.shift)], 1u);
  }
  __syncthreads();
  a.counts[(size_t)blockIdx.x * RADIX + t] = bins[t];
}

// One block: counts[b][k] -> start of block b's run in bucket k.
__global__ void __launch_bounds__(256) k_bucket_offsets(BucketArgs a, uint32_t blocks) {
  __shared__ uint32_t wtot[8];
  const uint32_t k = threadIdx.x, lane = k & 31, warp = k >> 5;
  uint32_t total = 0;
#pragma unroll 16
  for (uint32_t b = 0; b < blocks; ++b) total += a.counts[(size_t)b * RADIX + k];
  const uint32_t incl = warp_inclusive(total, OpAdd());
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t run = incl - total;
#pragma unroll
  for (int w = 0; w < 8; ++w) run += (uint32_t)w < warp ? wtot[w] : 0u;
  for (uint32_t b0 = 0; b0 < blocks; b0 += 16) {
    uint32_t c[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
      c[i] = b0 + i < blocks ? a.counts[(size_t)(b0 + i) * RADIX + k] : 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (b0 + i < blocks) a.counts[(size_t)(b0 + i) * RADIX + k] = run;
      run += c[i];
    }
  }
  if (a.total_out && k == RADIX - 1) *a.total_out = run;  // the end of the last bucket
}

// Per chunk: rank each entry in its bucket (shared atomics), scan the
// chunk's bucket counts into local offsets, stage the chunk in shared memory
// grouped by bucket, then write it out so that consecutive threads store
// consecutive slots of each bucket run.
__global__ void __launch_bounds__(256, 4) k_bucket_scatter(BucketArgs a) {
  __shared__ uint64_t stage[BK_CHUNK];
  __shared__ uint32_t run[RADIX], cnt[RADIX], at0[RADIX], lofs[RADIX];
  __shared__ uint32_t wtot[8];
  __shared__ uint32_t kept_sh;
  const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
  run[t] = a.counts[(size_t)blockIdx.x * RADIX + t];
  cnt[t] = 0u;
  __syncthreads();
  const Range r = entry_range(a);
  const uint64_t b0 = (uint64_t)blockIdx.x * r.per;
  const uint64_t b1 = min(b0 + r.per, r.n);
  for (uint64_t c0 = b0; c0 < b1; c0 += BK_CHUNK) {
    const uint32_t len = (uint32_t)min((uint64_t)BK_CHUNK, b1 - c0);
    uint64_t e[BK_ITEMS];
    uint32_t rk[BK_ITEMS];
    uint32_t keep = 0;  // bit k: entry k is written
#pragma unroll
    for (int k = 0; k < BK_ITEMS; ++k) {
      const uint32_t x = (uint32_t)k * 256 + t;
      e[k] = x < len ? a.in[r.lo + c0 + x] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < BK_ITEMS; ++k)
      if ((uint32_t)k * 256 + t < len && translate(a, e[k])) {
        keep |= 1u << k;
        rk[k] = atomicAdd(&cnt[bucket_of(e[k], a.shift)], 1u);
      }
    __syncthreads();
    {
      const uint32_t c = cnt[t];
      const uint32_t incl = warp_inclusive(c, OpAdd());
      if (lane == 31) wtot[warp] = incl;
      at0[t] = run[t];
      run[t] += c;
      __syncthreads();
      uint32_t before = incl - c;
#pragma unroll
      for (int w = 0; w < 8; ++w) before += (uint32_t)w < warp ? wtot[w] : 0u;
      lofs[t] = before;
      if (t == RADIX - 1) kept_sh = before + c;  // entries the chunk keeps
      cnt[t] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK_ITEMS; ++k)
      if ((keep >> k) & 1u) stage[lofs[bucket_of(e[k], a.shift)] + rk[k]] = e[k];
    __syncthreads();
    const uint32_t kept = kept_sh;  // == len unless the partition translates
    for (uint32_t i = t; i < kept; i += 256) {
      const uint64_t v = stage[i];
      const uint32_t b = bucket_of(v, a.shift);
      const uint32_t at = at0[b] + (i - lofs[b]);
      if (at < a.max_count) a.out[at] = v;
    }
    __syncthreads();
  }
}

cudaError_t launch_bucket_count(const BucketArgs &a, cudaStream_t stream) {
  k_bucket_count<<<a.blocks, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucket_offsets(const BucketArgs &a, cudaStream_t stream) {
  k_bucket_offsets<<<1, 256, 0, stream>>>(a, a.blocks);
  return cudaGetLastError();
}

cudaError_t launch_bucket_scatter(const BucketArgs &a, cudaStream_t stream) {
  k_bucket_scatter<<<a.blocks, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace gbsa
