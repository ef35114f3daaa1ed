// Prefix doubling using sorting (Section 2.1, Algorithms 1, 2 and 3; Eq. 1):
// every round sorts all n suffixes, and the partner names come from a
// second sort instead of random reads of an inverse suffix array.
//
//   Initial triples (i, T[i], T[i+1]) with T[n] = $ (Algorithm 1), as the
//   key (T[i] + 1, T[i+1] + 1 or 0).
//   Per round k = 1, 2, ...:
//     sort S by its name pair; CmpName (Algorithm 2): a flag where the pair
//     differs from its predecessor; the new name of item x is the largest
//     flagged x' <= x (PrefixSum with max: the head rank), computed from an
//     inclusive sum of the flags (group g of x) and the head of every group.
//     If all n flags are set, the positions in S's order are SA.
//     Otherwise (Algorithm 3) sort the (position, name) items by the
//     comparator of Eq. 1, i.e. by the key (i mod 2^k, i div 2^k), so that
//     the item after i is i + 2^k whenever that position exists, and pair
//     each name with its successor's (+1; 0, the sentinel, where the
//     successor is not i + 2^k).
// Reading: names start at 0, so the partner sentinel is 0 and a partner
// name is stored + 1 (the paper's sentinel 0 would equal the name 0).
//
// Bound: HBM. Per round two radix sorts of n (key, value) pairs (the pair
// key has 2 bits(n) significant bits, the comparator key bits(n)), three
// streaming passes for flags, scan and names, and the window pass.
#include "dcx.cuh"

#define GBSA_API extern "C" __attribute__((visibility("default")))

namespace gbsa {
namespace {

__global__ void k_ps_pairs(const uint8_t *__restrict__ T, uint32_t n, uint64_t *__restrict__ keys,
                           uint32_t *__restrict__ vals) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c0 = (uint32_t)T[i] + 1u, c1 = i + 1 < n ? (uint32_t)T[i + 1] + 1u : 0u;
    keys[i] = ((uint64_t)c0 << 9) | c1;
    vals[i] = (uint32_t)i;
  }
}

// CmpName: 1 where the key differs from its predecessor (and at x = 0).
__global__ void k_ps_flags(const uint64_t *__restrict__ keys, uint32_t n,
                           uint32_t *__restrict__ flags) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x)
    flags[x] = (x == 0 || keys[x] != keys[x - 1]) ? 1u : 0u;
}

// g = inclusive sum of the flags: head[g - 1] = x where x starts group g.
__global__ void k_ps_heads(const uint32_t *__restrict__ g, uint32_t n, uint32_t *__restrict__ head) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t gx = g[x];
    if ((x == 0 || g[x - 1] != gx) && gx >= 1 && gx <= n) head[gx - 1] = (uint32_t)x;
  }
}

// The new name of item x (its group's head rank) with its position, keyed
// for the next round's sort by Eq. 1: key = (i mod 2^k) << wd | (i div 2^k).
// trace (if not NULL): trace[pos] = name.
__global__ void k_ps_names(const uint32_t *__restrict__ g, const uint32_t *__restrict__ head,
                           const uint32_t *__restrict__ pos, uint32_t n, uint32_t k, uint32_t wd,
                           uint64_t *__restrict__ kN, uint32_t *__restrict__ vN,
                           uint32_t *__restrict__ trace) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t gx = g[x];
    const uint32_t name = gx >= 1 && gx <= n ? head[gx - 1] : 0u;
    const uint32_t i = pos[x];
    if (trace && i < n) trace[i] = name;
    if (kN) {
      kN[x] = ((uint64_t)(i & ((1u << k) - 1u)) << wd) | (uint64_t)(i >> k);
      vN[x] = name;
    }
  }
}

// Window of two over the items in Eq. 1's order: the pair (name of i, name
// of i + 2^k + 1, or 0 if the next item is not i + 2^k) keyed for the sort
// by name pair; the position rides along.
__global__ void k_ps_window(const uint64_t *__restrict__ kN, const uint32_t *__restrict__ vN,
                            uint32_t n, uint32_t k, uint32_t wd, uint32_t wr,
                            uint64_t *__restrict__ kS, uint32_t *__restrict__ vS) {
  const uint64_t low = ((uint64_t)1 << wd) - 1;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = kN[x];
    const uint64_t i = ((key & low) << k) | (key >> wd);
    uint32_t r1 = 0;
    if (x + 1 < n) {
      const uint64_t kn = kN[x + 1];
      const uint64_t inext = ((kn & low) << k) | (kn >> wd);
      if (inext == i + ((uint64_t)1 << k)) r1 = vN[x + 1] + 1u;
    }
    kS[x] = ((uint64_t)vN[x] << wr) | r1;
    vS[x] = (uint32_t)i;
  }
}

struct PdSort : DcxRun {
  sa_status run(const uint8_t *text, uint32_t n, uint32_t *sa, uint32_t *trace, uint32_t cap,
                uint32_t *rounds_out) {
    Scope sc(this);
    uint64_t *kS, *kN;
    uint32_t *vS, *vN, *g, *head, *sums;
    const uint64_t tiles = ((uint64_t)n + SC_TILE - 1) / SC_TILE;
    sa_status s;
    if ((s = sc.get(&kS, n)) != SA_OK || (s = sc.get(&kN, n)) != SA_OK ||
        (s = sc.get(&vS, n)) != SA_OK || (s = sc.get(&vN, n)) != SA_OK ||
        (s = sc.get(&g, n)) != SA_OK || (s = sc.get(&head, n)) != SA_OK ||
        (s = sc.get(&sums, tiles)) != SA_OK)
      return s;
    const uint32_t wr = bits_for_value(n);  // names in [0, n), partners in [0, n]
    k_ps_pairs<<<grid(n), DC_BLOCK, 0, st>>>(text, n, kS, vS);
    if ((s = ok()) != SA_OK || (s = sort(kS, vS, n, 18)) != SA_OK) return s;
    for (uint32_t round = 0;; ++round) {
      if (round > 40) return SA_ERR_INTERNAL;
      // CmpName and PrefixSum(max): head-rank names in S's order.
      k_ps_flags<<<grid(n), DC_BLOCK, 0, st>>>(kS, n, g);
      if ((s = ok()) != SA_OK || (s = scan(g, g, n, sums)) != SA_OK) return s;
      k_ps_heads<<<grid(n), DC_BLOCK, 0, st>>>(g, n, head);
      uint32_t count = 0;
      if ((s = ok()) != SA_OK ||
          cudaMemcpyAsync(&count, g + n - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return s != SA_OK ? s : SA_ERR_CUDA;
      const bool done = count == n;
      const uint32_t k = round + 1;  // the names resolve 2^k characters
      const uint32_t wd = bits_for_value((n - 1) >> std::min<uint32_t>(k, 31));
      uint32_t *tr = trace && round < cap ? trace + (uint64_t)round * n : nullptr;
      if (done || k >= 32) {
        if (tr) k_ps_names<<<grid(n), DC_BLOCK, 0, st>>>(g, head, vS, n, 0, 0, nullptr,
                                                          nullptr, tr);
        if ((s = ok()) != SA_OK) return s;
        if (!done) return SA_ERR_INTERNAL;
        if (rounds_out) *rounds_out = round + 1;
        if (cudaMemcpyAsync(sa, vS, (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          return SA_ERR_CUDA;
        return SA_OK;
      }
      // Algorithm 3: sort by Eq. 1, then pair each name with its successor's.
      k_ps_names<<<grid(n), DC_BLOCK, 0, st>>>(g, head, vS, n, k, wd, kN, vN, tr);
      if ((s = ok()) != SA_OK || (s = sort(kN, vN, n, k + wd)) != SA_OK) return s;
      k_ps_window<<<grid(n), DC_BLOCK, 0, st>>>(kN, vN, n, k, wd, wr, kS, vS);
      if ((s = ok()) != SA_OK || (s = sort(kS, vS, n, 2 * wr)) != SA_OK) return s;
    }
  }
};

}  // namespace
}  // namespace gbsa

GBSA_API sa_status sa_build_pd_sort(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                                    uint32_t *trace_names, uint32_t trace_cap, uint32_t *rounds,
                                    gbsa_stream_t stream) {
  if (n > SA_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  if (rounds) *rounds = 0;
  if (n == 0) return SA_OK;
  gbsa::PdSort d;
  d.st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SA_ERR_CUDA;
  sa_status s = d.run(text, (uint32_t)n, sa_out, trace_names, trace_names ? trace_cap : 0, rounds);
  if (s == SA_OK && cudaStreamSynchronize(d.st) != cudaSuccess) return SA_ERR_CUDA;
  return s;
}
