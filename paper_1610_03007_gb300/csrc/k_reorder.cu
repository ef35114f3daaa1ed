// Group order for the rounds after round 0 (Section 2.1, Algorithm 5: the
// order of the groups in the active list is free, since names are
// absolute ranks and a round only needs each group contiguous).
//
// Round 0 leaves the groups in rank order, in which neighbouring groups
// are unrelated text positions: every partner-name read ISA[i' + h] of a
// later round is then a random 4-byte access (a DRAM sector or two per
// read on a text far larger than L2). Repeats make groups of positions
// that move together: the suffixes of a copied segment and of its source
// form pairs (p, p + d), (p + 1, p + 1 + d), ..., and the copies of a
// repeated text groups {p, p + B, p + 2B, ...}, {p + 1, ...}. With the
// groups ordered by their first member's position, neighbouring groups --
// handled by neighbouring threads and by tiles in flight at the same time
// -- read neighbouring ISA entries, so the reads share cache lines and L2
// sectors. The rounds keep the order approximately (each tile writes its
// subgroups in place of its groups, and tiles start in order), so the
// groups are reordered once, after round 0:
//
//   k_group_minpos: key = the group's smallest member position, value = g,
//                   and a 16-byte record (start, size, name, head rank)
//   radix sort of (key, g) by the 32 key bits (the pass of step A2)
//   k_group_sizes:  the records in the new order (one random read each)
//                   and the sizes
//   inclusive scan: their ends (three-phase, from the DC3/DC7 helpers)
//   k_regroup:      entries (g' << 32) | i', starts, names and head ranks
//                   written to the other buffer set under the new ordinals
//
// then the classification runs again on the new tables.
#include "dcx.cuh"

namespace gbsa {

// keys[g] = smallest member position, vals[g] = g, info[g] = (start, size,
// name, head rank): read here in group order (coalesced), so that after
// the sort one 16-byte record per group is all that is read at random.
// After round 0 a group's members are in increasing position order (the
// keys are laid out with positions ascending after a text's tails, which
// are never survivors, and the sort is stable), so the smallest is the
// first: one read per group. (Were it not, the order would only be
// approximate; every order of the groups is valid.)
__global__ void __launch_bounds__(256) k_group_minpos(const uint64_t *__restrict__ act,
                                                     const uint32_t *__restrict__ gstart,
                                                     const uint32_t *__restrict__ gname,
                                                     const uint32_t *__restrict__ ghead,
                                                     uint32_t G, uint64_t *__restrict__ keys,
                                                     uint32_t *__restrict__ vals,
                                                     uint4 *__restrict__ info) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < G; g0 += 4 * stride) {
    uint32_t s[4], e[4];  // four groups' loads in flight before any is used
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t g = g0 + u * stride;
      s[u] = g < G ? gstart[g] : 0u;
      e[u] = g < G ? gstart[g + 1] : 0u;
    }
    uint64_t first[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) first[u] = g0 + u * stride < G ? act[s[u]] : 0ull;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t g = g0 + u * stride;
      if (g >= G) break;
      keys[g] = (uint32_t)first[u];
      vals[g] = (uint32_t)g;
      info[g] = make_uint4(s[u], e[u] - s[u], gname[g], ghead[g]);
    }
  }
}

// The records in the new order (one random 16-byte read per group), and
// the sizes for the scan.
// RG_UNROLL groups per thread and iteration in the two gathering kernels
// below: their loads are issued before any is used, so each thread keeps
// several random reads in flight.
constexpr int RG_UNROLL = 4;

__global__ void __launch_bounds__(256) k_group_sizes(const SortPlan *__restrict__ plan,
                                                    const uint4 *__restrict__ info, uint32_t G,
                                                    uint4 *__restrict__ info_new,
                                                    uint32_t *__restrict__ sizes, Ctrl *ctrl) {
  const uint32_t *order = plan->vfinal;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < G;
       x0 += RG_UNROLL * stride) {
    uint32_t g[RG_UNROLL];
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) g[u] = x0 + u * stride < G ? order[x0 + u * stride] : 0u;
    uint4 r[RG_UNROLL];
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) {
      if (g[u] >= G) {  // never taken unless a logic error
        raise_error(ctrl, ERR_INTERNAL, 17);
        return;
      }
      r[u] = x0 + u * stride < G ? info[g[u]] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) {
      const uint64_t x = x0 + u * stride;
      if (x < G) {
        info_new[x] = r[u];
        sizes[x] = r[u].y;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_regroup(RegroupArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < a.G;
       x0 += RG_UNROLL * stride) {
    uint4 r[RG_UNROLL];  // (start, size, name, head) of new group x
    uint32_t end[RG_UNROLL];
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) {
      const uint64_t x = x0 + u * stride;
      r[u] = x < a.G ? a.info[x] : make_uint4(0u, 0u, 0u, 0u);
      end[u] = x < a.G ? a.ends[x] : 0u;
    }
    // The first two members of each group (most groups are pairs), loaded
    // together; longer groups read the rest in their own loop.
    uint64_t e0[RG_UNROLL], e1[RG_UNROLL];
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) {
      const uint32_t s = r[u].x, z = r[u].y;
      // never taken unless a logic error
      if ((uint64_t)end[u] > a.m || (uint64_t)s + z > a.m || z > end[u]) {
        raise_error(a.ctrl, ERR_INTERNAL, 18);
        return;
      }
      e0[u] = z > 0 ? a.act_in[s] : 0ull;
      e1[u] = z > 1 ? a.act_in[s + 1] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < RG_UNROLL; ++u) {
      const uint64_t x = x0 + u * stride;
      if (x >= a.G) break;
      const uint32_t s = r[u].x, z = r[u].y, ns = end[u] - z;
      a.gstart_out[x] = ns;
      a.gname_out[x] = r[u].z;
      a.ghead_out[x] = r[u].w;
      if (z > 0) a.act_out[ns] = (x << 32) | (uint32_t)e0[u];
      if (z > 1) a.act_out[ns + 1] = (x << 32) | (uint32_t)e1[u];
      for (uint32_t k = 2; k < z; ++k) a.act_out[ns + k] = (x << 32) | (uint32_t)a.act_in[s + k];
      if (x == 0) a.gstart_out[a.G] = a.m;
    }
  }
}

cudaError_t launch_group_minpos(const uint64_t *act, const uint32_t *gstart, const uint32_t *gname,
                                const uint32_t *ghead, uint32_t G, uint64_t *keys, uint32_t *vals,
                                uint4 *info, int num_sms, cudaStream_t stream) {
  if (G == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)G + 255) / 256, cap = (uint64_t)num_sms * 16;
  k_group_minpos<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(act, gstart, gname,
                                                                        ghead, G, keys, vals, info);
  return cudaGetLastError();
}

cudaError_t launch_group_sizes(const SortPlan *plan, const uint4 *info, uint32_t G,
                               uint4 *info_new, uint32_t *sizes, Ctrl *ctrl, int num_sms,
                               cudaStream_t stream) {
  if (G == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)G + 255) / 256, cap = (uint64_t)num_sms * 16;
  k_group_sizes<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(plan, info, G, info_new,
                                                                       sizes, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_inclusive_scan(const uint32_t *in, uint32_t *out, uint64_t m, uint32_t *sums,
                                  cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  DcxRun d;
  d.st = stream;
  return d.scan(in, out, m, sums) == SA_OK ? cudaSuccess : cudaErrorLaunchFailure;
}

uint64_t inclusive_scan_sums_words(uint64_t m) { return (m + SC_TILE - 1) / SC_TILE; }

cudaError_t launch_regroup(const RegroupArgs &a, int num_sms, cudaStream_t stream) {
  if (a.G == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)a.G + 255) / 256, cap = (uint64_t)num_sms * 16;
  k_regroup<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace gbsa
