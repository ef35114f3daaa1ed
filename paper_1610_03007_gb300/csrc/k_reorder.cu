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
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = gstart[g], e = gstart[g + 1];
    keys[g] = (uint32_t)act[s];
    vals[g] = (uint32_t)g;
    info[g] = make_uint4(s, e - s, gname[g], ghead[g]);
  }
}

// The records in the new order (one random 16-byte read per group), and
// the sizes for the scan.
__global__ void __launch_bounds__(256) k_group_sizes(const SortPlan *__restrict__ plan,
                                                    const uint4 *__restrict__ info, uint32_t G,
                                                    uint4 *__restrict__ info_new,
                                                    uint32_t *__restrict__ sizes, Ctrl *ctrl) {
  const uint32_t *order = plan->vfinal;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < G;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = order[x];
    if (g >= G) {  // never taken unless a logic error
      raise_error(ctrl, ERR_INTERNAL, 17);
      return;
    }
    const uint4 r = info[g];
    info_new[x] = r;
    sizes[x] = r.y;
  }
}

__global__ void __launch_bounds__(256) k_regroup(RegroupArgs a) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.G;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 r = a.info[x];  // (start, size, name, head) of new group x
    const uint32_t s = r.x, z = r.y;
    const uint32_t ns = a.ends[x] - z;
    if ((uint64_t)ns + z > a.m || (uint64_t)s + z > a.m) {  // never taken unless a logic error
      raise_error(a.ctrl, ERR_INTERNAL, 18);
      return;
    }
    a.gstart_out[x] = ns;
    a.gname_out[x] = r.z;
    a.ghead_out[x] = r.w;
    for (uint32_t k = 0; k < z; ++k)
      a.act_out[ns + k] = (x << 32) | (uint32_t)a.act_in[s + k];
    if (x == 0) a.gstart_out[a.G] = a.m;
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
