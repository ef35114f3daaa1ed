// Device-driven rounds: the loop of Algorithm 5 (Section 2.1; repeat the
// doubling step until no suffix is active, the `I.Size() = 0` test) run on
// the GPU, without a host round trip per round.
//
// The host captures rounds >= 1 once into a CUDA graph: a while-node whose
// body is two rounds (the active lists and group tables alternate between
// two buffers) followed by k_round_end. Each round starts with
// k_round_begin, which turns the previous round's counters into this
// round's sizes (the round state the kernels read instead of host
// arguments), clears the round's counters and histograms, and sets the
// if-nodes of the round's optional steps: the large-group gather and radix
// sort, their rename, and the position bucketing of the ISA writes. Every
// kernel of a round returns at once when the state says the loop is over,
// so the second round of a body costs nothing after the first ended it.
// k_round_end sets the while-node's condition: another iteration while
// suffixes are active and no error was raised.
#include "launch.h"

namespace gbsa {

__global__ void __launch_bounds__(256) k_round_begin(RoundBeginArgs a) {
  Ctrl *c = a.ctrl;
  RoundState &rs = c->rs;
  __shared__ uint32_t s_go;
  if (threadIdx.x == 0) {
    uint32_t go = 0;
    if (rs.live) {
      const RoundCounts rc = c->rc;
      if (rs.round >= 1 && rs.round < (uint32_t)DEV_MAX_ROUNDS) {
        RoundRecord &done = c->rec[rs.round];  // what the previous round produced
        done.m_s = rc.m_s;
        done.g_s = rc.g_s;
        done.m_l = rc.m_l;
        done.g_l = rc.g_l;
        done.upd = rc.upd;
        done.passes = c->passes;
      }
      const uint32_t m = rc.m_s + rc.m_l;
      if (m == 0 || has_error(c)) {
        rs.live = 0;
      } else if (rs.round + 1 >= (uint32_t)DEV_MAX_ROUNDS || rs.h_next > a.N) {
        raise_error(c, ERR_INTERNAL, 14);  // more rounds than the method can take
        rs.live = 0;
      } else {
        const uint32_t r = rs.round + 1;
        const uint32_t mL = (uint32_t)rc.large, GL = (uint32_t)(rc.large >> 32);
        rs.round = r;
        rs.m = m;
        rs.G = rc.g_s + rc.g_l;
        rs.mL = mL;
        rs.GL = GL;
        rs.h = rs.h_next;
        rs.h_next = rs.h_next * 2u;
        rs.tiles = (m + a.nominal - 1) / a.nominal;
        rs.epoch += ROUND_EPOCHS;
        rs.bucket_upd = m >= a.bucket_min ? 1u : 0u;
        rs.bucket_surv = mL >= a.bucket_min ? 1u : 0u;
        // the large groups' keys: (large-group ordinal << W) | partner name
        const uint32_t kbits = a.W + (GL > 1 ? 32u - __clz(GL - 1) : 0u);
        DigitSpec sp{};
        sp.P = (kbits + RADIX_BITS - 1) / RADIX_BITS;
        for (uint32_t p = 0; p < sp.P; ++p) {
          sp.shift[p] = (uint8_t)(p * RADIX_BITS);
          sp.bits[p] = (uint8_t)min((uint32_t)RADIX_BITS, kbits - p * RADIX_BITS);
        }
        rs.spec = sp;
        RoundRecord &now = c->rec[r];
        now.m = m;
        now.G = rs.G;
        now.mL = mL;
        now.GL = GL;
        c->passes = 0;
        go = 1;
      }
    }
    s_go = go;
    const bool large = go && rs.mL > 0;
    cudaGraphSetConditional(a.if_sort, large ? 1u : 0u);
    cudaGraphSetConditional(a.if_rename, large ? 1u : 0u);
    cudaGraphSetConditional(a.if_bucket_upd, go && rs.bucket_upd ? 1u : 0u);
    cudaGraphSetConditional(a.if_bucket_surv, large && rs.bucket_surv ? 1u : 0u);
  }
  __syncthreads();
  if (!s_go) return;
  // The round's counters start at zero (thread 0 read them above).
  for (uint32_t x = threadIdx.x; x < (uint32_t)TILE_COUNTERS; x += blockDim.x) c->tile_ctr[x] = 0u;
  for (uint32_t x = threadIdx.x; x < (uint32_t)(MAX_PASSES * RADIX); x += blockDim.x)
    a.hist[x] = 0u;
  if (threadIdx.x == 0) c->rc = RoundCounts{};
}

__global__ void k_round_end(const Ctrl *c, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  const bool more = c->rs.live && (c->rc.m_s + c->rc.m_l) > 0 && !has_error(c);
  cudaGraphSetConditional(loop, more ? 1u : 0u);
}

cudaError_t launch_round_begin(const RoundBeginArgs &a, cudaStream_t stream) {
  k_round_begin<<<1, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_round_end(const Ctrl *c, cudaGraphConditionalHandle loop, cudaStream_t stream) {
  k_round_end<<<1, 32, 0, stream>>>(c, loop);
  return cudaGetLastError();
}

}  // namespace gbsa
