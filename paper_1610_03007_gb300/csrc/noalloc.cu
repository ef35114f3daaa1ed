// sa_build_noalloc: suffix array of a short text without any device memory
// allocation.
//
// Who needs it: callers that must not call cudaMalloc (or any allocator)
// at the point where they build a suffix array. Typical cases are a host
// process in which another component already owns the device memory (a
// serving engine or framework allocator that reserved the GPU up front, so
// a new cudaMalloc would fail or fragment its pool), latency-sensitive paths
// where cudaMalloc's implicit synchronisation and variable cost are not
// acceptable, and plug-ins whose host forbids device allocation.
//
// How: the whole build workspace lives in the file-scope array below, which
// the CUDA runtime places in device memory when the library's module loads
// on a GPU; every GPU that loads the library keeps these NOALLOC_SCRATCH_BYTES
// until the process exits. Host code cannot use `g_noalloc_scratch` as a
// device address (in host code the name is only a host-side shadow), so
// every call looks up the real device address with cudaGetSymbolAddress in
// the context current at the call. The lookup is a host-side query that
// allocates nothing; it is not cached, because the address belongs to one
// context (after cudaDeviceReset, or in another context on the same device,
// the array lives elsewhere).
//
// The build itself is the ordinary sa_build_ex path given that array as its
// caller-owned workspace; it clears at start everything that must start at
// zero, so the array's leftover contents from the previous call do not
// matter. Like sa_build, it synchronises the stream once per doubling round
// to read the round's counters, so it cannot run while that stream is being
// captured into a CUDA graph. All calls share the one array: calls whose GPU
// work overlaps (two host threads, or two streams without ordering between
// them) race on it and produce garbage, so callers must serialise them.
#include "launch.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

// Largest text accepted: 2^18 bytes; its workspace (sa_workspace_bytes) is
// about 17.8 MiB, checked against the array's size on every call.
constexpr uint64_t NOALLOC_MAX_N = 1ull << 18;
constexpr size_t NOALLOC_SCRATCH_BYTES = 20ull << 20;  // 20 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

GBSA_API sa_status sa_build_noalloc(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                                    gbsa_stream_t stream) {
  if (n > NOALLOC_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  const size_t need = sa_workspace_bytes(n);
  if (need > NOALLOC_SCRATCH_BYTES) return SA_ERR_TOO_LARGE;
  if (n == 0) return SA_OK;
  // The array's device address in the current context (see above).
  void *ws = nullptr;
  if (cudaGetSymbolAddress(&ws, g_noalloc_scratch) != cudaSuccess || !ws) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  // sa_build_ex with its small readbacks on the copy engine: the pinned
  // staging the other entry points use is a host allocation.
  return gbsa::build_single(text, n, sa_out, nullptr, ws, NOALLOC_SCRATCH_BYTES, nullptr,
                            nullptr, stream, false);
}
