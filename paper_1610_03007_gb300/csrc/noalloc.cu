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
// device address (in host code the name is only a host-side shadow), so the
// first call on each device looks up the real device address with
// cudaGetSymbolAddress while that device is current and caches it. That
// first call therefore does a runtime query and should happen before any
// stream capture is begun on that device.
//
// The build itself is the ordinary sa_build_ex path given that array as its
// caller-owned workspace; it clears at start everything that must start at
// zero, so the array's leftover contents from the previous call do not
// matter. All calls share the one array: calls whose GPU work overlaps (two
// host threads, or two streams without ordering between them) race on it
// and produce garbage, so callers must serialise them.
#include <mutex>

#include "../../include/gbsa.h"

#define GBSA_API extern "C" __attribute__((visibility("default")))

// Largest text accepted: 2^18 bytes; its workspace is about 17.8 MiB.
constexpr uint64_t NOALLOC_MAX_N = 1ull << 18;
constexpr size_t NOALLOC_SCRATCH_BYTES = 20ull << 20;  // 20 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device). Returns nullptr on failure.
void *scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

GBSA_API sa_status sa_build_noalloc(const uint8_t *text, uint64_t n, uint32_t *sa_out,
                                    gbsa_stream_t stream) {
  if (n > NOALLOC_MAX_N) return SA_ERR_TOO_LARGE;
  if (n > 0 && (!text || !sa_out)) return SA_ERR_INVALID_ARG;
  const size_t need = sa_workspace_bytes(n);
  if (need > NOALLOC_SCRATCH_BYTES) return SA_ERR_TOO_LARGE;
  if (n == 0) return SA_OK;
  void *ws = scratch_address();
  if (!ws) return SA_ERR_CUDA;
  return sa_build_ex(text, n, sa_out, nullptr, ws, NOALLOC_SCRATCH_BYTES, nullptr, nullptr,
                     stream);
}
