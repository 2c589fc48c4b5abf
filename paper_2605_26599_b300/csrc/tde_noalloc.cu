// tde_eigvals_noalloc: the single-matrix solve with its workspace in a fixed
// device array that ships inside the library, for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// for example a plugin or callback that is handed device pointers by a host
// framework which owns every allocation (and may forbid allocating while it is
// capturing or replaying work), or a caller that must not add allocator
// traffic or fragmentation to a pool it does not control.  Such a caller can
// pass d, e and lambda but has no way to provide the O(n) workspace that
// tde_eigvals asks for.
//
// How: the workspace is the file-scope array g_noalloc_scratch below
// (kNoallocBytes = 4 MiB, enough for n <= TDE_NOALLOC_MAX_N = 16384 with any leaf
// order).  Every GPU on which this library is loaded keeps that array until the
// process exits.  Host code cannot use the array's name as a device address, so
// the first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; later calls on the device reuse it.
// Because the lookup may load the module, make the first call on a device
// before any stream capture begins.  The cached address belongs to the device's
// primary context: after cudaDeviceReset, or from a different context on the
// same device, the module is loaded again and the array may move, so such
// callers must not use this entry point (it has no way to notice the change).
//
// Sharing: every call on a device uses the same array and it keeps the previous
// call's contents.  The solver resets what must start at zero (the status word,
// the root counters, the per-matrix scale words) at the start of each call with
// cudaMemsetAsync, and writes every other section before reading it.  Calls whose
// execution overlaps on the GPU (different streams without ordering, or several
// host threads) race on the array and corrupt each other's results; serialise
// them.  The device status word (no convergence, non-finite input) sits at the
// start of the array like at the start of a caller workspace; tde_noalloc_get_info
// reads it.  tde_read_work does not apply to this entry point.
#include <mutex>

#include "tde_internal.cuh"

namespace tde {

constexpr size_t kNoallocBytes = size_t(4) << 20;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

__global__ void k_noalloc_offsets(int64_t* off, int64_t n) {
  off[0] = 0;
  off[1] = n;
}

// Device address of the scratch array on the current device (looked up once).
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDE_ECUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return TDE_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
      return TDE_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return TDE_OK;
}

}  // namespace tde

extern "C" int tde_eigvals_noalloc(int64_t n, const double* d, const double* e, double* lambda,
                                   int32_t leaf, void* stream) {
  using namespace tde;
  g_launches = 0;
  if (n < 0) return TDE_EINVAL;
  if (n > TDE_NOALLOC_MAX_N) return TDE_EWORKSPACE;
  if (n == 0) return TDE_OK;
  if (d == nullptr || lambda == nullptr || (n > 1 && e == nullptr)) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  if (carve_workspace(p, nullptr, nullptr) > kNoallocBytes) return TDE_EWORKSPACE;
  void* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc != TDE_OK) return rc;
  Workspace w;
  carve_workspace(p, base, &w);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_noalloc_offsets<<<1, 1, 0, s>>>(w.offsets, n);
  g_launches += 1;
  return run_solver(p, w, w.offsets, d, e, lambda, s);
}

extern "C" int tde_noalloc_get_info(void* stream, int32_t* info) {
  using namespace tde;
  if (info == nullptr) return TDE_EINVAL;
  void* base = nullptr;
  const int rc = noalloc_scratch(&base);
  if (rc != TDE_OK) return rc;
  // the Status record opens the workspace carved from the array (carve_workspace)
  return tde_get_info(base, stream, info);
}
