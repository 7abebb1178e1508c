// Allocation-free max |x_i| reduction (the lambda scale ||A^H s||_inf of the
// solve), for callers that must not allocate device memory: a host thread that
// is recording a CUDA stream capture owned by another framework (a cudaMalloc
// there breaks or serialises the capture), an acquisition loop that fixed its
// memory budget at start-up and cannot absorb the latency or fragmentation of
// a new allocation, or code whose device memory is entirely held by a pooling
// allocator such as PyTorch's, where an extra cudaMalloc can fail even though
// the pool has room.
//
// The per-block partial maxima live in one file-scope device array of
// ISAM_NOALLOC_MAX_PARTIALS doubles (512 KiB), which every GPU that loads the
// library keeps until the process exits.  Host code cannot pass the array's
// name to a kernel (in host code it names a host-side stand-in, not device
// memory), so each device's address is looked up with cudaGetSymbolAddress,
// with that device current, on the first call made on it; make that first
// call before any stream capture.  The address belongs to the device's CUDA
// context: after cudaDeviceReset the module is loaded again into a new
// primary context, possibly elsewhere, so the cache is keyed on the context's
// unique ID and a call in a new context looks the address up again (that call,
// too, must come before any capture).  All calls share the array: calls whose
// kernels overlap on the GPU (different streams, or different host threads on
// one stream) race on it and must be serialised by the caller.  Every slot a
// call reads is written earlier in the same call, so nothing has to be
// cleared between calls.
#include <cuda.h>

#include <mutex>

#include "isam.h"
#include "internal.cuh"

namespace {

__device__ __align__(256) double g_noalloc_partial[ISAM_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
constexpr int kElemsPerPartial = 256 * 8;   // elements reduced into one partial

struct DeviceEntry {
  unsigned long long ctx_id = 0;   // context the address was looked up in
  double* ptr = nullptr;
};

std::mutex g_setup_mutex;
DeviceEntry g_partial_dev[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context (driver entry points
// found through the runtime, so nothing extra is linked); false when there is
// no current context or the driver lacks the call.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    looked_up = true;
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the static array in the current device's context: looked
// up on the first call in that context (without a context ID, on every call).
isam_status partial_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISAM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceEntry& e = g_partial_dev[dev];
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (!e.ptr || !have_id || e.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) return ISAM_ERR_CUDA;
    // the lookup creates the context when there was none yet: take its ID now
    unsigned long long id_after = 0;
    e.ctx_id = current_context_id(&id_after) ? id_after : 0;
    e.ptr = static_cast<double*>(p);
  }
  *out = e.ptr;
  return ISAM_OK;
}

}  // namespace

extern "C" isam_status isam_max_abs_noalloc(const void* x, int64_t n, int32_t precision,
                                            double* out, void* stream) {
  if (!x || !out || n < 1) return ISAM_ERR_INVALID;
  if (precision != ISAM_FP32 && precision != ISAM_FP64) return ISAM_ERR_INVALID;
  const int64_t nparts = (n + kElemsPerPartial - 1) / kElemsPerPartial;
  if (nparts > ISAM_NOALLOC_MAX_PARTIALS) return ISAM_ERR_UNSUPPORTED;
  double* partial = nullptr;
  const isam_status st = partial_address(&partial);
  if (st != ISAM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (precision == ISAM_FP64)
    e = isam::launch_max_abs<double>(static_cast<const double2*>(x), size_t(n), partial,
                                     int(nparts), out, s);
  else
    e = isam::launch_max_abs<float>(static_cast<const float2*>(x), size_t(n), partial,
                                    int(nparts), out, s);
  return e == cudaSuccess ? ISAM_OK : ISAM_ERR_CUDA;
}
