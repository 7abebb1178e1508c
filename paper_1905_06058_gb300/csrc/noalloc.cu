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
// memory), so each device's address is looked up once with
// cudaGetSymbolAddress, with that device current, on the first call made on
// it; make that first call before any stream capture.  All calls share the
// array: calls whose kernels overlap on the GPU (different streams, or
// different host threads on one stream) race on it and must be serialised by
// the caller.  Every slot a call reads is written earlier in the same call,
// so nothing has to be cleared between calls.
#include <mutex>

#include "isam.h"
#include "internal.cuh"

namespace {

__device__ __align__(256) double g_noalloc_partial[ISAM_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
constexpr int kElemsPerPartial = 256 * 8;   // elements reduced into one partial

std::mutex g_setup_mutex;
double* g_partial_dev[kMaxDevices] = {nullptr};

// Device address of the static array on the current device (set up once).
isam_status partial_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ISAM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) return ISAM_ERR_CUDA;
    g_partial_dev[dev] = static_cast<double*>(p);
  }
  *out = g_partial_dev[dev];
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
