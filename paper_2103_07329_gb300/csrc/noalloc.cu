// noalloc.cu -- column dot products without any device allocation.
//
// xamg_coldot allocates a small device buffer for its per-block partial sums
// on every call.  Some callers cannot allow that: a host framework that has
// already reserved the whole device memory for its own pool (cudaMalloc then
// fails), or a latency-critical loop in which a call into the CUDA allocator
// (which may synchronize the device) is not acceptable.  xamg_coldot_noalloc
// runs the same two kernels as xamg_coldot but keeps the partial sums in a
// fixed array that is part of this library's device image.
//
// The array is file-scope device memory: every GPU that loads the library
// keeps it (256 KiB) until the process exits.  Host code may not use the
// array's name as a device address -- in host code it names a host-side
// stand-in -- so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and handed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/xamg_gpu.h"
#include "launch.h"

namespace {

constexpr int kScratchBlocks = 1024;  // partial sums of at most 1024 blocks ...
constexpr int kScratchCols = XAMG_MAX_RHS;  // ... times 32 columns
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_coldot_scratch[kScratchBlocks * kScratchCols];

std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of g_coldot_scratch on the current device, looked up on the
// first call for that device.
int scratch_on_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XAMG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return XAMG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_coldot_scratch) != cudaSuccess || !p) return XAMG_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return XAMG_OK;
}

}  // namespace

extern "C" int xamg_coldot_noalloc(const double *U, const double *V, int64_t n, int32_t m,
                                   double *out, void *stream) {
  if (!U || !V || !out || n < 0) return XAMG_ERR_INVALID_ARG;
  if (m < 1 || m > kScratchCols) return XAMG_ERR_INVALID_ARG;  // the array holds 32 columns
  const int grid = std::min(xamg::coldot_rt_grid(n, m), kScratchBlocks);
  if ((int64_t)grid * m > (int64_t)kScratchBlocks * kScratchCols) return XAMG_ERR_INVALID_ARG;
  double *part = nullptr;
  const int rc = scratch_on_current_device(&part);
  if (rc != XAMG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every slot the reduction reads is written by the first kernel of this
  // call, so nothing in the array has to be cleared beforehand.
  xamg::launch_coldot_rt(n, m, U, V, part, grid, st);
  xamg::launch_reduce_rt(m, part, grid, out, st);
  if (cudaGetLastError() != cudaSuccess) return XAMG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return XAMG_ERR_CUDA;
  return XAMG_OK;
}
