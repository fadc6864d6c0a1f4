// clbm_residual_fields_noalloc: the steady-state residual of clbm_residual,
// computed from caller-owned macroscopic fields without any allocation.
//
// Why it exists: some callers cannot call cudaMalloc/cudaFree at all or at the
// moment they need the residual -- applications that hand all device memory
// to their own pool allocator up front, host frameworks that embed this
// library and forbid foreign allocations, and time-critical loops that cannot
// afford the implicit device synchronisation cudaFree brings.  Such callers
// pass their own input fields and output pointer; the per-block partial sums
// the reduction needs live in a fixed file-scope device array instead of
// memory obtained at run time.
//
// The scratch array is `g_noalloc_scratch` below: kNoAllocMaxBlocks blocks x 8
// partial sums + 8 result slots, 256-byte aligned, 65,600 bytes.  Every GPU
// that loads this library holds it until the process exits.  Host code cannot
// use the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks its device address up
// with cudaGetSymbolAddress while that device is current and caches it.  All
// calls share the array: calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race on it and must be
// serialised by the caller.  Each call rewrites every slot it later reads
// (each block stores its own partials, the final pass stores the result), so
// no slot has to start at zero and leftovers of an earlier call are never read.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/clbm.h"
#include "clbm_internal.h"
#include "clbm_kernels.cuh"

namespace clbm {
namespace {

constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocWidth = 8;
constexpr long long kNoAllocMaxNodes = 1LL << 31;  // same lattice limit as clbm_create
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * kNoAllocWidth + kNoAllocWidth];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Residual partial sums from two snapshots of (T, ux, uy): the same quantities
// as residual_kernel, read from dense FP64 arrays instead of distribution planes.
__global__ void __launch_bounds__(kRedThreads)
    residual_fields_kernel(const double* __restrict__ T1, const double* __restrict__ u1,
                           const double* __restrict__ v1, const double* __restrict__ T0,
                           const double* __restrict__ u0, const double* __restrict__ v0,
                           const uint8_t* __restrict__ solid, long long n,
                           double* __restrict__ partials) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (solid && solid[k]) continue;
    const double t1 = T1[k], a1 = u1[k], b1 = v1[k];
    const double t0 = T0[k], a0 = u0[k], b0 = v0[k];
    acc[0] += (t1 - t0) * (t1 - t0);
    acc[1] += t1 * t1;
    acc[2] += (a1 - a0) * (a1 - a0);
    acc[3] += a1 * a1;
    acc[4] += (b1 - b0) * (b1 - b0);
    acc[5] += b1 * b1;
    if (!isfinite(t1) || !isfinite(a1) || !isfinite(b1)) acc[6] += 1.0;
  }
  block_sum_store<8>(acc, partials + kNoAllocWidth * blockIdx.x);
}

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace clbm

extern "C" clbm_status clbm_residual_fields_noalloc(const double* T_now, const double* ux_now,
                                                    const double* uy_now, const double* T_prev,
                                                    const double* ux_prev, const double* uy_prev,
                                                    const uint8_t* solid, int64_t n, void* stream,
                                                    double* r_out) {
  using namespace clbm;
  if (!T_now || !ux_now || !uy_now || !T_prev || !ux_prev || !uy_prev || !r_out)
    return CLBM_EINVAL;
  if (n < 1 || n > kNoAllocMaxNodes) return CLBM_EINVAL;  // beyond the supported lattice size
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the scratch address is the current device's: the stream must belong to it
  int cur_dev = 0, stream_dev = 0;
  if (cudaGetDevice(&cur_dev) != cudaSuccess) return CLBM_ECUDA;
  if (cudaStreamGetDevice(s, &stream_dev) != cudaSuccess) return CLBM_EINVAL;
  if (stream_dev != cur_dev) return CLBM_EINVAL;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return CLBM_ECUDA;
  long long b = (n + kRedThreads - 1) / kRedThreads;
  const int nblocks = (int)(b < kNoAllocMaxBlocks ? b : kNoAllocMaxBlocks);
  double* result = scratch + kNoAllocMaxBlocks * kNoAllocWidth;
  residual_fields_kernel<<<nblocks, kRedThreads, 0, s>>>(T_now, ux_now, uy_now, T_prev, ux_prev,
                                                          uy_prev, solid, (long long)n, scratch);
  if (cudaGetLastError() != cudaSuccess) return CLBM_ECUDA;
  if (launch_reduce_partials(scratch, nblocks, kNoAllocWidth, result, s) != cudaSuccess)
    return CLBM_ECUDA;
  double h[kNoAllocWidth];
  if (cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CLBM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CLBM_ECUDA;
  if (h[6] != 0.0 || !std::isfinite(h[0] + h[1] + h[2] + h[3] + h[4] + h[5])) {
    *r_out = INFINITY;
    return CLBM_EUNSTABLE;
  }
  double best = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double den = std::sqrt(h[2 * k + 1]) > 1e-30 ? std::sqrt(h[2 * k + 1]) : 1e-30;
    const double v = std::sqrt(h[2 * k]) / den;
    best = v > best ? v : best;
  }
  *r_out = best;
  return CLBM_OK;
}
