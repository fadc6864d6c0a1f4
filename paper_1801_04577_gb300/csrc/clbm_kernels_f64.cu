// FP64 storage and FP64 collision, plus the fixed-order partial-sum reduction.
#include "clbm_kernels.cuh"

namespace clbm {

const Launchers kLaunchF64 = LaunchImpl<double>::table();

// One block adds nblocks rows of `width` partials in index order, so a
// reduction gives the same bits on every run.
__global__ void __launch_bounds__(kRedThreads)
    reduce_partials_kernel(const double* __restrict__ partials, int nblocks, int width,
                           double* __restrict__ out) {
  for (int k = 0; k < width; ++k) {
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc[0] += partials[(long long)b * width + k];
    __shared__ double tmp[1];
    block_sum_store<1>(acc, tmp);
    __syncthreads();
    if (threadIdx.x == 0) out[k] = tmp[0];
    __syncthreads();
  }
}

__global__ void advance_kernel(long long* t, int k) { *t += k; }
__global__ void set_kernel(long long* t, long long v) { *t = v; }

cudaError_t launch_set_step(long long* t, long long v, cudaStream_t s) {
  set_kernel<<<1, 1, 0, s>>>(t, v);
  return cudaGetLastError();
}

cudaError_t launch_advance(long long* t, int k, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(t, k);
  return cudaGetLastError();
}

// All halo rows of an exchange in one launch: blockIdx.y = copy, 16-byte words.
__global__ void halo_kernel(const HaloTable t) {
  const HaloCopy h = t.c[blockIdx.y];
  const long long words = t.row_bytes / 16;
  const long long total = words * t.planes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / words, w = i - q * words;
    *reinterpret_cast<uint4*>(h.dst + q * h.dplane + 16 * w) =
        *reinterpret_cast<const uint4*>(h.src + q * h.splane + 16 * w);
  }
}

cudaError_t launch_halo(const HaloTable& t, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  const long long total = t.row_bytes / 16 * t.planes;
  const int bx = (int)std::min<long long>((total + 255) / 256, 1024);
  halo_kernel<<<dim3(bx, t.n), 256, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int nblocks, int width, double* out,
                                   cudaStream_t s) {
  reduce_partials_kernel<<<1, kRedThreads, 0, s>>>(partials, nblocks, width, out);
  return cudaGetLastError();
}

}  // namespace clbm
