// Surrogate network for warm starts: a small convolutional encoder-decoder
// (U-Net) mapping problem descriptors on a G x G grid to steady T, ux, uy,
// trained and evaluated entirely by the kernels in this file.
//
// Layers (L levels, base width B, widths c_l = B 2^l):
//   encoder l = 0..L-2 : conv3x3 + ReLU, conv3x3 + ReLU (= skip_l), 2x2 average pool
//   bottleneck L-1     : conv3x3 + ReLU, conv3x3 + ReLU
//   decoder l = L-2..0 : nearest 2x upsample, concat [up, skip_l], conv3x3 + ReLU, conv3x3 + ReLU
//   head               : conv1x1 (no activation)
// Activations are FP32 NCHW; weights are kept as an FP32 master copy (Adam)
// and a BF16 copy that every convolution reads; accumulation is FP32.
//
// Every convolution pass is one implicit GEMM with on-the-fly im2col loaders,
// run either on the tensor cores (tc::gemm_kernel in clbm_tc.cuh: both
// operands rounded to BF16 as they are staged in shared memory, tcgen05.mma,
// FP32 accumulator in TMEM; the default) or on the FP32 CUDA cores
// (gemm_kernel below: FP32 activations, BF16 weights):
//   forward      Y[co, p]      = sum_{ci,t} W[co, ci t] X[ci, p + t]
//   input grad   dX[ci, p]    += sum_{co,t} W'[ci, co t] dY[co, p + t]   (W' = W flipped, transposed)
//   weight grad  dW[co, ci t]  = sum_p dY[co, p] X[ci, p + t]          (split-K over pixels,
//                                                                       partials summed in order)
// so the training step is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_tc.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

// ---------------------------------------------------------------------------
// Loaders (element (m, k) of A, (k, n) of B) and stores for the GEMM
// ---------------------------------------------------------------------------
struct Act {  // one activation tensor view: sample n, channel c at base + n*cs*HW + (coff + c)*HW
  const float* base;
  int cs, coff, C, H, W;
  __device__ __forceinline__ float at(int n, int c, int y, int x) const {
    if (y < 0 || y >= H || x < 0 || x >= W) return 0.0f;
    return base[((long long)n * cs + coff + c) * H * W + (long long)y * W + x];
  }
};

// A(m, k) = weights[m][k] (BF16, row-major M x K)
struct LoadW {
  const __nv_bfloat16* w;
  int K;
  __device__ __forceinline__ float operator()(int m, int k) const {
    return __bfloat162float(w[(long long)m * K + k]);
  }
};

// B(k, n) = im2col(X): k = (c, tap), n = pixel (sample, y, x); ks = 1 or 3
struct LoadIm2col {
  Act x;
  int ks;
  __device__ __forceinline__ float operator()(int k, int n) const {
    const int hw = x.H * x.W;
    const int t = k % (ks * ks), c = k / (ks * ks);
    const int nb = n / hw, p = n - nb * hw;
    const int y = p / x.W, xx = p - y * x.W;
    const int r = ks / 2;
    return x.at(nb, c, y + t / ks - r, xx + t % ks - r);
  }
};

// A(m, k) = act[sample][m][pixel]: m = channel, k = pixel (for weight gradients)
struct LoadActMK {
  Act a;
  __device__ __forceinline__ float operator()(int m, int k) const {
    const int hw = a.H * a.W;
    const int nb = k / hw, p = k - nb * hw;
    return a.base[((long long)nb * a.cs + a.coff + m) * hw + p];
  }
};

// B(k, n) = im2col(X) transposed: k = pixel, n = (c, tap)
struct LoadIm2colT {
  Act x;
  int ks;
  __device__ __forceinline__ float operator()(int k, int n) const {
    const int hw = x.H * x.W;
    const int t = n % (ks * ks), c = n / (ks * ks);
    const int nb = k / hw, p = k - nb * hw;
    const int y = p / x.W, xx = p - y * x.W;
    const int r = ks / 2;
    return x.at(nb, c, y + t / ks - r, xx + t % ks - r);
  }
};

// C(m = channel, n = pixel) into an activation view, with bias / ReLU / accumulate.
struct StoreAct {
  float* base;
  int cs, coff, H, W;
  const float* bias;
  int relu, accumulate;
  // ReLU backward of the accumulated gradient: zero where the forward
  // activation (same layout as base) is not positive; nullptr = none
  const float* relu_of = nullptr;
  __device__ __forceinline__ void operator()(int m, int n, float v) const {
    const int hw = H * W;
    const int nb = n / hw, p = n - nb * hw;
    const long long off = ((long long)nb * cs + coff + m) * hw + p;
    float* dst = base + off;
    if (bias) v += bias[m];
    if (relu) v = v > 0.0f ? v : 0.0f;
    if (accumulate) v += *dst;
    if (relu_of && !(relu_of[off] > 0.0f)) v = 0.0f;
    *dst = v;
  }
};

// C(m, n) into a dense partial buffer: part[split][m][n]
struct StorePartial {
  float* part;
  int M, N;
  __device__ __forceinline__ void operator()(int m, int n, float v, int split) const {
    part[((long long)split * M + m) * N + n] = v;
  }
};

// ---------------------------------------------------------------------------
// Operands of the tensor-core GEMM (rows m of D are TMEM lanes): the
// convolutions put pixels on m for the forward and input-gradient passes, and
// (channel, tap) pairs on m for the weight gradient.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put_chunk(uint8_t* dst, int r, int kc, const float (&v)[8]) {
  *reinterpret_cast<uint4*>(dst + tc::chunk_off(r, kc)) =
      make_uint4(tc::pack_bf16(v[0], v[1]), tc::pack_bf16(v[2], v[3]), tc::pack_bf16(v[4], v[5]),
                 tc::pack_bf16(v[6], v[7]));
}

// A(m = pixel, k = tap * C + channel) = x[channel] at pixel + tap offset
// (zero outside the image; tap-major K, the order of the packed weights).
// Thread r gathers row r, so every load of a warp reads 32 consecutive
// pixels.  With C a multiple of 8 every 16-byte chunk holds one tap and eight
// channels: one offset and one bounds test per chunk.
template <int KS>
struct GatherIm2col {
  static constexpr bool kBulk = false;
  Act x;
  __device__ __forceinline__ void operator()(uint8_t* dst, int row0, int rows_valid, int, int k0,
                                             int kend) const {
    constexpr int KK = KS * KS, R = KS / 2;
    const int r = threadIdx.x;
    const int hw = x.H * x.W, C = x.C;
    const bool rv = r < rows_valid;
    int nb = 0, p = 0, yy = 0, xx = 0;
    if (rv) {
      const int m = row0 + r;
      nb = m / hw;
      p = m - nb * hw;
      yy = p / x.W;
      xx = p - yy * x.W;
    }
    const float* src = x.base + ((long long)nb * x.cs + x.coff) * hw + p;
    uint32_t vm = 0;  // taps inside the image
#pragma unroll
    for (int t = 0; t < KK; ++t) {
      const int sy = yy + t / KS - R, sx = xx + t % KS - R;
      if (rv && sy >= 0 && sy < x.H && sx >= 0 && sx < x.W) vm |= 1u << t;
    }
    if ((C & 7) == 0) {
      // all 64 loads of the slice are issued before any is packed (the gather
      // is bound by load latency, not by issue)
      int t = k0 / C, c = k0 - t * C;
      float v[tc::kBK / 8][8];
#pragma unroll
      for (int kc = 0; kc < tc::kBK / 8; ++kc) {
        const bool ok = k0 + kc * 8 < kend && ((vm >> t) & 1u);
        const float* s = src + c * hw + (t / KS - R) * x.W + (t % KS - R);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[kc][e] = ok ? __ldg(s + e * hw) : 0.0f;
        c += 8;
        if (c == C) {
          c = 0;
          ++t;
        }
      }
#pragma unroll
      for (int kc = 0; kc < tc::kBK / 8; ++kc) put_chunk(dst, r, kc, v[kc]);
    } else {  // channels not a multiple of 8: walk (tap, channel) element by element
      int t = k0 / C, c = k0 - t * C;
      int off = (t / KS - R) * x.W + (t % KS - R);
#pragma unroll 2
      for (int kc = 0; kc < tc::kBK / 8; ++kc) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const bool ok = k0 + kc * 8 + e < kend && ((vm >> t) & 1u);
          v[e] = ok ? __ldg(src + c * hw + off) : 0.0f;
          if (++c == C) {
            c = 0;
            ++t;
            off = (t / KS - R) * x.W + (t % KS - R);
          }
        }
        put_chunk(dst, r, kc, v);
      }
    }
  }
};

// A(m = (channel, tap), k = pixel) = x[channel] at pixel + tap offset: eight
// consecutive threads gather the 64 pixels of one row, 8 each.
template <int KS>
struct GatherIm2colT {
  static constexpr bool kBulk = false;
  Act x;
  __device__ __forceinline__ void operator()(uint8_t* dst, int row0, int rows_valid, int, int k0,
                                             int kend) const {
    constexpr int KK = KS * KS, R = KS / 2;
    constexpr int kGroup = 4;  // tasks whose loads are in flight together
    static_assert((tc::kBM * 8) % (kGroup * tc::kThreads) == 0, "whole groups of tasks");
    static_assert(tc::kThreads % 8 == 0, "a thread keeps its pixel chunk across tasks");
    const int hw = x.H * x.W;
    // every task of this thread covers the same 8 pixels k .. k + 7 (task & 7 is
    // threadIdx.x & 7); with W a multiple of 8 they lie in one image row
    const int k = k0 + (threadIdx.x & 7) * 8;
    const int nb = k / hw, p = k - nb * hw;
    const int yy = p / x.W, xx = p - yy * x.W;
    const bool row8 = (x.W & 7) == 0 && k + 8 <= kend;
    for (int task0 = threadIdx.x; task0 < tc::kBM * 8; task0 += kGroup * tc::kThreads) {
      float v[kGroup][8];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int task = task0 + u * tc::kThreads;
        const int r = task >> 3;
        const int row = row0 + r;
        const int c = row / KK, t = row - c * KK;
        const int dy = t / KS - R, dx = t % KS - R;
        if (row8) {
          // one row segment: the row test once, the columns as the range [lo, hi) of e
          const int sy = yy + dy, sx0 = xx + dx;
          const bool ok = r < rows_valid && sy >= 0 && sy < x.H;
          const int lo = sx0 < 0 ? -sx0 : 0, hi = min(8, x.W - sx0);
          const float* src = x.base + ((long long)nb * x.cs + x.coff + c) * hw + (long long)sy * x.W + sx0;
#pragma unroll
          for (int e = 0; e < 8; ++e) v[u][e] = (ok && e >= lo && e < hi) ? __ldg(src + e) : 0.0f;
        } else {  // pixels may cross rows or samples: element by element
          int nb1 = nb, yy1 = yy, xx1 = xx;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int sy = yy1 + dy, sx = xx1 + dx;
            const bool ok = r < rows_valid && k + e < kend && sy >= 0 && sy < x.H && sx >= 0 && sx < x.W;
            v[u][e] = ok ? __ldg(x.base + ((long long)nb1 * x.cs + x.coff + c) * hw + sy * x.W + sx) : 0.0f;
            if (++xx1 == x.W) {
              xx1 = 0;
              if (++yy1 == x.H) {
                yy1 = 0;
                ++nb1;
              }
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int task = task0 + u * tc::kThreads;
        put_chunk(dst, task >> 3, task & 7, v[u]);
      }
    }
  }
};

// B(n = channel, k = pixel) = g[channel][pixel] of an activation(-gradient)
// view: eight consecutive threads read one row's 64 pixels (two float4 each
// when a sample's pixel count is a multiple of 8).
struct GatherRows {
  static constexpr bool kBulk = false;
  Act a;
  __device__ __forceinline__ void operator()(uint8_t* dst, int row0, int rows_valid, int nrows, int k0,
                                             int kend) const {
    const int hw = a.H * a.W;
    const bool vec = (hw & 7) == 0;
    constexpr int kGroup = 4;  // tasks whose loads are in flight together
    const int ntask = nrows * 8;
    for (int task0 = threadIdx.x; task0 < ntask; task0 += kGroup * tc::kThreads) {
      float v[kGroup][8];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int task = task0 + u * tc::kThreads;
        const int r = task >> 3, kc = task & 7;
        const int k = k0 + kc * 8;
        const long long ch = a.coff + row0 + r;
        if (task < ntask && r < rows_valid && vec && k + 8 <= kend) {
          const int nb = k / hw, p = k - nb * hw;
          const float4* s4 = reinterpret_cast<const float4*>(a.base + ((long long)nb * a.cs + ch) * hw + p);
          const float4 u0 = __ldg(s4), u1 = __ldg(s4 + 1);
          v[u][0] = u0.x; v[u][1] = u0.y; v[u][2] = u0.z; v[u][3] = u0.w;
          v[u][4] = u1.x; v[u][5] = u1.y; v[u][6] = u1.z; v[u][7] = u1.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int kk = k + e;
            const int nb = kk / hw, p = kk - nb * hw;
            v[u][e] = (task < ntask && r < rows_valid && kk < kend)
                          ? __ldg(a.base + ((long long)nb * a.cs + ch) * hw + p)
                          : 0.0f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int task = task0 + u * tc::kThreads;
        if (task < ntask) put_chunk(dst, task >> 3, task & 7, v[u]);
      }
    }
  }
};

struct TStoreAct {  // D(m = pixel, n = channel)
  StoreAct s;
  __device__ __forceinline__ void operator()(int m, int n, float v, int) const { s(n, m, v); }
};
struct TStoreSplit {  // D(m = pixel, n = channel) of split z -> part[z][n][m]
  float* part;
  int M, N;
  __device__ __forceinline__ void operator()(int m, int n, float v, int z) const {
    part[((long long)z * N + n) * M + m] = v;
  }
};
struct TStorePartial {  // D(m = (ci, tap), n = co) of split z
  StorePartial s;
  __device__ __forceinline__ void operator()(int m, int n, float v, int z) const { s(n, m, v, z); }
};

// Pre-packed BF16 weights for the tensor-core GEMMs (tc::Packed layout), one
// entry per layer and direction, K tap-major: forward B(n = co, k = tap * ci
// + c) = W[co][c][tap], input gradient B(n = ci, k = tap' * co + o) =
// W[o][ci][taps - 1 - tap'] (taps flipped).
struct PackDesc {
  long long w_off;    // layer weights in the parameter vector
  long long dst_off;  // first element of this layer's packed buffer
  int co, ci, kk;     // output / input channels, taps
  int transpose;      // 0: forward, 1: input gradient
  int N, K, bn, slices;
  long long size;     // packed elements (N tiles x slices x bn x 64)
};

__global__ void pack_weights_kernel(const PackDesc* __restrict__ descs, const __nv_bfloat16* __restrict__ w,
                                    __nv_bfloat16* __restrict__ out) {
  const PackDesc d = descs[blockIdx.y];
  const long long tile_e = (long long)d.bn * tc::kBK;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.size;
       i += (long long)gridDim.x * blockDim.x) {
    const long long tile = i / tile_e;
    const int within = (int)(i - tile * tile_e);
    const int nt = (int)(tile / d.slices), ks = (int)(tile - (long long)nt * d.slices);
    // inverse of chunk_off: 512 elements per 8-row group, 64 per K chunk, 8 per row
    const int rg = within >> 9, kc = (within >> 6) & 7, r7 = (within >> 3) & 7, e = within & 7;
    const int n = nt * d.bn + rg * 8 + r7, k = ks * tc::kBK + kc * 8 + e;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    if (n < d.N && k < d.K) {
      if (!d.transpose) {  // n = co, k = t * ci + c
        const int t = k / d.ci, c = k - t * d.ci;
        v = w[d.w_off + ((long long)n * d.ci + c) * d.kk + t];
      } else {  // n = ci, k = t' * co + o
        const int tp = k / d.co, o = k - tp * d.co;
        v = w[d.w_off + ((long long)o * d.ci + n) * d.kk + (d.kk - 1 - tp)];
      }
    }
    out[d.dst_off + i] = v;
  }
}

// ---------------------------------------------------------------------------
// Tiled FP32 GEMM: 64 x 64 output tile per block, 4 x 4 per thread, K in
// chunks of 16 staged in shared memory.  blockIdx.z = K split.
// ---------------------------------------------------------------------------
template <class LA, class LB, class ST>
__global__ void __launch_bounds__(GT) gemm_kernel(LA la, LB lb, ST st, int M, int N, int K,
                                                  int kper) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kper;
  const int kend = min(K, kbeg + kper);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BK * BM) / GT; ++r) {
      const int e = tid + r * GT;
      const int kk = e / BM, mm = e % BM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < kend) ? la(m, k) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < (BK * BN) / GT; ++r) {
      const int e = tid + r * GT;
      const int kk = e / BN, nn = e % BN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < kend) ? lb(k, n) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) {
        if constexpr (std::is_same<ST, StorePartial>::value)
          st(m, n, acc[i][j], blockIdx.z);
        else
          st(m, n, acc[i][j]);
      }
    }
}

// Split-K forward / input-gradient GEMMs: D(pixel m, channel n) = sum over
// splits of part[z][n][m] in order, then bias / ReLU / accumulation as the
// unsplit epilogue would apply them.
__global__ void splitk_finish_kernel(const float* __restrict__ part, int splits, int M, int N, StoreAct st) {
  for (int n = blockIdx.y; n < N; n += gridDim.y)
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
      float v = 0.0f;
      for (int z = 0; z < splits; ++z) v += part[((long long)z * N + n) * M + m];
      st(n, m, v);
    }
}

// out[i] = sum_s part[s][i] in a fixed order. Block (32 x R) owns 32 outputs;
// thread row r adds splits r, r + R, ... in turn, then the R row sums are
// combined by a fixed pairwise tree, so many loads are in flight even when
// there are few outputs and many splits.
constexpr int kSumRows = 32;
__global__ void sum_splits_kernel(const float* __restrict__ part, int splits, long long n,
                                  float* __restrict__ out) {
  __shared__ float sh[kSumRows][33];
  const int R = blockDim.y, r = threadIdx.y, l = threadIdx.x;
  for (long long i0 = (long long)blockIdx.x * 32; i0 < n; i0 += (long long)gridDim.x * 32) {
    const long long i = i0 + l;
    float s = 0.0f;
    if (i < n)
      for (int k = r; k < splits; k += R) s += part[(long long)k * n + i];
    sh[r][l] = s;
    __syncthreads();
    for (int o = R / 2; o > 0; o >>= 1) {
      if (r < o) sh[r][l] += sh[r + o][l];
      __syncthreads();
    }
    if (r == 0 && i < n) out[i] = sh[0][l];
    __syncthreads();
  }
}

// launch shape of sum_splits_kernel: R = largest power of two <= min(splits, 32)
// and <= the rows that keep about one GPU's worth of threads (sms x 2048) busy:
// many outputs take few rows, each thread then adding more splits in turn (the
// tree of 32 rows had made the widest sums latency-bound: 51 us for 249 k
// outputs).
void sum_splits(const float* part, int splits, long long n, float* out, int sms, cudaStream_t s) {
  const long long want = std::max<long long>(1, (sms * 2048LL) / std::max<long long>(n, 1));
  int R = 1;
  while (2 * R <= std::min(splits, kSumRows) && 2 * R <= want) R *= 2;
  const long long blocks = std::min<long long>((n + 31) / 32, 65535);
  sum_splits_kernel<<<(unsigned)std::max<long long>(blocks, 1), dim3(32, R), 0, s>>>(part, splits, n, out);
}

// Bias gradient db[c] = sum over samples and pixels of g[n][c][p], in two
// deterministic stages: block (s, c) sums chunk s of channel c's values
// (sample-major) into part[s][c]; sum_splits_kernel then adds the chunks in
// order.
constexpr int kBiasChunk = 4096;

__global__ void bias_partial_kernel(Act g, int N, float* __restrict__ part) {
  __shared__ float sh[GT];
  const int s = blockIdx.x, c = blockIdx.y;
  const int hw = g.H * g.W;
  const int tot = N * hw;  // below 2^31 (checked at network creation)
  const int k0 = s * kBiasChunk, k1 = min(tot, k0 + kBiasChunk);
  float acc = 0.0f;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int nb = k / hw, p = k - nb * hw;
    acc += g.base[((long long)nb * g.cs + g.coff + c) * hw + p];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = GT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)s * gridDim.y + c] = sh[0];
}

// Element-wise kernels over activation views, launched on a 2-D grid: blockIdx.y
// walks the (sample, channel) planes, blockIdx.x / threadIdx.x the pixels of
// a plane, so the only index division is one per plane (plane_grid).
dim3 plane_grid(int pixels, long long planes) {
  const int bx = std::max(1, std::min((pixels + 255) / 256, 64));
  return dim3((unsigned)bx, (unsigned)std::max<long long>(1, std::min<long long>(planes, 65535)));
}

// 2x2 average pool: out (H/2 x W/2) from in; backward adds g_out/4 to the four inputs
__global__ void pool_kernel(Act in, float* __restrict__ out, int ocs, int ocoff, int N) {
  const int Wo = in.W / 2, ho = (in.H / 2) * Wo, hw = in.H * in.W;
  for (int pc = blockIdx.y; pc < N * in.C; pc += gridDim.y) {
    const int nb = pc / in.C, c = pc - nb * in.C;
    const float* ip = in.base + ((long long)nb * in.cs + in.coff + c) * hw;
    float* op = out + ((long long)nb * ocs + ocoff + c) * ho;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ho; p += gridDim.x * blockDim.x) {
      const int y = p / Wo, x = p - y * Wo;
      const float* q = ip + 2 * y * in.W + 2 * x;
      op[p] = 0.25f * ((q[0] + q[1]) + (q[in.W] + q[in.W + 1]));
    }
  }
}
// relu_of (same layout as gin, or nullptr): the ReLU backward of the
// accumulated gradient, zero where that forward activation is not positive
__global__ void pool_back_kernel(Act gout, float* __restrict__ gin, int gcs, int gcoff, int N,
                                 const float* __restrict__ relu_of) {
  const int W = gout.W * 2, hw = gout.H * 2 * W, ho = gout.H * gout.W;
  for (int pc = blockIdx.y; pc < N * gout.C; pc += gridDim.y) {
    const int nb = pc / gout.C, c = pc - nb * gout.C;
    const float* gp = gout.base + ((long long)nb * gout.cs + gout.coff + c) * ho;
    const long long base = ((long long)nb * gcs + gcoff + c) * hw;
    float* ip = gin + base;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x) {
      const int y = p / W, x = p - y * W;
      float v = ip[p] + 0.25f * gp[(y >> 1) * gout.W + (x >> 1)];
      if (relu_of && !(relu_of[base + p] > 0.0f)) v = 0.0f;
      ip[p] = v;
    }
  }
}

// nearest 2x upsample; backward sums the four outputs of each input
__global__ void up_kernel(Act in, float* __restrict__ out, int ocs, int ocoff, int N) {
  const int W = in.W * 2, hw = in.H * 2 * W, hi = in.H * in.W;
  for (int pc = blockIdx.y; pc < N * in.C; pc += gridDim.y) {
    const int nb = pc / in.C, c = pc - nb * in.C;
    const float* ip = in.base + ((long long)nb * in.cs + in.coff + c) * hi;
    float* op = out + ((long long)nb * ocs + ocoff + c) * hw;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x) {
      const int y = p / W, x = p - y * W;
      op[p] = ip[(y >> 1) * in.W + (x >> 1)];
    }
  }
}
__global__ void up_back_kernel(Act gout, float* __restrict__ gin, int gcs, int gcoff, int N,
                               const float* __restrict__ relu_of) {
  const int Wi = gout.W / 2, hi = (gout.H / 2) * Wi, hw = gout.H * gout.W;
  for (int pc = blockIdx.y; pc < N * gout.C; pc += gridDim.y) {
    const int nb = pc / gout.C, c = pc - nb * gout.C;
    const float* gp = gout.base + ((long long)nb * gout.cs + gout.coff + c) * hw;
    const long long base = ((long long)nb * gcs + gcoff + c) * hi;
    float* ip = gin + base;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x) {
      const int y = p / Wi, x = p - y * Wi;
      const float* q = gp + 2 * y * gout.W + 2 * x;
      float v = ip[p] + ((q[0] + q[1]) + (q[gout.W] + q[gout.W + 1]));
      if (relu_of && !(relu_of[base + p] > 0.0f)) v = 0.0f;
      ip[p] = v;
    }
  }
}

// masked MSE: loss = sum mask (y - t)^2 / (sum mask * C); g = dloss/dy.  One block
// per sample writes FP64 partials (fixed order), summed on the host.
// Loss chunks per sample (blockIdx.y of the mask and loss kernels).
constexpr int kLossChunks = 16;

// Block sum of a double in fixed order (GT threads).
__device__ double block_sum_fixed(double s) {
  __shared__ double sh[GT];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = GT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Mask weight sum of each sample: part[nb] = sum of mask over sample nb's pixels.
__global__ void mask_sum_kernel(const float* __restrict__ mask, int HW, double* __restrict__ part) {
  const int nb = blockIdx.x;
  double s = 0.0;
  for (int p = threadIdx.x; p < HW; p += blockDim.x) s += mask[(long long)nb * HW + p];
  s = block_sum_fixed(s);
  if (threadIdx.x == 0) part[nb] = s;
}

// Masked MSE over N samples of C channels: every block first forms the
// normaliser norm = C * sum of the N mask sums (or C * N * HW without a mask)
// in the same fixed order, then its chunk of sample nb gives
// g = 2 mask (y - t) / norm and the chunk's sum of mask (y - t)^2 in
// part[nb * kLossChunks + chunk]; the host divides the sum of the parts by the
// same normaliser.
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                            const float* __restrict__ mask, const double* __restrict__ mpart, int N,
                            int C, int HW, float* __restrict__ g, double* __restrict__ part) {
  __shared__ double inv_norm;
  if (threadIdx.x == 0) {
    double m = 0.0;
    if (mask) {
      for (int i = 0; i < N; ++i) m += mpart[i];
    } else {
      m = (double)N * HW;
    }
    inv_norm = 1.0 / (m * C);
  }
  __syncthreads();
  const int nb = blockIdx.x, ch = blockIdx.y;
  const int tot = C * HW;
  const int per = (tot + kLossChunks - 1) / kLossChunks, k0 = ch * per, k1 = min(tot, k0 + per);
  double s = 0.0;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int c = k / HW, p = k - c * HW;
    const long long i = ((long long)nb * C + c) * HW + p;
    const double w = mask ? mask[(long long)nb * HW + p] : 1.0;
    const double d = (double)y[i] - (double)t[i];
    s += w * d * d;
    g[i] = (float)(2.0 * w * d * inv_norm);
  }
  s = block_sum_fixed(s);
  if (threadIdx.x == 0) part[nb * kLossChunks + ch] = s;
}

// Adam on the FP32 master parameters, refreshing the BF16 copy.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ pb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

// W'[ci][co t'] = W[co][ci t] with t' = flipped tap (for input gradients)
__global__ void flip_kernel(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt,
                            int Co, int Ci, int ks) {
  const int kk = ks * ks;
  const long long tot = (long long)Co * Ci * kk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % kk), ci = (int)((i / kk) % Ci), co = (int)(i / ((long long)kk * Ci));
    wt[((long long)ci * Co + co) * kk + (kk - 1 - t)] = w[i];
  }
}

int grid1(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

struct Conv {  // one convolution layer
  int index, ci, co, ks, H, W;
  long long w_off, b_off;  // offsets in the parameter vector (weights, then bias)
};

// activation buffers of the U-Net, in forward order
enum { kMaxLevels = 6 };

struct Plan {
  // buffer ids
  int in, a1[kMaxLevels], cat[kMaxLevels], pool[kMaxLevels], b1, b2, d1[kMaxLevels], d2[kMaxLevels], out;
};

}  // namespace

struct clbm_net {
  clbm_net_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Conv> convs;
  long long nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *pb = nullptr, *pt = nullptr;  // BF16 weights and flipped copy
  __nv_bfloat16* packed = nullptr;             // tensor-core weight tiles (PackDesc layout)
  PackDesc* d_pack = nullptr;
  std::vector<PackDesc> pack;                  // [2 * layer + transpose]
  long long packed_max = 0;
  std::vector<float*> act, gact;               // per buffer
  std::vector<int> act_c, act_hw;              // channels and H (= W) of each buffer
  float* part = nullptr;                       // split-K partials
  long long part_cap = 0;
  double* loss_part = nullptr;  // [max_batch][kLossChunks] loss partials, then [max_batch] mask sums
  int* tflag = nullptr;  // mapped pinned host flag: a tensor-core wait timed out
  int* d_tflag = nullptr;
  int64_t steps = 0;
  int sms = 152;  // multiprocessors of the device (one wave = 5 CTAs per SM)
  Plan plan{};
  std::string err;
  // A pass captured as a CUDA graph on its first call with a given key (batch
  // size, mask or none) and replayed while the key stays the same; the pass
  // reads and writes the network's own buffers only.
  struct Captured {
    cudaGraphExec_t exec = nullptr;
    const void *a = nullptr, *b = nullptr, *c = nullptr;
    int N = 0;
  };
  Captured grad_pass, fwd_pass;
  double* h_loss = nullptr;  // page-locked copy of the loss partials and mask sums
  float *tgt = nullptr, *msk = nullptr;  // the caller's target and mask, copied in before a pass
};

namespace {

Plan make_plan(clbm_net* net) {
  const int L = net->cfg.levels, B = net->cfg.base, G = net->cfg.grid;
  Plan P;
  auto add = [&](int c, int h) {
    net->act_c.push_back(c);
    net->act_hw.push_back(h);
    return (int)net->act_c.size() - 1;
  };
  P.in = add(net->cfg.in_ch, G);
  for (int l = 0; l < L - 1; ++l) {
    const int c = B << l, h = G >> l;
    P.a1[l] = add(c, h);
    P.cat[l] = add((B << (l + 1)) + c, h);  // [up (c_{l+1}) | skip (c_l)]
    P.pool[l] = add(c, h / 2);
  }
  const int cb = B << (L - 1), hb = G >> (L - 1);
  P.b1 = add(cb, hb);
  P.b2 = add(cb, hb);
  for (int l = L - 2; l >= 0; --l) {
    const int c = B << l, h = G >> l;
    P.d1[l] = add(c, h);
    P.d2[l] = add(c, h);
  }
  P.out = add(net->cfg.out_ch, G);
  return P;
}

Act view(clbm_net* net, int id, int coff, int C, bool grad = false) {
  Act a;
  a.base = grad ? net->gact[id] : net->act[id];
  a.cs = net->act_c[id];
  a.coff = coff;
  a.C = C;
  a.H = a.W = net->act_hw[id];
  return a;
}

bool tensor_math(const clbm_net* net) { return net->cfg.math == CLBM_NET_TENSOR; }

// D[M][N] (+ split-K along z) on the tensor cores
template <class GA, class GB, class ST>
cudaError_t tc_gemm(clbm_net* net, GA ga, GB gb, ST st, int M, int N, int K, int kper) {
  const int bn = tc::tile_n(N);
  auto kern = tc::gemm_kernel<GA, GB, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::smem_bytes(tc::kMaxBN));
  if (e) return e;
  dim3 grid((M + tc::kBM - 1) / tc::kBM, (N + bn - 1) / bn, (K + kper - 1) / kper);
  kern<<<grid, tc::kThreads, tc::smem_bytes(bn), net->stream>>>(ga, gb, st, M, N, K, kper, bn, net->d_tflag);
  return cudaGetLastError();
}

// K ranges of a forward / input-gradient GEMM: with less than one wave of CTAs
// (five resident per SM) and at least eight 64-wide K slices, K is split (at
// least four slices per range) until there is about one wave (measured against
// two CTAs per SM: 2.43 -> 2.44 ms per 64^2 training step, 6.33 -> 6.23 ms at
// 128^2).
int conv_splits(int sms, int M, int N, int K) {
  const int bn = tc::tile_n(N);
  const long long ctas = (long long)((M + tc::kBM - 1) / tc::kBM) * ((N + bn - 1) / bn);
  const int slices = (K + tc::kBK - 1) / tc::kBK;
  const long long wave = 5LL * sms;
  if (ctas >= wave || slices < 8) return 1;
  const long long s = std::min<long long>((wave + ctas - 1) / ctas, slices / 4);
  if (s <= 1) return 1;
  const int kper = (int)(((K + s - 1) / s + tc::kBK - 1) / tc::kBK) * tc::kBK;
  return (K + kper - 1) / kper;
}

// Implicit-im2col forward or input-gradient GEMM; split GEMMs finish in
// splitk_finish_kernel.
template <int KS, class GB>
cudaError_t tc_conv_gemm(clbm_net* net, Act x, GB gb, StoreAct st, int M, int N, int K) {
  const int splits = conv_splits(net->sms, M, N, K);
  if (splits == 1) return tc_gemm(net, GatherIm2col<KS>{x}, gb, TStoreAct{st}, M, N, K, K);
  if ((long long)splits * M * N > net->part_cap) return cudaErrorInvalidValue;
  const int kper = (K + splits - 1) / splits;
  const int kp = (kper + tc::kBK - 1) / tc::kBK * tc::kBK;
  cudaError_t e = tc_gemm(net, GatherIm2col<KS>{x}, gb, TStoreSplit{net->part, M, N}, M, N, K, kp);
  if (e) return e;
  splitk_finish_kernel<<<dim3((unsigned)std::min((M + 255) / 256, 64), (unsigned)std::min(N, 65535)), 256, 0, net->stream>>>(
      net->part, (K + kp - 1) / kp, M, N, st);
  return cudaGetLastError();
}

// Refresh the packed weight tiles from the BF16 weights (one launch, all layers).
cudaError_t pack_weights(clbm_net* net) {
  if (!tensor_math(net)) return cudaSuccess;
  dim3 grid((unsigned)std::min<long long>((net->packed_max + 255) / 256, 1024), (unsigned)net->pack.size());
  pack_weights_kernel<<<grid, 256, 0, net->stream>>>(net->d_pack, net->pb, net->packed);
  return cudaGetLastError();
}

tc::Packed packed_of(const clbm_net* net, int layer, int transpose) {
  const PackDesc& d = net->pack[2 * layer + transpose];
  return tc::Packed{net->packed + d.dst_off, d.slices};
}

// K range per split of a weight-gradient GEMM (K = pixels): the FP32 kernel
// takes 4096 pixels per split; the tensor-core one enough splits for about one
// wave of CTAs (five resident per SM, the shared-memory limit), at least four
// 64-wide K slices each (measured: 3, 5, 8 and 10 CTAs per SM gave 2.53,
// 2.55, 2.60 and 2.57 ms per 64^2 training step, 6.86, 6.80, 7.01 and
// 6.83 ms at 128^2).
long long dw_kper(int sms, bool tensor, long long Np, int Kd, int co) {
  if (!tensor) return 4096;
  const long long tiles = (long long)((Kd + tc::kBM - 1) / tc::kBM) * ((co + tc::kMaxBN - 1) / tc::kMaxBN);
  long long splits = std::max<long long>(1, (5LL * sms + tiles - 1) / tiles);
  splits = std::min<long long>(splits, std::max<long long>(1, Np / 256));
  const long long per = (Np + splits - 1) / splits;
  return ((per + tc::kBK - 1) / tc::kBK) * tc::kBK;
}

cudaError_t conv_forward(clbm_net* net, const Conv& cv, Act x, int out_id, int out_coff, int relu,
                         int N) {
  const int M = cv.co, Kd = cv.ci * cv.ks * cv.ks, Np = N * cv.H * cv.W;
  LoadW la{net->pb + cv.w_off, Kd};
  LoadIm2col lb{x, cv.ks};
  StoreAct st{net->act[out_id], net->act_c[out_id], out_coff, cv.H, cv.W, net->p + cv.b_off, relu, 0};
  if (tensor_math(net)) {  // D(pixel, co) = sum_k im2col(x)(pixel, k) W(co, k)
    const tc::Packed w = packed_of(net, cv.index, 0);
    if (cv.ks == 3) return tc_conv_gemm<3>(net, x, w, st, Np, M, Kd);
    return tc_conv_gemm<1>(net, x, w, st, Np, M, Kd);
  }
  dim3 grid((Np + BN - 1) / BN, (M + BM - 1) / BM, 1);
  gemm_kernel<<<grid, GT, 0, net->stream>>>(la, lb, st, M, Np, Kd, Kd);
  return cudaGetLastError();
}

// Backward of y = act(conv(x)): gy is the gradient buffer of y (ReLU already applied
// by the caller); accumulates into gx (if gx_id >= 0), writes dW, db.
// relu_gx: gx is the gradient of a ReLU output whose only contribution is
// this one, so the ReLU backward is applied in the store (no separate pass).
cudaError_t conv_backward(clbm_net* net, const Conv& cv, Act x, Act gy, int gx_id, int gx_coff,
                          int N, bool relu_gx = false) {
  const int Kd = cv.ci * cv.ks * cv.ks, Np = N * cv.H * cv.W;
  // weight gradient: M = co, N = ci*t, K = pixels, split-K
  {
    const bool tensor = tensor_math(net);
    const int kper = (int)dw_kper(net->sms, tensor, Np, Kd, cv.co);
    const int splits = (Np + kper - 1) / kper;
    const long long need = (long long)splits * cv.co * Kd;
    if (need > net->part_cap) return cudaErrorInvalidValue;
    LoadActMK la{gy};
    LoadIm2colT lb{x, cv.ks};
    StorePartial st{net->part, cv.co, Kd};
    if (tensor) {  // D((ci, t), co) = sum_p im2col(x)(p, (ci, t)) gy(co, p)
      cudaError_t e = cv.ks == 3
                          ? tc_gemm(net, GatherIm2colT<3>{x}, GatherRows{gy}, TStorePartial{st}, Kd, cv.co, Np, kper)
                          : tc_gemm(net, GatherIm2colT<1>{x}, GatherRows{gy}, TStorePartial{st}, Kd, cv.co, Np, kper);
      if (e) return e;
    } else {
      dim3 grid((Kd + BN - 1) / BN, (cv.co + BM - 1) / BM, splits);
      gemm_kernel<<<grid, GT, 0, net->stream>>>(la, lb, st, cv.co, Kd, Np, kper);
    }
    const long long n = (long long)cv.co * Kd;
    sum_splits(net->part, splits, n, net->g + cv.w_off, net->sms, net->stream);
    // bias: the split-K partials are consumed, so part holds the chunk sums next
    const int chunks = (Np + kBiasChunk - 1) / kBiasChunk;
    if ((long long)chunks * cv.co > net->part_cap) return cudaErrorInvalidValue;
    bias_partial_kernel<<<dim3(chunks, cv.co), GT, 0, net->stream>>>(gy, N, net->part);
    sum_splits(net->part, chunks, cv.co, net->g + cv.b_off, net->sms, net->stream);
  }
  if (gx_id >= 0) {  // input gradient: M = ci, N = pixels, K = co*t, with flipped weights
    const int kk = cv.ks * cv.ks;
    StoreAct st{net->gact[gx_id], net->act_c[gx_id], gx_coff, cv.H, cv.W, nullptr, 0, 1};
    if (relu_gx) st.relu_of = net->act[gx_id];
    if (tensor_math(net)) {  // D(pixel, ci) = sum_k im2col(gy)(pixel, k) W'(ci, k)
      const tc::Packed w = packed_of(net, cv.index, 1);
      const int K = cv.co * kk;
      if (cv.ks == 3) return tc_conv_gemm<3>(net, gy, w, st, Np, cv.ci, K);
      return tc_conv_gemm<1>(net, gy, w, st, Np, cv.ci, K);
    }
    flip_kernel<<<grid1((long long)cv.co * cv.ci * kk), 256, 0, net->stream>>>(
        net->pb + cv.w_off, net->pt + cv.w_off, cv.co, cv.ci, cv.ks);
    LoadW la{net->pt + cv.w_off, cv.co * kk};
    LoadIm2col lb{gy, cv.ks};
    dim3 grid((Np + BN - 1) / BN, (cv.ci + BM - 1) / BM, 1);
    gemm_kernel<<<grid, GT, 0, net->stream>>>(la, lb, st, cv.ci, Np, cv.co * kk, cv.co * kk);
  }
  return cudaGetLastError();
}

// Full forward pass over N samples already in act[in].
cudaError_t forward(clbm_net* net, const Plan& P, int N) {
  const int L = net->cfg.levels, B = net->cfg.base;
  cudaError_t e;
  int ci = 0;
  Act x = view(net, P.in, 0, net->cfg.in_ch);
  for (int l = 0; l < L - 1; ++l) {
    const int c = B << l, cup = B << (l + 1);
    if ((e = conv_forward(net, net->convs[ci++], x, P.a1[l], 0, 1, N))) return e;
    if ((e = conv_forward(net, net->convs[ci++], view(net, P.a1[l], 0, c), P.cat[l], cup, 1, N))) return e;
    Act skip = view(net, P.cat[l], cup, c);
    pool_kernel<<<plane_grid((skip.H / 2) * (skip.W / 2), (long long)N * c), 256, 0, net->stream>>>(
        skip, net->act[P.pool[l]], c, 0, N);
    x = view(net, P.pool[l], 0, c);
  }
  const int cb = B << (L - 1);
  if ((e = conv_forward(net, net->convs[ci++], x, P.b1, 0, 1, N))) return e;
  if ((e = conv_forward(net, net->convs[ci++], view(net, P.b1, 0, cb), P.b2, 0, 1, N))) return e;
  Act prev = view(net, P.b2, 0, cb);
  for (int l = L - 2; l >= 0; --l) {
    const int c = B << l, cup = B << (l + 1);
    up_kernel<<<plane_grid(prev.H * 2 * prev.W * 2, (long long)N * cup), 256, 0, net->stream>>>(
        prev, net->act[P.cat[l]], net->act_c[P.cat[l]], 0, N);
    if ((e = conv_forward(net, net->convs[ci++], view(net, P.cat[l], 0, cup + c), P.d1[l], 0, 1, N))) return e;
    if ((e = conv_forward(net, net->convs[ci++], view(net, P.d1[l], 0, c), P.d2[l], 0, 1, N))) return e;
    prev = view(net, P.d2[l], 0, c);
  }
  if ((e = conv_forward(net, net->convs[ci++], prev, P.out, 0, 0, N))) return e;
  return cudaGetLastError();
}

// Backward pass; gact[out] holds dloss/dout on entry; writes net->g.
cudaError_t backward(clbm_net* net, const Plan& P, int N) {
  const int L = net->cfg.levels, B = net->cfg.base;
  cudaError_t e;
  // zero all activation gradients except the output's
  for (size_t id = 0; id + 1 < net->gact.size(); ++id) {
    const long long n = (long long)N * net->act_c[id] * net->act_hw[id] * net->act_hw[id];
    if ((e = cudaMemsetAsync(net->gact[id], 0, n * sizeof(float), net->stream))) return e;
  }
  int ci = (int)net->convs.size() - 1;
  // head
  {
    const Conv& cv = net->convs[ci--];
    if ((e = conv_backward(net, cv, view(net, P.d2[0], 0, B), view(net, P.out, 0, net->cfg.out_ch, true),
                           P.d2[0], 0, N, true))) return e;
  }
  // Every ReLU backward is applied where its gradient is complete: in the
  // input-gradient store of a convolution that is its only source (d2[0], d1,
  // b1, a1), in the upsampling backward (d2[l > 0], b2) and in the pooling
  // backward, which adds the last contribution to a skip connection.
  // decoder, shallowest level first (reverse of the forward order)
  for (int l = 0; l <= L - 2; ++l) {
    const int c = B << l, cup = B << (l + 1);
    const Conv& c2 = net->convs[ci--];
    const Conv& c1 = net->convs[ci--];
    if ((e = conv_backward(net, c2, view(net, P.d1[l], 0, c), view(net, P.d2[l], 0, c, true), P.d1[l], 0, N,
                           true))) return e;
    if ((e = conv_backward(net, c1, view(net, P.cat[l], 0, cup + c), view(net, P.d1[l], 0, c, true), P.cat[l], 0, N))) return e;
    // gradient of the upsampled part flows to the level below (d2[l+1] or b2)
    const int below = (l + 1 <= L - 2) ? P.d2[l + 1] : P.b2;
    Act gup = view(net, P.cat[l], 0, cup, true);
    up_back_kernel<<<plane_grid((gup.H / 2) * (gup.W / 2), (long long)N * cup), 256, 0, net->stream>>>(
        gup, net->gact[below], net->act_c[below], 0, N, net->act[below]);
  }
  // bottleneck
  {
    const int cb = B << (L - 1);
    const Conv& c2 = net->convs[ci--];
    const Conv& c1 = net->convs[ci--];
    if ((e = conv_backward(net, c2, view(net, P.b1, 0, cb), view(net, P.b2, 0, cb, true), P.b1, 0, N,
                           true))) return e;
    const int inb = P.pool[L - 2];
    if ((e = conv_backward(net, c1, view(net, inb, 0, B << (L - 2)), view(net, P.b1, 0, cb, true),
                           inb, 0, N))) return e;
  }
  // encoder, deepest first
  for (int l = L - 2; l >= 0; --l) {
    const int c = B << l, cup = B << (l + 1);
    const Conv& c2 = net->convs[ci--];
    const Conv& c1 = net->convs[ci--];
    // pool backward adds into the skip part of cat[l]
    Act gp = view(net, P.pool[l], 0, c, true);
    pool_back_kernel<<<plane_grid(gp.H * 2 * gp.W * 2, (long long)N * c), 256, 0, net->stream>>>(
        gp, net->gact[P.cat[l]], net->act_c[P.cat[l]], cup, N, net->act[P.cat[l]]);
    if ((e = conv_backward(net, c2, view(net, P.a1[l], 0, c), view(net, P.cat[l], cup, c, true), P.a1[l], 0, N,
                           true))) return e;
    const int inb = l > 0 ? P.pool[l - 1] : P.in;
    const int cin = l > 0 ? (B << (l - 1)) : net->cfg.in_ch;
    if ((e = conv_backward(net, c1, view(net, inb, 0, cin), view(net, P.a1[l], 0, c, true),
                           l > 0 ? inb : -1, 0, N))) return e;
  }
  return cudaGetLastError();
}

// Enqueue a pass (`body` launches it on net->stream) as a replayed graph: the
// first call with a new key (batch size, mask or none) captures it, later
// calls with the same key launch the instantiated graph, one launch for the
// whole pass.  A stream that cannot be captured (the legacy default stream)
// runs the pass directly.
template <class F>
cudaError_t run_captured(clbm_net* net, clbm_net::Captured& g, const void* a, const void* b, const void* c,
                         int N, F body) {
  if (g.exec && g.a == a && g.b == b && g.c == c && g.N == N) return cudaGraphLaunch(g.exec, net->stream);
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return body();
  }
  const cudaError_t eb = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(net->stream, &graph);
  if (eb || ec) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return eb ? eb : ec;
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei) {
    g.exec = nullptr;
    return ei;
  }
  g.a = a;
  g.b = b;
  g.c = c;
  g.N = N;
  return cudaGraphLaunch(g.exec, net->stream);
}

clbm_status nfail(clbm_net* n, clbm_status s, const std::string& m) {
  if (n) n->err = m;
  return s;
}

const char* const kTimeoutMsg =
    "a tensor-core GEMM gave up waiting for its MMAs (results of this and later calls are invalid)";

bool timed_out(const clbm_net* n) { return *(volatile int*)n->tflag != 0; }

clbm_status cuda_status(clbm_net* n, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return CLBM_OK;
  return nfail(n, CLBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// splitmix64 -> uniform [0, 1)
double u01(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

extern "C" {

const char* clbm_net_last_error(const clbm_net* n) { return n ? n->err.c_str() : ""; }

clbm_status clbm_net_destroy(clbm_net* n) {
  if (!n) return CLBM_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->pb);
  cudaFree(n->pt);
  for (float* a : n->act) cudaFree(a);
  for (float* a : n->gact) cudaFree(a);
  cudaFree(n->part);
  cudaFree(n->loss_part);
  if (n->grad_pass.exec) cudaGraphExecDestroy(n->grad_pass.exec);
  if (n->fwd_pass.exec) cudaGraphExecDestroy(n->fwd_pass.exec);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  cudaFree(n->tgt);
  cudaFree(n->msk);
  if (n->tflag) cudaFreeHost(n->tflag);
  cudaFree(n->packed);
  cudaFree(n->d_pack);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
  return CLBM_OK;
}

clbm_status clbm_net_create(const clbm_net_config* cfg, uint64_t seed, void* stream, clbm_net** out) {
  if (!out || !cfg) return CLBM_EINVAL;
  *out = nullptr;
  const clbm_net_config& c = *cfg;
  if (c.levels < 2 || c.levels > kMaxLevels || c.base < 1 || c.in_ch < 1 || c.out_ch < 1 ||
      c.max_batch < 1 || c.grid < 2 || (c.grid % (1 << (c.levels - 1))) != 0 ||
      (c.math != CLBM_NET_TENSOR && c.math != CLBM_NET_FP32) ||
      (long long)c.max_batch * c.grid * c.grid >= (1LL << 31))
    return CLBM_EINVAL;
  clbm_net* n = new (std::nothrow) clbm_net();
  if (!n) return CLBM_ENOMEM;
  n->cfg = c;
  auto bail = [&](clbm_status s) {
    clbm_net_destroy(n);
    return s;
  };
  if (stream) {
    n->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(CLBM_ECUDA);
    n->own_stream = true;
  }
  // layers in forward order
  const int L = c.levels, B = c.base, G = c.grid;
  long long off = 0;
  auto add_conv = [&](int ci, int co, int ks, int h) {
    Conv cv{(int)n->convs.size(), ci, co, ks, h, h, off, off + (long long)co * ci * ks * ks};
    off = cv.b_off + co;
    n->convs.push_back(cv);
  };
  for (int l = 0; l < L - 1; ++l) {
    const int cin = l == 0 ? c.in_ch : (B << (l - 1));
    add_conv(cin, B << l, 3, G >> l);
    add_conv(B << l, B << l, 3, G >> l);
  }
  add_conv(B << (L - 2), B << (L - 1), 3, G >> (L - 1));
  add_conv(B << (L - 1), B << (L - 1), 3, G >> (L - 1));
  for (int l = L - 2; l >= 0; --l) {
    add_conv((B << (l + 1)) + (B << l), B << l, 3, G >> l);
    add_conv(B << l, B << l, 3, G >> l);
  }
  add_conv(B, c.out_ch, 1, G);
  n->nparam = off;
  // parameters: uniform(+-sqrt(6/fan_in)) weights (He), zero biases
  std::vector<float> h((size_t)off, 0.0f);
  uint64_t s = seed;
  for (const Conv& cv : n->convs) {
    const double a = std::sqrt(6.0 / (cv.ci * cv.ks * cv.ks));
    for (long long k = 0; k < (long long)cv.co * cv.ci * cv.ks * cv.ks; ++k)
      h[cv.w_off + k] = (float)((2.0 * u01(s) - 1.0) * a);
  }
  if (cudaMalloc(&n->p, off * sizeof(float)) || cudaMalloc(&n->g, off * sizeof(float)) ||
      cudaMalloc(&n->m, off * sizeof(float)) || cudaMalloc(&n->v, off * sizeof(float)) ||
      cudaMalloc(&n->pb, off * sizeof(__nv_bfloat16)) || cudaMalloc(&n->pt, off * sizeof(__nv_bfloat16)))
    return bail(CLBM_ENOMEM);
  cudaMemcpy(n->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(n->m, 0, off * sizeof(float));
  cudaMemset(n->v, 0, off * sizeof(float));
  cudaMemset(n->g, 0, off * sizeof(float));
  to_bf16_kernel<<<grid1(off), 256, 0, n->stream>>>(n->p, n->pb, off);
  if (c.math == CLBM_NET_TENSOR) {
    long long total = 0;
    for (const Conv& cv : n->convs)
      for (int tr = 0; tr < 2; ++tr) {
        PackDesc d{};
        d.w_off = cv.w_off;
        d.dst_off = total;
        d.co = cv.co;
        d.ci = cv.ci;
        d.kk = cv.ks * cv.ks;
        d.transpose = tr;
        d.N = tr ? cv.ci : cv.co;
        d.K = (tr ? cv.co : cv.ci) * d.kk;
        d.bn = tc::tile_n(d.N);
        d.slices = (d.K + tc::kBK - 1) / tc::kBK;
        d.size = (long long)((d.N + d.bn - 1) / d.bn) * d.slices * d.bn * tc::kBK;
        total += (d.size + 63) / 64 * 64;  // keep every layer's tiles 128-byte aligned
        n->packed_max = std::max(n->packed_max, d.size);
        n->pack.push_back(d);
      }
    if (cudaMalloc(&n->packed, total * sizeof(__nv_bfloat16)) ||
        cudaMalloc(&n->d_pack, n->pack.size() * sizeof(PackDesc)))
      return bail(CLBM_ENOMEM);
    cudaMemcpy(n->d_pack, n->pack.data(), n->pack.size() * sizeof(PackDesc), cudaMemcpyHostToDevice);
    if (pack_weights(n) != cudaSuccess) return bail(CLBM_ECUDA);
  }
  // activations
  n->plan = make_plan(n);
  for (size_t id = 0; id < n->act_c.size(); ++id) {
    const long long e = (long long)c.max_batch * n->act_c[id] * n->act_hw[id] * n->act_hw[id];
    float *a = nullptr, *ga = nullptr;
    if (cudaMalloc(&a, e * sizeof(float)) || cudaMalloc(&ga, e * sizeof(float))) {
      cudaFree(a);
      return bail(CLBM_ENOMEM);
    }
    n->act.push_back(a);
    n->gact.push_back(ga);
  }
  {  // one wave of CTAs is sized from the device's multiprocessor count
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      n->sms = sms;
  }
  // split-K partials: enough for the largest batch (fewer pixels never need more splits)
  long long cap = 0;
  for (const Conv& cv : n->convs) {
    const int Kd = cv.ci * cv.ks * cv.ks;
    for (long long nb = 1; nb <= c.max_batch; ++nb) {
      const long long Np = nb * cv.H * cv.W;
      const long long kper = dw_kper(n->sms, c.math == CLBM_NET_TENSOR, Np, Kd, cv.co);
      cap = std::max(cap, ((Np + kper - 1) / kper) * cv.co * Kd);
      cap = std::max(cap, ((Np + kBiasChunk - 1) / kBiasChunk) * cv.co);  // bias chunk sums
      if (c.math == CLBM_NET_TENSOR) {  // split-K forward and input-gradient GEMMs
        cap = std::max(cap, (long long)conv_splits(n->sms, (int)Np, cv.co, Kd) * Np * cv.co);
        cap = std::max(cap, (long long)conv_splits(n->sms, (int)Np, cv.ci, cv.co * cv.ks * cv.ks) * Np * cv.ci);
      }
    }
  }
  n->part_cap = cap;
  if (cudaHostAlloc(&n->tflag, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return bail(CLBM_ENOMEM);
  *n->tflag = 0;
  if (cudaHostGetDevicePointer(&n->d_tflag, n->tflag, 0) != cudaSuccess) return bail(CLBM_ECUDA);
  if (cudaMalloc(&n->part, cap * sizeof(float)) ||
      cudaMalloc(&n->loss_part, (size_t)c.max_batch * (kLossChunks + 1) * sizeof(double)) ||
      cudaHostAlloc(&n->h_loss, (size_t)c.max_batch * (kLossChunks + 1) * sizeof(double), cudaHostAllocDefault) ||
      cudaMalloc(&n->tgt, (size_t)c.max_batch * c.out_ch * c.grid * c.grid * sizeof(float)) ||
      cudaMalloc(&n->msk, (size_t)c.max_batch * c.grid * c.grid * sizeof(float)))
    return bail(CLBM_ENOMEM);
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) return bail(CLBM_ECUDA);
  *out = n;
  return CLBM_OK;
}

clbm_status clbm_net_param_count(const clbm_net* n, int64_t* count) {
  if (!n || !count) return CLBM_EINVAL;
  *count = n->nparam;
  return CLBM_OK;
}

clbm_status clbm_net_get_params(const clbm_net* n, float* dst, int32_t on_device) {
  if (!n || !dst) return CLBM_EINVAL;
  if (cudaStreamSynchronize(n->stream)) return CLBM_ECUDA;
  return cudaMemcpy(dst, n->p, n->nparam * sizeof(float),
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost) ? CLBM_ECUDA : CLBM_OK;
}

clbm_status clbm_net_set_params(clbm_net* n, const float* src, int32_t on_device) {
  if (!n || !src) return CLBM_EINVAL;
  if (cudaStreamSynchronize(n->stream) ||
      cudaMemcpy(n->p, src, n->nparam * sizeof(float),
                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice))
    return CLBM_ECUDA;
  to_bf16_kernel<<<grid1(n->nparam), 256, 0, n->stream>>>(n->p, n->pb, n->nparam);
  if (pack_weights(n) != cudaSuccess) return nfail(n, CLBM_ECUDA, "pack weights");
  cudaMemsetAsync(n->m, 0, n->nparam * sizeof(float), n->stream);
  cudaMemsetAsync(n->v, 0, n->nparam * sizeof(float), n->stream);
  n->steps = 0;
  return cuda_status(n, cudaStreamSynchronize(n->stream), "set_params");
}

clbm_status clbm_net_forward(clbm_net* n, const float* x, int32_t N, float* y) {
  if (!n || !x || !y || N < 1 || N > n->cfg.max_batch) return CLBM_EINVAL;
  if (timed_out(n)) return nfail(n, CLBM_ETIMEOUT, kTimeoutMsg);
  const Plan& P = n->plan;
  const long long in_e = (long long)N * n->cfg.in_ch * n->cfg.grid * n->cfg.grid;
  const long long out_e = (long long)N * n->cfg.out_ch * n->cfg.grid * n->cfg.grid;
  // the caller's buffers are copied in and out around the replayed pass, whose
  // graph then depends on the batch size alone
  cudaError_t e = cudaMemcpyAsync(n->act[P.in], x, in_e * sizeof(float), cudaMemcpyDeviceToDevice, n->stream);
  if (!e) e = run_captured(n, n->fwd_pass, nullptr, nullptr, nullptr, N, [&]() { return forward(n, P, N); });
  if (!e) e = cudaMemcpyAsync(y, n->act[P.out], out_e * sizeof(float), cudaMemcpyDeviceToDevice, n->stream);
  return cuda_status(n, e, "forward");
}

clbm_status clbm_net_gradients(clbm_net* n, const float* x, const float* target, const float* mask,
                               int32_t N, float* grad, double* loss) {
  if (!n || !x || !target || N < 1 || N > n->cfg.max_batch) return CLBM_EINVAL;
  const Plan& P = n->plan;
  const int G = n->cfg.grid, C = n->cfg.out_ch;
  const long long in_e = (long long)N * n->cfg.in_ch * G * G;
  // loss normalisation (sum of mask weights times channels) on the device, so
  // that the backward pass follows the forward pass without a host round trip
  double* mpart = n->loss_part + (size_t)n->cfg.max_batch * kLossChunks;
  const double* lp = n->h_loss;
  // inputs copied in first: the replayed pass depends on the batch size and on
  // whether there is a mask, not on the caller's buffers
  const float* msk = mask ? n->msk : nullptr;
  cudaError_t e = cudaMemcpyAsync(n->act[P.in], x, in_e * sizeof(float), cudaMemcpyDeviceToDevice, n->stream);
  if (!e)
    e = cudaMemcpyAsync(n->tgt, target, (size_t)N * C * G * G * sizeof(float), cudaMemcpyDeviceToDevice,
                        n->stream);
  if (!e && mask)
    e = cudaMemcpyAsync(n->msk, mask, (size_t)N * G * G * sizeof(float), cudaMemcpyDeviceToDevice, n->stream);
  if (!e) e = run_captured(n, n->grad_pass, msk, nullptr, nullptr, N, [&]() {
    cudaError_t e = forward(n, P, N);
    if (!e && msk) {
      mask_sum_kernel<<<N, GT, 0, n->stream>>>(msk, G * G, mpart);
      e = cudaGetLastError();
    }
    if (!e) {
      loss_kernel<<<dim3(N, kLossChunks), GT, 0, n->stream>>>(n->act[P.out], n->tgt, msk, mpart, N, C, G * G,
                                                              n->gact[P.out], n->loss_part);
      e = cudaGetLastError();
    }
    if (!e) e = backward(n, P, N);
    if (!e)
      e = cudaMemcpyAsync(n->h_loss, n->loss_part, (size_t)N * kLossChunks * sizeof(double),
                          cudaMemcpyDeviceToHost, n->stream);
    if (!e && mask)
      e = cudaMemcpyAsync(n->h_loss + (size_t)N * kLossChunks, mpart, (size_t)N * sizeof(double),
                          cudaMemcpyDeviceToHost, n->stream);
    return e;
  });
  if (!e) e = cudaStreamSynchronize(n->stream);
  if (e) return cuda_status(n, e, "gradients");
  if (timed_out(n)) return nfail(n, CLBM_ETIMEOUT, kTimeoutMsg);
  // the normaliser in the loss kernel's order
  double norm = 0.0;
  if (mask) {
    for (int i = 0; i < N; ++i) norm += lp[(size_t)N * kLossChunks + i];
  } else {
    norm = (double)N * G * G;
  }
  norm *= C;
  if (!(norm > 0)) return nfail(n, CLBM_EINVAL, "empty loss mask");
  double s = 0.0;
  for (int i = 0; i < N * kLossChunks; ++i) s += lp[i];
  if (loss) *loss = s / norm;
  if (grad) {
    e = cudaMemcpy(grad, n->g, n->nparam * sizeof(float), cudaMemcpyDefault);
    if (e) return cuda_status(n, e, "copy gradients");
  }
  return CLBM_OK;
}

clbm_status clbm_net_train_step(clbm_net* n, const float* x, const float* target, const float* mask,
                                int32_t N, float lr, double* loss) {
  clbm_status st = clbm_net_gradients(n, x, target, mask, N, nullptr, loss);
  if (st != CLBM_OK) return st;
  n->steps += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - std::pow(b1, (float)n->steps));
  const float c2 = 1.0f / (1.0f - std::pow(b2, (float)n->steps));
  adam_kernel<<<grid1(n->nparam), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->pb, n->nparam, lr,
                                                        b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (!e) e = pack_weights(n);
  return cuda_status(n, e, "adam");
}

}  // extern "C"
