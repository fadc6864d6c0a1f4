// Tensor-core (tcgen05) GEMM for the warm-start network's convolutions:
//
//   D[m][n] = sum_k A(m, k) B(n, k),   A, B rounded to BF16, D accumulated in FP32
//
// One CTA computes a 128-row tile of D (rows = TMEM lanes) for BN columns
// (16 <= BN <= 256, a multiple of 16) over a range of k (split-K along
// blockIdx.z).  Operands come from functors (implicit im2col, weights, ...):
// all 128 threads gather a 64-wide K slice of A and B, convert it to BF16 and
// write it into shared memory in the canonical no-swizzle K-major layout
// (core matrices of 8 rows x 16 bytes; the eight 16-byte K chunks of a row
// group are adjacent, 128 B apart, and row groups are 1024 B apart).  One
// thread issues four tcgen05.mma (M = 128, K = 16 each) per slice and commits
// them to the slice's mbarrier; the stage is refilled only after that barrier
// fires, so the gather of slice i+1 overlaps the MMAs of slice i.  The
// epilogue reads the accumulator with tcgen05.ld (warp w owns lanes
// 32w..32w+31) and hands every element to the store functor.
//
// The B operand can instead be pre-packed in global memory in exactly that
// layout and moved per slice by one cp.async.bulk copy (Packed).
//
// Every wait is bounded: a barrier that does not fire within about a second
// sets *err, the CTA stops issuing, waits (bounded) for what it issued, frees
// its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tc {

constexpr int kBM = 128;       // rows of D per CTA = TMEM lanes
constexpr int kBK = 64;        // K per shared-memory stage (four MMAs of K = 16)
constexpr int kStages = 2;
constexpr int kThreads = 128;  // one thread per row of A and per TMEM lane
constexpr int kMaxBN = 256;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

// bytes of dynamic shared memory for a tile width bn
__host__ __device__ constexpr int stage_bytes(int bn) { return (kBM + bn) * kBK * 2; }
__host__ __device__ constexpr int smem_bytes(int bn) { return kStages * stage_bytes(bn) + 64; }  // + barriers, TMEM slot

// byte offset of the 16-byte chunk kc (elements 8kc..8kc+7) of row r
__host__ __device__ constexpr uint32_t chunk_off_host(int r, int kc) {
  return (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
}
__device__ __forceinline__ uint32_t chunk_off(int r, int kc) { return chunk_off_host(r, kc); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between the two K core matrices of one MMA), stride byte offset
// (between 8-row groups), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits
// 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 columns of 32 bits: thread t of the warp gets lane (base + t)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr uint32_t tmem_cols(int bn) {
  return bn <= 32 ? 32u : bn <= 64 ? 64u : bn <= 128 ? 128u : 256u;
}

// Element-wise gatherer: operand(row, k) from a functor ld(row, k).  Fills
// rows [0, nrows) of a 64-wide K slice starting at k0 (zero beyond
// rows_valid or kend); row r's eight chunks are written by one thread (rows
// strided by the block), so the global reads of a warp walk 32 consecutive
// rows for each k.
template <class L>
struct Elementwise {
  static constexpr bool kBulk = false;
  L ld;
  __device__ __forceinline__ void operator()(uint8_t* dst, int row0, int rows_valid, int nrows, int k0,
                                             int kend) const {
    for (int r = threadIdx.x; r < nrows; r += kThreads) {
      const int row = row0 + r;
      const bool rv = r < rows_valid;
#pragma unroll 2
      for (int kc = 0; kc < kBK / 8; ++kc) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + kc * 8 + 2 * j;
          const float x0 = (rv && k < kend) ? ld(row, k) : 0.0f;
          const float x1 = (rv && k + 1 < kend) ? ld(row, k + 1) : 0.0f;
          w[j] = pack_bf16(x0, x1);
        }
        *reinterpret_cast<uint4*>(dst + chunk_off(r, kc)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
};

// Pre-packed BF16 operand: the (bn x 64) tile of N tile nt and K slice ks is
// stored, already in the shared-memory layout above, at
// base + (nt * slices + ks) * bn * 64 elements; one bulk copy moves it.
struct Packed {
  static constexpr bool kBulk = true;
  const __nv_bfloat16* base;
  int slices;  // K slices per N tile (K rounded up to 64, divided by 64)
  __device__ __forceinline__ const void* tile(int nt, int ks, int bn) const {
    return base + ((long long)nt * slices + ks) * bn * kBK;
  }
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// D tile (blockIdx.x over M in 128-row tiles, blockIdx.y over N in bn-column
// tiles, blockIdx.z over K in kper-long ranges, kper a multiple of 64 when
// there is more than one range); st(m, n, value, split).  A is gathered by all
// threads; B is gathered too, or (GB::kBulk) bulk-copied by thread 0 from a
// Packed buffer into the stage, completing on the stage's load barrier.
// Launch with kThreads threads and smem_bytes(bn) bytes of dynamic shared memory.
template <class GA, class GB, class ST>
__global__ void __launch_bounds__(kThreads) gemm_kernel(GA ga, GB gb, ST st, int M, int N, int K, int kper,
                                                        int bn, int* err) {
  static_assert(!GA::kBulk, "the A operand is always gathered");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int sbytes = stage_bytes(bn);
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(smem + kStages * sbytes);
  uint64_t* load_bar = mma_bar + kStages;
  uint32_t* slot = reinterpret_cast<uint32_t*>(load_bar + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * bn;
  const int kbeg = blockIdx.z * kper;
  const int kend = min(K, kbeg + kper);
  const int nk = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;
  const uint32_t ncols = tmem_cols(bn);
  const int mvalid = min(kBM, M - m0), nvalid = min(bn, N - n0);

  if (warp == 0) tmem_alloc(slot, ncols);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&mma_bar[s], 1);
      mbar_init(&load_bar[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *slot;
  const uint32_t idesc = idesc_bf16_f32(kBM, bn);

  int issued = -1;  // last slice whose MMAs were committed
  bool failed = false;
  for (int i = 0; i < nk; ++i) {
    const int s = i % kStages;
    uint8_t* As = smem + s * sbytes;
    uint8_t* Bs = As + kBM * kBK * 2;
    if (i >= kStages && !mbar_wait(&mma_bar[s], (uint32_t)(((i - kStages) / kStages) & 1))) failed = true;
    const int k0 = kbeg + i * kBK;
    if constexpr (GB::kBulk) {
      if (tid == 0 && !failed) {
        const uint32_t bytes = (uint32_t)bn * kBK * 2;
        mbar_expect_tx(&load_bar[s], bytes);
        bulk_load(Bs, gb.tile(blockIdx.y, k0 / kBK, bn), bytes, &load_bar[s]);
      }
    }
    if (!failed) {
      ga(As, m0, mvalid, kBM, k0, kend);
      if constexpr (!GB::kBulk) gb(Bs, n0, nvalid, bn, k0, kend);
    }
    if constexpr (GB::kBulk) {
      if (!failed && !mbar_wait(&load_bar[s], (uint32_t)((i / kStages) & 1))) failed = true;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    if (tid == 0) {
      fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        mma_bf16(tmem, smem_desc(a0 + kk * 256, 128, 1024), smem_desc(b0 + kk * 256, 128, 1024), idesc,
                 (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&mma_bar[s]);
    }
    issued = i;
  }
  // the last commit covers every MMA issued before it
  bool done = true;
  if (issued >= 0) done = mbar_wait(&mma_bar[issued % kStages], (uint32_t)((issued / kStages) & 1));
  if (failed || !done) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    fence_after();
    const int r = warp * 32 + lane;
    const int m = m0 + r;
    for (int c0 = 0; c0 < bn; c0 += 16) {
      float v[16];
      if (issued >= 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.0f;
      }
      if (r < mvalid) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < nvalid) st(m, n0 + c0 + j, v[j], (int)blockIdx.z);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Columns per N tile: the smallest multiple of 16 that covers N in
// ceil(N / 256) tiles.
inline int tile_n(int N) {
  const int tiles = (N + kMaxBN - 1) / kMaxBN;
  const int per = (N + tiles - 1) / tiles;
  return ((per + 15) / 16) * 16;
}

}  // namespace tc
