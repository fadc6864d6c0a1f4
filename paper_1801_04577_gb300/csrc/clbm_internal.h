// Internal interface between the C ABI (clbm_api.cu) and the per-precision
// kernel translation units (clbm_kernels_*.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace clbm {

// Node flag bits of the masked lattice layout (one uint16_t per node).
//   bits 0..7 : the pull source x - e_j of D2Q9 direction j = bit + 1 is a wall
//               (a solid node or a non-periodic box side)
//   bit 8     : the node itself is solid
//   bit 9     : the node has listed (curved / obstacle) thermal wall links
constexpr uint16_t kFlagSolid = 1u << 8;
constexpr uint16_t kFlagLinks = 1u << 9;

// Lattice geometry as seen by the kernels.  Distribution planes are stored
// structure-of-arrays: plane q (f_0..f_8, then g_0..g_4) holds ny rows of
// `pitch` elements, pitch = nx rounded up to a whole warp of vectors.
struct DevGeom {
  int nx, ny, pitch, px, py;
  long long plane;             // elements per plane = ny * pitch
  const uint16_t* flags;       // [ny][pitch] or nullptr (box walls only)
  const int32_t* slot;         // [ny][pitch] link slot, -1 = none (masked lattices)
  const double* lk_ne;         // [nslots][4] n.e_i per link direction i = 1..4
  const int32_t* lk_tbc;       // [nslots][4] condition index, -1 = no link
  const double* tbc;           // [ntbc][3] (b1, b2, b3)
  double side_b[4][3];         // conditions of the box sides x0, x1, y0, y1
};

// Relaxation and forcing constants in FP64 (converted to the compute type
// inside the kernels).  s3 and lambda2 are already resolved.
struct DevCoef {
  double s_nu, s_b, s3, s4, l0, l1, l2;
  double rho0, T0, gbeta, Fvx, Fvy, Q, cT2;
};

struct StepArgs {
  DevGeom g;
  DevCoef c;
  const void* src;  // post-collision state at time t
  void* dst;        // post-collision state at time t + 1
  uint32_t seed;    // per-step key of the stochastic-rounding hash
  int stochastic;   // 16-bit stores: 0 = nearest even, 1 = stochastic
};

// One Nusselt link, prepared on the host: node index (pitch layout) of x_f,
// index of x_f - e_i (or -1 when it is not a fluid node), n.e_i, (b1, b2, b3).
struct NuLink {
  long long own, second;
  double ne, b1, b2, b3;
};

// Launchers implemented once per storage type (S = double, float, __half,
// __nv_bfloat16).  All enqueue on `stream` and return cudaGetLastError().
struct Launchers {
  int vec;  // nodes per thread in the step kernel (pitch granularity = 32 * vec)
  cudaError_t (*step)(const StepArgs& a, cudaStream_t s);
  cudaError_t (*init)(const DevGeom& g, const DevCoef& c, void* dst, const double* rho,
                      const double* ux, const double* uy, const double* T, cudaStream_t s);
  cudaError_t (*moments)(const DevGeom& g, const DevCoef& c, const void* buf, double* rho,
                         double* ux, double* uy, double* T, cudaStream_t s);
  // residual partial sums: out[b*8 + k], k = sum dT^2, T^2, dux^2, ux^2, duy^2, uy^2, nonfinite
  cudaError_t (*residual)(const DevGeom& g, const DevCoef& c, const void* cur, const void* prev,
                          double* partials, int nblocks, cudaStream_t s);
  cudaError_t (*nusselt)(const DevGeom& g, const DevCoef& c, const void* buf, const NuLink* links,
                         int nlinks, double* partials, int nblocks, cudaStream_t s);
  size_t elem_bytes;
};

extern const Launchers kLaunchF64;
extern const Launchers kLaunchF32;
extern const Launchers kLaunchF16;
extern const Launchers kLaunchBF16;

// Fixed-order sum of nblocks x width partials into out[width] (one block).
cudaError_t launch_reduce_partials(const double* partials, int nblocks, int width, double* out,
                                   cudaStream_t s);

}  // namespace clbm
