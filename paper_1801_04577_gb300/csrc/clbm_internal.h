// Internal interface between the C ABI (clbm_api.cu) and the per-precision
// kernel translation units (clbm_kernels_*.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/clbm.h"

namespace clbm {

// Node flag bits of the masked lattice layout (one uint16_t per node).
//   bits 0..7 : the pull source x - e_j of D2Q9 direction j = bit + 1 is a wall
//               (a solid node or a non-periodic box side)
//   bit 8     : the node itself is solid
//   bit 9     : the node has listed (curved / obstacle) thermal wall links
constexpr uint16_t kFlagSolid = 1u << 8;
constexpr uint16_t kFlagLinks = 1u << 9;

// Planes per buffer: 14 distributions, plus the viscous source Q_v when enabled.
inline int planes_of(int vh) { return vh ? 15 : 14; }

// Lattice geometry as seen by the kernels.  Distribution planes are stored
// structure-of-arrays: plane q (f_0..f_8, then g_0..g_4) holds ny rows of
// `pitch` elements, pitch = nx rounded up to a whole warp of vectors.
struct DevGeom {
  int nx, ny, pitch, px, py;   // ny: stored rows (own rows plus any ghost rows)
  // Rows [ylo, yhi) of the storage are updated by the step; the rest are ghost
  // rows (a y-slab of a larger lattice keeps one on each side, holding its
  // neighbours' edge rows).  ywlo / ywhi: a box wall lies below row ylo /
  // above row yhi - 1.  yoff: global row of storage row 0 (stochastic-rounding
  // keys).  A whole lattice has ylo = 0, yhi = ny, ywlo = ywhi = !py, yoff = 0.
  int ylo, yhi, ywlo, ywhi, yoff;
  long long plane;             // elements per plane = ny * pitch
  const uint16_t* flags;       // [ny][pitch] or nullptr (box walls only)
  const int32_t* slot;         // [ny][pitch] link slot, -1 = none (masked lattices)
  const double* lk_ne;         // [nslots][4] n.e_i per link direction i = 1..4
  const int32_t* lk_tbc;       // [nslots][4] condition index, -1 = no link
  const double* lk_q;          // [nslots][8] wall fraction q per link direction i = 1..8 (0.5 = half-way)
  const double* tbc;           // [ntbc][3] (b1, b2, b3)
  const uint8_t* tile_fluid;   // [ny][tiles_per_row] class of each warp tile (32 V nodes of a row): 0 = no
                               // fluid node, 1 = no flagged node, 2 = holds flagged nodes; nullptr = box lattice
  int tiles_per_row, pad_tiles;
  double side_b[4][3];         // conditions of the box sides x0, x1, y0, y1
  float side_bf[4][3];         // the same rounded to FP32 (for FP32 arithmetic)
  // moving box sides (not in the paper): wall velocity of each side, and the
  // same rounded to FP32; moving = 0 when every side is at rest
  double side_u[4][2];
  float side_uf[4][2];
  int moving, pad_moving;
};

// Relaxation and forcing constants in FP64 (converted to the compute type
// inside the kernels).  s3 and lambda2 are already resolved.
// The same constants rounded once to FP32 on the host, for the kernels that
// compute in FP32 (GB300's FP64 rate is a small fraction of its FP32 rate, so
// converting them per thread is not free).
struct CoefF32 {
  float rho0, T0, s_nu, s_b, s3, s4, l1, l2;
  float rgb;  // rho0 * g beta
  float Fvx, Fvy, Q, hQ, cT2;
  float vhc;  // viscous source: 3 s_nu^2 (1/s_nu - 1/2), 0 when off
  float pad;
};

// The collision's rates combined with the exact power-of-two scalings of the
// form it relaxes in (moments of order one and two halved per direction, so
// that the back-transformation needs no halving of its own): computed once on
// the host in FP64, and rounded once for the FP32 kernels.
template <typename T>
struct CollideK {
  T hFx;                     // Fvx / 2
  T al, be;                  // -(s_b + s_nu) / 4, (s_nu - s_b) / 4 (the k~20, k~02 block)
  T snu4, snur4;             // (1 - s_nu) / 4, s_nu rho0 / 4
  T s3m4, s3r4, hs3q;        // (1 - s3) / 4, s3 rho0 / 4, (1 - s3 / 2) / 12
  T s4m4, s4r4, s4n, s4r9;   // (1 - s4) / 4, s4 rho0 / 4, s4 / 36, s4 rho0 / 36
  T l1m2, l1T2, l2m2, l2T2;  // (1 - l1) / 2, l1 T0 / 2, (1 - l2) / 2, l2 T0 / 2
  T srcq2, srct2;            // (1 - l2 / 2) cT2 / 2, l2 cT2 / 2
};

struct DevCoef {
  double s_nu, s_b, s3, s4, l0, l1, l2;
  double rho0, T0, gbeta, Fvx, Fvy, Q, cT2;
  int vh;  // 1: viscous dissipation source (stored as a 15th plane, Q_v at each node)
  int pad;
  CoefF32 f;            // filled by fill_f32
  CollideK<double> kd;  // filled by fill_f32
  CollideK<float> kf;
};

// FP32 copies of a DevCoef's constants (each computed in FP64, then rounded),
// and the combined collision constants in both precisions.
inline void fill_f32(DevCoef& k) {
  CollideK<double>& d = k.kd;
  d.hFx = 0.5 * k.Fvx;
  d.al = -0.25 * (k.s_b + k.s_nu);
  d.be = 0.25 * (k.s_nu - k.s_b);
  d.snu4 = 0.25 * (1.0 - k.s_nu);
  d.snur4 = 0.25 * k.s_nu * k.rho0;
  d.s3m4 = 0.25 * (1.0 - k.s3);
  d.s3r4 = 0.25 * k.s3 * k.rho0;
  d.hs3q = (1.0 - 0.5 * k.s3) / 12.0;
  d.s4m4 = 0.25 * (1.0 - k.s4);
  d.s4r4 = 0.25 * k.s4 * k.rho0;
  d.s4n = k.s4 / 36.0;
  d.s4r9 = k.s4 * k.rho0 / 36.0;
  d.l1m2 = 0.5 * (1.0 - k.l1);
  d.l1T2 = 0.5 * k.l1 * k.T0;
  d.l2m2 = 0.5 * (1.0 - k.l2);
  d.l2T2 = 0.5 * k.l2 * k.T0;
  d.srcq2 = 0.5 * (1.0 - 0.5 * k.l2) * k.cT2;
  d.srct2 = 0.5 * k.l2 * k.cT2;
  CollideK<float>& e = k.kf;
  e.hFx = (float)d.hFx;
  e.al = (float)d.al;
  e.be = (float)d.be;
  e.snu4 = (float)d.snu4;
  e.snur4 = (float)d.snur4;
  e.s3m4 = (float)d.s3m4;
  e.s3r4 = (float)d.s3r4;
  e.hs3q = (float)d.hs3q;
  e.s4m4 = (float)d.s4m4;
  e.s4r4 = (float)d.s4r4;
  e.s4n = (float)d.s4n;
  e.s4r9 = (float)d.s4r9;
  e.l1m2 = (float)d.l1m2;
  e.l1T2 = (float)d.l1T2;
  e.l2m2 = (float)d.l2m2;
  e.l2T2 = (float)d.l2T2;
  e.srcq2 = (float)d.srcq2;
  e.srct2 = (float)d.srct2;
  CoefF32& o = k.f;
  o.rho0 = (float)k.rho0;
  o.T0 = (float)k.T0;
  o.s_nu = (float)k.s_nu;
  o.s_b = (float)k.s_b;
  o.s3 = (float)k.s3;
  o.s4 = (float)k.s4;
  o.l1 = (float)k.l1;
  o.l2 = (float)k.l2;
  o.rgb = (float)(k.rho0 * k.gbeta);
  o.Fvx = (float)k.Fvx;
  o.Fvy = (float)k.Fvy;
  o.Q = (float)k.Q;
  o.hQ = (float)(0.5 * k.Q);
  o.cT2 = (float)k.cT2;
  o.vhc = (float)(k.vh ? 3.0 * k.s_nu * k.s_nu * (1.0 / k.s_nu - 0.5) : 0.0);
  o.pad = 0.0f;
}

struct StepArgs {
  DevGeom g;
  DevCoef c;
  const void* src;  // post-collision state at time t
  void* dst;        // post-collision state at time t + 1
  uint32_t seed;    // per-step key of the stochastic-rounding hash
  int stochastic;   // 16-bit stores: 0 = nearest even, 1 = stochastic
  const int32_t* bnodes;  // boundary nodes (pitch-layout indices) recomputed after the interior
  int nb;
  int reverse;  // walk the rows from the last one (alternate steps: reuse of L2-resident rows)
  const long long* tdev;  // if set: the step count lives on the device (graph replays); seed from *tdev + tstep
  int tstep;
};

// One Nusselt link, prepared on the host: node index (pitch layout) of x_f,
// index of x_f - e_i (or -1 when it is not a fluid node), n.e_i, (b1, b2, b3).
struct NuLink {
  long long own, second;
  double ne, b1, b2, b3;
  double q;  // wall fraction of the link (0.5 = half-way)
};

// ---------------------------------------------------------------------------
// Batched solves: many independent lattices advanced by the same launches.
// ---------------------------------------------------------------------------
constexpr int kBatchGroups = 3;  // tile width 32, 64, 128 nodes

// One lattice of a batch as the batched kernels see it.
struct BatchLat {
  DevGeom g;
  DevCoef c;
  void* buf[2];  // this lattice's two distribution buffers inside the batch arena
  double* snap;  // (T, ux, uy) at the previous convergence check, dense [3][ny][nx]
};

// Device-resident control block of a batched solve.
struct BatchCtl {
  long long t;                 // steps taken since the solve started
  int n_active;                // lattices still iterating
  int pad;
  int count[kBatchGroups];     // tiles per launch group
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
  // conservation partial sums: out[b*8 + k], k = sum of d_i, d_i e_ix, d_i e_iy, h_j over the fluid
  // nodes, fluid-node count, non-finite count
  cudaError_t (*totals)(const DevGeom& g, const void* buf, double* partials, int nblocks,
                        cudaStream_t s);
  size_t elem_bytes;
  // batched interior step over a tile list (tile = {lattice, row, first x, 0}; tiles skip the
  // first and last column); V = nodes per lane
  cudaError_t (*batch_step)(int V, const BatchLat* lats, const int4* tiles, const int* count,
                            int parity, const long long* t, int tstep, int stochastic, int grid,
                            cudaStream_t s);
  // batched boundary nodes: entries {lattice, node index}, skipped when the lattice is inactive
  cudaError_t (*batch_boundary)(const BatchLat* lats, const int2* entries, int n, const int* active,
                                int parity, const long long* t, int tstep, int stochastic,
                                cudaStream_t s);
  // persistent grid size (blocks) of the batched interior step for V
  int (*batch_grid)(int V);
  // a <- (a + b) / 2 over n stored values (all planes)
  cudaError_t (*average)(void* a, const void* b, long long n, cudaStream_t s);

  // per-lattice residual: change of (T, ux, uy) since the previous check (snapshot), per step
  // (divided by K); 1e300 when there is no snapshot yet, +inf if a value is non-finite.
  // part: n * maxchunks * 8 doubles of scratch, maxchunks >= chunks of the largest lattice
  cudaError_t (*batch_residual)(const BatchLat* lats, const int* active, int* snap_valid,
                                double* res, int n, int K, double* part, int maxchunks,
                                cudaStream_t s);
  int residual_chunk;  // nodes per residual chunk
};

extern const Launchers kLaunchF64;
extern const Launchers kLaunchF32;
extern const Launchers kLaunchF16;
extern const Launchers kLaunchBF16;

// Internal view API used by batches: a context whose two distribution buffers
// belong to someone else (the batch arena).
struct ViewInfo {
  DevGeom g;
  DevCoef c;
  void* buf[2];
  int pitch;
  long long plane;
  const int32_t* bnodes_host;  // boundary node list of the lattice (host copy)
  int nb;
};
int view_pitch(int nx, int precision);
size_t view_buffer_bytes(int nx, int ny, int precision, int vh);
clbm_status create_view(const clbm_params* p, cudaStream_t s, void* buf_a, void* buf_b,
                        clbm_ctx** out);
ViewInfo describe_view(const clbm_ctx* c);
void set_view_time(clbm_ctx* c, int64_t t, int cur);

// *t += k on the device (advances the step counter of a captured step graph)
cudaError_t launch_advance(long long* t, int k, cudaStream_t s);
cudaError_t launch_set_step(long long* t, long long v, cudaStream_t s);

// Halo rows of slabs held by one process: each entry copies one row of every
// plane (row_bytes, a multiple of 16, at planes plane strides) from src to dst.
constexpr int kMaxHaloCopies = 32;
struct HaloCopy {
  const char* src;
  char* dst;
  long long splane, dplane;  // plane strides in bytes
};
struct HaloTable {
  HaloCopy c[kMaxHaloCopies];
  int n, planes;
  long long row_bytes;
};
cudaError_t launch_halo(const HaloTable& t, cudaStream_t s);

// Fixed-order sum of nblocks x width partials into out[width] (one block).
cudaError_t launch_reduce_partials(const double* partials, int nblocks, int width, double* out,
                                   cudaStream_t s);

}  // namespace clbm
