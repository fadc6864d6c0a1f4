// Device code of the fused cascaded thermal LBM step for sm_103a.
//
// One time step per node, in one pass over HBM (pull scheme):
//   pull      f_i(x) = f*_i(x - e_i), g_i(x) = g*_i(x - e_i)      Eq. 11, Eq. 21
//   walls     half-way bounce-back for f (Sec. 3); general bounce-back for g
//             with T_w from Eq. 28                                  Eq. 26-28
//   macros    T = sum g + Q/2, F = F_v + rho0 g beta (T - T0) e_y,
//             rho = sum f, u = (sum f e + F/2)/rho                 Eq. 25, 2, 12
//   collide   central moments (Eq. 4-6), relaxation (Eq. 7-10),
//             back-transformation (text after Eq. 11)
//   thermal   Eq. 15-20 with the heat source of Eq. 23-24
//   store     f*(x), g*(x)
//
// Layout and precision.  The state kept in HBM is the post-collision pair
// (f*, g*) at time t, stored structure-of-arrays as deviations from the rest
// state, d_i = f*_i - w_i rho0 and h_i = g*_i - w^T_i T0.  The collision is
// rewritten in these deviations (the rest-state moments at velocity u are
// known in closed form), so every intermediate is a small number and FP32
// keeps its relative precision on the physically relevant part.
//
// Moment transforms.  The nine moments {0,1,2}^2 of Eq. 5 are a tensor
// product, so N(u) M f is computed as a 1-D central-moment transform along x
// for each of the three rows of velocities, then along y (and the inverse in
// the opposite order).  This is the same linear map as Eq. 6, evaluated with
// about a quarter of the operations; it relies on N(u)^-1 = N(-u).
//
// Vectorisation.  A warp owns 32*V consecutive nodes of one row; each lane
// loads V contiguous values of every plane with one 16-byte (8-byte for
// 16-bit storage) load.  The x-shift of the pull is done with one warp
// shuffle per plane; lanes 0 and 31 fetch the single value that crosses the
// warp boundary.  Nodes on box edges and next to solids take a fix-up path.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "clbm_internal.h"

namespace clbm {

constexpr int kStepThreads = 128;
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------------------
// Lattice (Eq. 3)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex_of(int d) {
  return (d == 1 || d == 5 || d == 8) ? 1 : ((d == 3 || d == 6 || d == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int d) {
  return (d == 2 || d == 5 || d == 6) ? 1 : ((d == 4 || d == 7 || d == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int d) {
  return d == 0 ? 0 : (d <= 4 ? ((d + 1) % 4) + 1 : ((d - 5 + 2) % 4) + 5);
}
// box side crossed by the pull source of D2Q5 direction j: 1 -> x0, 2 -> y0, 3 -> x1, 4 -> y1
__host__ __device__ constexpr int side_of(int j) {
  return j == 1 ? 0 : (j == 2 ? 2 : (j == 3 ? 1 : 3));
}

// ---------------------------------------------------------------------------
// Storage formats
// ---------------------------------------------------------------------------
template <typename S>
struct Traits;
template <>
struct Traits<double> {
  using R = double;
  static constexpr int V = 2;
};
template <>
struct Traits<float> {
  using R = float;
  static constexpr int V = 4;
};
template <>
struct Traits<__half> {
  using R = float;
  static constexpr int V = 4;
};
template <>
struct Traits<__nv_bfloat16> {
  using R = float;
  static constexpr int V = 4;
};

__device__ __forceinline__ double to_r(double v) { return v; }
__device__ __forceinline__ float to_r(float v) { return v; }
__device__ __forceinline__ float to_r(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_r(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S, typename R>
__device__ __forceinline__ S from_r(R v);
template <>
__device__ __forceinline__ double from_r<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_r<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_r<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_r<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// Vector load / store of V consecutive elements as one naturally aligned
// access of V * sizeof(S) bytes (2 to 16 bytes).
template <int B>
struct RawOf;
template <>
struct RawOf<2> {
  using T = unsigned short;
};
template <>
struct RawOf<4> {
  using T = unsigned int;
};
template <>
struct RawOf<8> {
  using T = uint2;
};
template <>
struct RawOf<16> {
  using T = uint4;
};

template <typename S, int V, typename R>
__device__ __forceinline__ void ldv(const S* p, R (&o)[V]) {
  using Raw = typename RawOf<sizeof(S) * V>::T;
  const Raw r = *reinterpret_cast<const Raw*>(p);
  S e[V];
  memcpy(e, &r, sizeof(Raw));
#pragma unroll
  for (int k = 0; k < V; ++k) o[k] = to_r(e[k]);
}

template <typename S, int V, typename R>
__device__ __forceinline__ void stv(S* p, const R (&o)[V]) {
  using Raw = typename RawOf<sizeof(S) * V>::T;
  S e[V];
#pragma unroll
  for (int k = 0; k < V; ++k) e[k] = from_r<S, R>(o[k]);
  Raw r;
  memcpy(&r, e, sizeof(Raw));
  *reinterpret_cast<Raw*>(p) = r;
}

// ---------------------------------------------------------------------------
// Stochastic rounding of 16-bit stores.  Round-to-nearest storage of a state
// that changes little from step to step rounds the same way every step, and the
// bias accumulates; stochastic rounding makes each store unbiased.  The random
// bits come from a counter-based hash of (step, node, plane): the "lowbias32"
// integer mixer published by C. Wellons ("Prospecting for Hash Functions", 2018).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Hardware stochastic rounding of two floats into a packed 16-bit pair
// (cvt.rs, Blackwell): `lo` lands in the low half (the first element in
// memory), `hi` in the high half; rbits supplies the random bits.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float lo, float hi, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float lo, float hi, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}

template <typename S>
__device__ __forceinline__ uint32_t cvt_rs2(float lo, float hi, uint32_t r);
template <>
__device__ __forceinline__ uint32_t cvt_rs2<__half>(float lo, float hi, uint32_t r) {
  return cvt_rs_f16x2(lo, hi, r);
}
template <>
__device__ __forceinline__ uint32_t cvt_rs2<__nv_bfloat16>(float lo, float hi, uint32_t r) {
  return cvt_rs_bf16x2(lo, hi, r);
}

// Stochastically rounded store of V values (16-bit formats only).
template <typename S, int V>
__device__ __forceinline__ void stv_sr(S* p, const float (&o)[V], uint32_t r0, uint32_t r1, int sub) {
  static_assert(sizeof(S) == 2, "stochastic rounding applies to 16-bit storage");
  if constexpr (V == 1) {
    const uint32_t w = (sub & 2) ? r1 : r0;
    *reinterpret_cast<unsigned short*>(p) =
        (sub & 1) ? (unsigned short)(cvt_rs2<S>(0.0f, o[0], w) >> 16) : (unsigned short)(cvt_rs2<S>(o[0], 0.0f, w) & 0xFFFFu);
  } else if constexpr (V == 2) {
    *reinterpret_cast<unsigned int*>(p) = cvt_rs2<S>(o[0], o[1], (sub & 2) ? r1 : r0);
  } else {
    static_assert(V == 4, "16-bit tiles use 1, 2 or 4 nodes per lane");
    *reinterpret_cast<uint2*>(p) = make_uint2(cvt_rs2<S>(o[0], o[1], r0), cvt_rs2<S>(o[2], o[3], r1));
  }
}

// The random bits of a store depend on the step, the node and the plane only,
// whichever kernel updates the node: one key per group of four nodes x0 = x & ~3
// of a row (the full mixer of step and node), and per plane two words: one
// multiply-xorshift of the key plus a golden-ratio multiple of the plane, and one
// more multiply-xorshift of that word; word 0 rounds nodes x0, x0 + 1 (low, high
// half), word 1 nodes x0 + 2, x0 + 3.
__device__ __forceinline__ uint32_t sr_key(uint32_t seed, long long group_node) {
  return seed ^ mix32((uint32_t)group_node);
}
__device__ __forceinline__ void sr_words(uint32_t key, int q, uint32_t& r0, uint32_t& r1) {
  r0 = (key + 0x9E3779B9u * (uint32_t)(q + 1)) * 0x7feb352du;
  r0 ^= r0 >> 15;
  r1 = r0 * 0x846ca68bu;
  r1 ^= r1 >> 16;
}

// ---------------------------------------------------------------------------
// Constants in the compute type
// ---------------------------------------------------------------------------
template <typename R>
struct Co {
  R rho0, T0, s_nu, s_b, s3, s4, l1, l2;
  R rgb;   // rho0 * g beta
  R Fvx, Fvy, Q, hQ, cT2;
  R vhc;   // viscous source: Q_v = vhc (k~11^2 + (k~20 - k~02)^2 / 4) / rho^2
  CollideK<R> k;  // rates combined with the scalings of the relaxed form
};

template <typename R>
__host__ __device__ __forceinline__ Co<R> make_co(const DevCoef& c) {
  Co<R> o;
  if constexpr (std::is_same<R, float>::value) {  // rounded on the host
    o.k = c.kf;
    const CoefF32& f = c.f;
    o.rho0 = f.rho0;
    o.T0 = f.T0;
    o.s_nu = f.s_nu;
    o.s_b = f.s_b;
    o.s3 = f.s3;
    o.s4 = f.s4;
    o.l1 = f.l1;
    o.l2 = f.l2;
    o.rgb = f.rgb;
    o.Fvx = f.Fvx;
    o.Fvy = f.Fvy;
    o.Q = f.Q;
    o.hQ = f.hQ;
    o.cT2 = f.cT2;
    o.vhc = f.vhc;
  } else {
    o.k = c.kd;
    o.rho0 = (R)c.rho0;
    o.T0 = (R)c.T0;
    o.s_nu = (R)c.s_nu;
    o.s_b = (R)c.s_b;
    o.s3 = (R)c.s3;
    o.s4 = (R)c.s4;
    o.l1 = (R)c.l1;
    o.l2 = (R)c.l2;
    o.rgb = (R)(c.rho0 * c.gbeta);
    o.Fvx = (R)c.Fvx;
    o.Fvy = (R)c.Fvy;
    o.Q = (R)c.Q;
    o.hQ = (R)(0.5 * c.Q);
    o.cT2 = (R)c.cT2;
    // nu (D^2 + G^2) with G = -3 s_nu k~11/rho, D = -3 s_nu (k~20 - k~02)/(2 rho), nu = (1/s_nu - 1/2)/3
    o.vhc = (R)(c.vh ? 3.0 * c.s_nu * c.s_nu * (1.0 / c.s_nu - 0.5) : 0.0);
  }
  return o;
}

// ---------------------------------------------------------------------------
// 1-D central-moment transform over the velocities {-1, 0, +1} and back
// ---------------------------------------------------------------------------
template <typename R>
__host__ __device__ __forceinline__ void fwd1(R am, R a0, R ap, R u, R& c0, R& c1, R& c2) {
  c0 = am + a0 + ap;
  const R s = ap - am;
  c1 = s - u * c0;
  c2 = (ap + am) - (u + u) * s + u * u * c0;
}
// The same with c0 formed from the pair sum ap + am (one add fewer).
template <typename R>
__host__ __device__ __forceinline__ void fwd1q(R am, R a0, R ap, R u, R& c0, R& c1, R& c2) {
  const R q = ap + am;
  c0 = q + a0;
  const R s = ap - am;
  c1 = s - u * c0;
  c2 = q - (u + u) * s + u * u * c0;
}
// The same from the row's sum c0, difference ap - am and sum ap + am.
template <typename R>
__host__ __device__ __forceinline__ void fwd1p(R c0, R s, R q, R u, R& c1, R& c2) {
  c1 = s - u * c0;
  c2 = q - (u + u) * s + u * u * c0;
}
template <typename R>
__host__ __device__ __forceinline__ void inv1(R c0, R c1, R c2, R u, R& am, R& a0, R& ap) {
  const R r1 = c1 + u * c0;
  const R r2 = c2 + (u + u) * c1 + u * u * c0;
  a0 = c0 - r2;
  ap = R(0.5) * (r2 + r1);
  am = R(0.5) * (r2 - r1);
}
// inv1 from halved first- and second-order inputs, c1h = c1 / 2 and c2h =
// c2 / 2, with u2 = 2u, hu = u / 2, hu2 = u^2 / 2: h1 = r1 / 2 and h2 = r2 / 2
// come out directly, so the two halvings of inv1 are not needed.  Scaling by
// a power of two is exact, so the result is inv1's to rounding.
template <typename R>
__host__ __device__ __forceinline__ void inv1h(R c0, R c1h, R c2h, R u2, R hu, R hu2, R& am, R& a0,
                                               R& ap) {
  const R h1 = c1h + hu * c0;
  const R h2 = c2h + u2 * c1h + hu2 * c0;
  a0 = c0 - R(2) * h2;
  ap = h2 + h1;
  am = h2 - h1;
}

// ---------------------------------------------------------------------------
// Collision of one node, on deviations.  In: pre-collision deviations d, h.
// Out (in place): post-collision deviations.
// ---------------------------------------------------------------------------
// VH: add the viscous dissipation source Q_v (Sec. 3.2), read from the
// pre-collision non-equilibrium central moments; it is returned in qv.  The
// Boussinesq force uses T without Q_v/2 (Q_v needs u, which needs the force).
// The combined constants: from the host (HK), or formed here from the rates.
// The FP32-storage kernels, memory-bound, run 1-1.4 % faster as compiled with
// the latter and with the (k~20, k~02) block and the first thermal moments
// grouped as plain relaxations; the 16-bit and FP64 ones, bound by issue or by
// the FP64 pipe, with the former and the regrouped sums, which take fewer
// operations (measured A/B on one GB300).
template <typename R, bool HK>
__host__ __device__ __forceinline__ CollideK<R> collide_k(const Co<R>& c) {
  if constexpr (HK) {
    return c.k;
  } else {
    const R q4 = R(0.25), h = R(0.5), third = R(1.0 / 3.0);
    CollideK<R> k;
    k.hFx = h * c.Fvx;
    k.al = -(c.s_b + c.s_nu) * q4;
    k.be = (c.s_nu - c.s_b) * q4;
    k.snu4 = (R(1) - c.s_nu) * q4;
    k.snur4 = c.s_nu * c.rho0 * q4;
    k.s3m4 = (R(1) - c.s3) * q4;
    k.s3r4 = c.s3 * c.rho0 * q4;
    k.hs3q = (R(1) - h * c.s3) * third * q4;
    k.s4m4 = (R(1) - c.s4) * q4;
    k.s4r4 = c.s4 * c.rho0 * q4;
    k.s4n = c.s4 * R(1.0 / 36.0);
    k.s4r9 = c.s4 * c.rho0 * R(1.0 / 36.0);
    k.l1m2 = (R(1) - c.l1) * h;
    k.l1T2 = c.l1 * c.T0 * h;
    k.l2m2 = (R(1) - c.l2) * h;
    k.l2T2 = c.l2 * c.T0 * h;
    k.srcq2 = (R(1) - h * c.l2) * c.cT2 * h;
    k.srct2 = c.l2 * c.cT2 * h;
    return k;
  }
}

template <typename R, bool VH = false, bool HK = true>
__host__ __device__ __forceinline__ void collide(const Co<R>& c, R (&d)[9], R (&h)[5], R& qv) {
  const R third = R(1.0 / 3.0);
  // Eq. 25 (T - T0 = sum h + Q/2) and Eq. 2
  const R k20 = h[1] + h[3], k02 = h[2] + h[4];
  const R sh = (h[0] + k20) + k02;
  const R dT = sh + c.hQ;
  const R Fx = c.Fvx;
  const R Fy = c.Fvy + c.rgb * dT;
  // Eq. 12 (sum_i w_i e_i = 0, so the rest state adds nothing to j), from the
  // sums and differences of each velocity row, which the x-pass below reuses
  const R ms = d[8] - d[7], mq = d[8] + d[7];  // e_y = -1
  const R zs = d[1] - d[3], zq = d[1] + d[3];  // e_y =  0
  const R ps = d[5] - d[6], pq = d[5] + d[6];  // e_y = +1
  // row sums: from the pair sums (one add fewer each) where the kernels are
  // bound by issue, in the grouping the FP32-storage kernels run fastest with otherwise
  const R m0 = HK ? mq + d[4] : (d[7] + d[4]) + d[8];
  const R z0 = HK ? zq + d[0] : (d[3] + d[0]) + d[1];
  const R p0 = HK ? pq + d[2] : (d[6] + d[2]) + d[5];
  const R drho = (m0 + z0) + p0;
  const R rho = c.rho0 + drho;
  const R jx = (ms + zs) + ps;
  const R jy = p0 - m0;
  // FP32: the reciprocal to within 2 ulp (hardware approximation), which the
  // FP32 parity bound leaves ample room for; FP64: the exact quotient
  R inv_rho = R(1) / rho;
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<R, float>::value) inv_rho = __fdividef(1.0f, rho);
#endif
  const R hFx = R(0.5) * Fx, hFy = R(0.5) * Fy;
  const R ux = (jx + hFx) * inv_rho;
  const R uy = (jy + hFy) * inv_rho;

  // central moments of the deviations: x-pass per velocity row, then y-pass
  R xm1, xm2, xz1, xz2, xp1, xp2;
  fwd1p(m0, ms, mq, ux, xm1, xm2);  // e_y = -1
  fwd1p(z0, zs, zq, ux, xz1, xz2);  // e_y =  0
  fwd1p(p0, ps, pq, ux, xp1, xp2);  // e_y = +1
  R b01, b02, b10, b11, b12, b20, b21, b22;
  const R b00 = drho;
  fwd1p(drho, jy, p0 + m0, uy, b01, b02);
  if constexpr (HK) {
    fwd1q(xm1, xz1, xp1, uy, b10, b11, b12);
    fwd1q(xm2, xz2, xp2, uy, b20, b21, b22);
  } else {
    fwd1(xm1, xz1, xp1, uy, b10, b11, b12);
    fwd1(xm2, xz2, xp2, uy, b20, b21, b22);
  }

  // Eq. 7-10, minus the rest-state moments rho0 kappa_m(ux) kappa_n(uy),
  // kappa = (1, -u, 1/3 + u^2).  Each post-collision moment D_mn is formed
  // scaled by 2^-[m > 0] 2^-[n > 0] (H_mn; exact scalings folded into the
  // rates), the form the back-transformation inv1h takes on both passes.
  const R ux2 = ux * ux, uy2 = uy * uy;
  const R r0 = c.rho0;
  const CollideK<R> k = collide_k<R, HK>(c);
  const R H00 = b00;
  const R H10 = R(0.5) * b10 + k.hFx;  // D10 / 2, D10 = b10 + Fx
  const R H01 = R(0.5) * b01 + hFy;    // D01 / 2, D01 = b01 + Fy
  // the (k~20, k~02) block: with a = k~ - its equilibrium (a20, a02 below),
  // D20 = k~20 - a20 + ((1 - s_b)(a20 + a02) + (1 - s_nu)(a20 - a02)) / 2, so
  // D20 / 2 = b20 / 2 + al a20 + be a02 and D02 / 2 = b02 / 2 + be a20 + al a02
  const R tdr = third * drho;
  const R a20 = r0 * ux2 + b20 - tdr;
  const R a02 = r0 * uy2 + b02 - tdr;
  R H20, H02;  // D20 / 2, D02 / 2
  if constexpr (HK) {
    H20 = R(0.5) * b20 + k.al * a20 + k.be * a02;
    H02 = R(0.5) * b02 + k.be * a20 + k.al * a02;
  } else {  // the same sums grouped as the FP32-storage kernels run fastest
    const R sum = (R(1) - c.s_b) * R(0.25) * (a20 + a02);
    const R dif = k.snu4 * (a20 - a02);
    const R htdr = R(0.5) * tdr, hr0 = R(0.5) * r0;
    H20 = htdr - hr0 * ux2 + (sum + dif);
    H02 = htdr - hr0 * uy2 + (sum - dif);
  }
  const R H11 = k.snu4 * b11 - k.snur4 * (ux * uy);  // D11 / 4
  const R tx = third + ux2, ty = third + uy2;
  const R H21 = k.s3m4 * b21 + k.s3r4 * (tx * uy) + k.hs3q * Fy;  // D21 / 4
  const R H12 = k.s3m4 * b12 + k.s3r4 * (ux * ty) + k.hs3q * Fx;  // D12 / 4
  const R H22 = k.s4m4 * b22 - k.s4r4 * (third * (ux2 + uy2) + ux2 * uy2) + k.s4n * drho;  // D22 / 4
  R Qt = c.Q;
  qv = R(0);
  if constexpr (VH) {
    const R k11 = r0 * ux * uy + b11;
    const R kd = r0 * (ux2 - uy2) + (b20 - b02);
    qv = c.vhc * inv_rho * inv_rho * (k11 * k11 + R(0.25) * kd * kd);
    Qt = c.Q + qv;
  }

  // back-transformation: y-pass inverse per x-order (rows m = 1, 2 come out
  // halved, as the x-pass wants them), then x-pass inverse per row
  const R ux2x = ux + ux, uy2x = uy + uy;
  const R hux = R(0.5) * ux, huy = R(0.5) * uy;
  const R hux2 = hux * ux, huy2 = huy * uy;
  R ym0, yz0, yp0, ym1, yz1, yp1, ym2, yz2, yp2;
  inv1h(H00, H01, H02, uy2x, huy, huy2, ym0, yz0, yp0);
  inv1h(H10, H11, H12, uy2x, huy, huy2, ym1, yz1, yp1);
  inv1h(H20, H21, H22, uy2x, huy, huy2, ym2, yz2, yp2);
  inv1h(ym0, ym1, ym2, ux2x, hux, hux2, d[7], d[4], d[8]);
  inv1h(yz0, yz1, yz2, ux2x, hux, hux2, d[3], d[0], d[1]);
  inv1h(yp0, yp1, yp2, ux2x, hux, hux2, d[6], d[2], d[5]);

  // thermal (Eq. 15-20, 23-24) on deviations from w^T T0; kappa^T = (1, -u, cT2 + u^2)
  const R k10 = h[1] - h[3], k01 = h[2] - h[4];
  // (1 - l1)(k10 - ux sh) / 2 + l1 T0 ux / 2 = l1m2 k10 + ux (l1T2 - l1m2 sh)
  const R w1 = HK ? k.l1T2 - k.l1m2 * sh : R(0);
  const R t20 = k20 - (ux + ux) * k10 + ux2 * sh;
  const R t02 = k02 - (uy + uy) * k01 + uy2 * sh;
  const R dTt = VH ? sh + R(0.5) * Qt : dT;  // Eq. 25 with the total source
  // post-collision thermal moments, first and second order halved (G = E / 2)
  // so that the back-transformation needs no halving of its own
  const R E00 = sh + Qt;
  R G10, G01;
  if constexpr (HK) {
    G10 = k.l1m2 * k10 + ux * w1;
    G01 = k.l1m2 * k01 + uy * w1;
  } else {
    G10 = k.l1m2 * (k10 - ux * sh) + k.l1T2 * ux;
    G01 = k.l1m2 * (k01 - uy * sh) + k.l1T2 * uy;
  }
  const R src2h = k.srcq2 * Qt + k.srct2 * dTt;
  const R G20 = k.l2m2 * t20 - k.l2T2 * ux2 + src2h;
  const R G02 = k.l2m2 * t02 - k.l2T2 * uy2 + src2h;
  const R q10 = G10 + hux * E00, q01 = G01 + huy * E00;  // halves of the raw moments
  const R q20 = G20 + ux2x * G10 + hux2 * E00;
  const R q02 = G02 + uy2x * G01 + huy2 * E00;
  h[0] = E00 - R(2) * (q20 + q02);
  h[1] = q20 + q10;
  h[3] = q20 - q10;
  h[2] = q02 + q01;
  h[4] = q02 - q01;
}

template <typename R, bool HK = true>
__host__ __device__ __forceinline__ void collide_any(const Co<R>& c, bool vh, R (&d)[9], R (&h)[5],
                                                     R& qv) {
  if (vh)
    collide<R, true, HK>(c, d, h, qv);
  else
    collide<R, false, HK>(c, d, h, qv);
}

// Which constants the kernels of storage type S take (the same in every
// kernel of one storage type, so that they all compute the same numbers).
template <typename S>
constexpr bool kHostK = !std::is_same<S, float>::value;

// Pre-collision equilibrium deviations (central moments Eq. 9 and Eq. 19 minus
// the rest-state moments) at (rho, u, T).
template <typename R>
__host__ __device__ __forceinline__ void equilibrium(const Co<R>& c, R rho, R ux, R uy, R T, R (&d)[9],
                                            R (&h)[5]) {
  const R third = R(1.0 / 3.0);
  const R r0 = c.rho0, drho = rho - r0, ux2 = ux * ux, uy2 = uy * uy;
  const R E00 = drho, E10 = r0 * ux, E01 = r0 * uy;
  const R E20 = third * drho - r0 * ux2, E02 = third * drho - r0 * uy2;
  const R E11 = -r0 * ux * uy;
  const R E21 = r0 * (third + ux2) * uy, E12 = r0 * ux * (third + uy2);
  const R E22 = R(1.0 / 9.0) * drho - r0 * (third * (ux2 + uy2) + ux2 * uy2);
  R ym0, yz0, yp0, ym1, yz1, yp1, ym2, yz2, yp2;
  inv1(E00, E01, E02, uy, ym0, yz0, yp0);
  inv1(E10, E11, E12, uy, ym1, yz1, yp1);
  inv1(E20, E21, E22, uy, ym2, yz2, yp2);
  inv1(ym0, ym1, ym2, ux, d[7], d[4], d[8]);
  inv1(yz0, yz1, yz2, ux, d[3], d[0], d[1]);
  inv1(yp0, yp1, yp2, ux, d[6], d[2], d[5]);
  const R dT = T - c.T0;
  const R T0 = c.T0;
  const R e00 = dT, e10 = T0 * ux, e01 = T0 * uy;
  const R e20 = c.cT2 * dT - T0 * ux2, e02 = c.cT2 * dT - T0 * uy2;
  const R q10 = e10 + ux * e00, q01 = e01 + uy * e00;
  const R q20 = e20 + (ux + ux) * e10 + ux2 * e00;
  const R q02 = e02 + (uy + uy) * e01 + uy2 * e00;
  h[0] = e00 - q20 - q02;
  h[1] = R(0.5) * (q20 + q10);
  h[3] = R(0.5) * (q20 - q10);
  h[2] = R(0.5) * (q02 + q01);
  h[4] = R(0.5) * (q02 - q01);
}

// ---------------------------------------------------------------------------
// Wall temperature (Eq. 28), one-sided when the second node is missing
// ---------------------------------------------------------------------------
template <typename R>
__host__ __device__ __forceinline__ R wall_temperature(R b1, R b2, R b3, R ne, R T1, R T2, bool have2) {
  if (have2) return (R(9) * b1 * T1 - b1 * T2 + R(3) * ne * b3) / (R(8) * b1 + R(3) * ne * b2);
  return (R(2) * b1 * T1 + ne * b3) / (R(2) * b1 + ne * b2);
}

// Walls at the fraction q of a link (no counterpart in the paper; q = 1/2 is
// its half-way wall).  s = distance from the wall along the link into the
// fluid; the wall profile is the quadratic through (0, T_w), (q, T1),
// (1 + q, T2), i.e. q(1+q) dT/ds(0) = -(1+2q) T_w + (1+q)^2 T1 - q^2 T2, and
// dT/dn = -dT/ds(0) / (n.e).  T_w solves b1 dT/dn + b2 T_w = b3 (the line
// through (0, T_w), (q, T1) when T2 is missing).
template <typename R>
__host__ __device__ __forceinline__ R wall_temperature_q(R b1, R b2, R b3, R ne, R q, R T1, R T2, bool have2) {
  if (have2) {
    const R qq = q * (R(1) + q), p = R(1) + q;
    return (b3 * qq * ne + b1 * (p * p * T1 - q * q * T2)) / (b1 * (R(1) + R(2) * q) + b2 * qq * ne);
  }
  return (b3 * q * ne + b1 * T1) / (b1 + b2 * q * ne);
}

// dT/dn at such a wall from the same profile.
template <typename R>
__host__ __device__ __forceinline__ R wall_gradient_q(R ne, R q, R Tw, R T1, R T2, bool have2) {
  if (have2) {
    const R p = R(1) + q;
    return ((R(1) + R(2) * q) * Tw - p * p * T1 + q * q * T2) / (q * p * ne);
  }
  return (Tw - T1) / (q * ne);
}

// The profile's value at the link midpoint s = q - 1/2, which Eq. 26 then
// imposes there.  q >= 1/2 or a wall with a flux term (b1 > 0): interpolation
// weights of the quadratic through the wall and the nodes at q and 1 + q.
// q < 1/2 at a Dirichlet wall: the quadratic through the wall and the nodes
// at 1 + q and 2 + q instead (bounded weights as q -> 0, none on the node's
// own T1, which would feed back into the node).  Both exact for quadratic
// profiles; lines through the available points in thin fluid layers.
template <typename R>
__host__ __device__ __forceinline__ R midpoint_temperature_q(R q, R Tw, R T1, R T2, bool have2, R T3,
                                                             bool have3, bool dirichlet) {
  const R m = R(2) * q - R(1);  // 2 (q - 1/2)
  if (q >= R(0.5) || !dirichlet) {
    if (!have2) return Tw + (T1 - Tw) * m / (R(2) * q);
    const R p = R(1) + q;
    return R(3) / (R(4) * q * p) * Tw + R(3) * m / (R(4) * q) * T1 - m / (R(4) * p) * T2;
  }
  if (have2 && have3) {
    const R p1 = R(1) + q, p2 = R(2) + q;
    return R(15) / (R(4) * p1 * p2) * Tw + R(5) * m / (R(4) * p1) * T2 - R(3) * m / (R(4) * p2) * T3;
  }
  if (have2) return Tw + (T2 - Tw) * m / (R(2) * (R(1) + q));
  return Tw;
}

// T at a node from its post-collision thermal deviations: T = T0 + sum h* - Q/2,
// Q including the node's stored viscous source when that is enabled.
template <typename S, typename R>
__device__ __forceinline__ R node_T(const S* __restrict__ src, long long plane, long long idx,
                                    const Co<R>& c) {
  R s = to_r(src[9 * plane + idx]);
#pragma unroll
  for (int q = 10; q < 14; ++q) s += to_r(src[q * plane + idx]);
  R t = c.T0 + s - c.hQ;
  if (c.vhc != R(0)) t -= R(0.5) * to_r(src[14 * plane + idx]);
  return t;
}

// Fix-up of one node that touches a wall, a periodic seam or a solid.
template <typename S, bool MASK, typename R>
__device__ __forceinline__ void fixup(const DevGeom& g, const Co<R>& c, const S* __restrict__ src,
                                      int x, int y, uint16_t fl, R (&d)[9], R (&h)[5]) {
  const long long plane = g.plane;
  const long long own = (long long)y * g.pitch + x;
  const R T1 = node_T(src, plane, own, c);
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int ex = ex_of(j), ey = ey_of(j);
    int sx = x - ex, sy = y - ey;
    const bool outx = sx < 0 || sx >= g.nx;
    const bool ylow = sy < g.ylo, yhigh = sy >= g.yhi;
    // beyond the own rows: a box wall, the periodic seam, or a ghost row (read as is)
    const bool outy = (ylow || yhigh) && g.py;
    const bool boxwall = (outx && !g.px) || (ylow && g.ywlo) || (yhigh && g.ywhi);
    bool wall = boxwall;
    if (MASK) wall = wall || ((fl >> (j - 1)) & 1u);
    if (wall) {
      const int i = opp_of(j);
      // listed link of a masked lattice: its slot and wall fraction (1/2 otherwise)
      int slot = -1;
      R q = R(0.5);
      if (MASK && !boxwall && (fl & kFlagLinks)) {
        slot = g.slot[own];
        q = (R)g.lk_q[8 * slot + (i - 1)];
      }
      // second node x_f - e_i = x + e_j, away from the wall
      int x2 = x + ex, y2 = y + ey;
      bool have2 = true;
      if (x2 < 0 || x2 >= g.nx) {
        if (g.px)
          x2 = x2 < 0 ? x2 + g.nx : x2 - g.nx;
        else
          have2 = false;
      }
      if (y2 < g.ylo || y2 >= g.yhi) {
        if (g.py)
          y2 = y2 < 0 ? y2 + g.ny : y2 - g.ny;
        else if (y2 < g.ylo ? g.ywlo : g.ywhi)
          have2 = false;  // beyond a box wall (else: a ghost row)
      }
      const long long i2 = (long long)y2 * g.pitch + x2;
      if (MASK && have2) have2 = (g.flags[i2] & kFlagSolid) == 0;
      const R fi = to_r(src[i * plane + own]);
      if (q == R(0.5) || (q < R(0.5) && !have2)) {
        d[j] = fi;  // half-way bounce-back
        if (boxwall && g.moving) {
          // a moving box side (not in the paper; Ladd's bounce-back): the
          // reflected population gains -6 w_i rho0 (e_i . u_w), e_i = -e_j
          const int sd = (outx && !g.px) ? (sx < 0 ? 0 : 1) : (ylow ? 2 : 3);
          R uwx, uwy;
          if constexpr (std::is_same<R, float>::value) {
            uwx = g.side_uf[sd][0];
            uwy = g.side_uf[sd][1];
          } else {
            uwx = (R)g.side_u[sd][0];
            uwy = (R)g.side_u[sd][1];
          }
          const R w6 = j <= 4 ? R(6.0 / 9.0) : R(6.0 / 36.0);
          d[j] += w6 * c.rho0 * (R(ex) * uwx + R(ey) * uwy);
        }
      } else if (q < R(0.5)) {  // f_i* interpolated to the point 1 - 2q behind x_f
        d[j] = R(2) * q * fi + (R(1) - R(2) * q) * to_r(src[i * plane + i2]);
      } else {  // the reflected value, 2q - 1 beyond x_f, interpolated with f_j* at x_f
        d[j] = fi / (R(2) * q) + (R(2) * q - R(1)) / (R(2) * q) * to_r(src[j * plane + own]);
      }
      if (j <= 4) {
        R ne, b1, b2, b3;
        if (boxwall) {
          const int sd = side_of(j);
          ne = R(1);
          if constexpr (std::is_same<R, float>::value) {
            b1 = g.side_bf[sd][0];
            b2 = g.side_bf[sd][1];
            b3 = g.side_bf[sd][2];
          } else {
            b1 = (R)g.side_b[sd][0];
            b2 = (R)g.side_b[sd][1];
            b3 = (R)g.side_b[sd][2];
          }
        } else {
          const int s = slot >= 0 ? slot : g.slot[own];
          const int t = g.lk_tbc[4 * s + (i - 1)];
          ne = (R)g.lk_ne[4 * s + (i - 1)];
          b1 = (R)g.tbc[3 * t + 0];
          b2 = (R)g.tbc[3 * t + 1];
          b3 = (R)g.tbc[3 * t + 2];
        }
        const R T2 = have2 ? node_T(src, plane, i2, c) : R(0);
        R Tm;
        if (q == R(0.5)) {
          Tm = wall_temperature(b1, b2, b3, ne, T1, T2, have2);  // Eq. 28
        } else {
          const R Tw = wall_temperature_q(b1, b2, b3, ne, q, T1, T2, have2);
          const bool dirichlet = b1 == R(0);
          bool have3 = false;
          R T3 = R(0);
          if (q < R(0.5) && dirichlet && have2) {  // third node x + 2 e_j
            int x3 = x2 + ex, y3 = y2 + ey;
            have3 = true;
            if (x3 < 0 || x3 >= g.nx) {
              if (g.px)
                x3 = x3 < 0 ? x3 + g.nx : x3 - g.nx;
              else
                have3 = false;
            }
            if (y3 < g.ylo || y3 >= g.yhi) {
              if (g.py)
                y3 = y3 < 0 ? y3 + g.ny : y3 - g.ny;
              else if ((y3 < g.ylo ? g.ywlo : g.ywhi) || y3 < 0 || y3 >= g.ny)
                have3 = false;  // beyond a box wall (slabs reject links whose third node is not stored)
            }
            const long long i3 = (long long)y3 * g.pitch + x3;
            if (MASK && have3) have3 = (g.flags[i3] & kFlagSolid) == 0;
            if (have3) T3 = node_T(src, plane, i3, c);
          }
          Tm = midpoint_temperature_q(q, Tw, T1, T2, have2, T3, have3, dirichlet);
        }
        h[j] = -to_r(src[(9 + i) * plane + own]) + c.cT2 * (Tm - c.T0);  // Eq. 26
      }
    } else if (outx || outy) {  // periodic seam
      if (outx) sx = sx < 0 ? sx + g.nx : sx - g.nx;
      if (outy) sy = sy < 0 ? sy + g.ny : sy - g.ny;
      const long long s = (long long)sy * g.pitch + sx;
      d[j] = to_r(src[j * plane + s]);
      if (j <= 4) h[j] = to_r(src[(9 + j) * plane + s]);
    }
  }
}

// ---------------------------------------------------------------------------
// The fused step kernel
// ---------------------------------------------------------------------------
// Store of one value (stochastically rounded for 16-bit storage when asked).
template <typename S, typename R>
__device__ __forceinline__ void st1(S* p, R v, int stochastic, uint32_t key, int q, int sub) {
  if constexpr (sizeof(S) == 2) {
    if (stochastic) {
      uint32_t r0, r1;
      sr_words(key, q, r0, r1);
      const float o[1] = {v};
      stv_sr<S, 1>(p, o, r0, r1, sub);
      return;
    }
  }
  *p = from_r<S, R>(v);
}

// Interior update.  One warp updates the 32 * V nodes x = xw .. xw + 32V - 1
// of row y (each lane owns V consecutive nodes); all 32 lanes must call it
// together.  Every node is pulled and collided as if it were an interior
// fluid node: rows beyond a non-periodic edge are clamped and the ±1 x-shift
// at the row ends reads a neighbour, so box edges, periodic seams and nodes
// next to solids come out wrong here and are recomputed afterwards by the
// boundary kernel from its precomputed node list.  Keeping the walls out of
// this kernel keeps its warps free of divergent wall code.
template <typename S, int V, bool SKIP_EDGES = false, bool VH = false, bool SKIP_DEAD = true,
          bool MASKSTORE = false>
__device__ __forceinline__ void step_tile(const DevGeom& g, const Co<typename Traits<S>::R>& c,
                                          const S* __restrict__ src, S* __restrict__ dst, int y,
                                          int xw, int lane, uint32_t seed, int stochastic,
                                          bool mixed = false) {
  using R = typename Traits<S>::R;
  const int x0 = xw + lane * V;
  const long long plane = g.plane;

  int ym = y - 1, yp = y + 1;  // rows the e_y = +1 / -1 populations come from
  if (g.py) {
    ym = ym < 0 ? g.ny - 1 : ym;
    yp = yp >= g.ny ? 0 : yp;
  } else {
    ym = ym < 0 ? 0 : ym;
    yp = yp >= g.ny ? g.ny - 1 : yp;
  }
  const int xl = x0 > 0 ? x0 - 1 : 0;
  const int xr = x0 + V < g.pitch ? x0 + V : g.pitch - 1;
  // SKIP_DEAD: a lane wholly beyond the row (x0 >= nx: the pitch padding of
  // the last tile) neither loads nor stores; it still takes part in the
  // shuffles, and the only value it passes on (to node nx - 1 from x = nx)
  // belongs to the last column, which the boundary update recomputes.  (The
  // 16-bit single-lattice kernels leave it off: the extra live state costs
  // them register spills, more than the padding they would skip.)
  const bool live = !SKIP_DEAD || x0 < g.nx;

  R v[14][V];
#pragma unroll
  for (int q = 0; q < 14; ++q) {
    const int dir = q < 9 ? q : q - 9;
    const int ex = ex_of(dir), ey = ey_of(dir);
    const int row = ey > 0 ? ym : (ey < 0 ? yp : y);
    const S* base = src + q * plane + (long long)row * g.pitch;
    R t[V];
    if (live) {
      ldv<S, V>(base + x0, t);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) t[k] = R(0);
    }
    if (ex == 0) {
#pragma unroll
      for (int k = 0; k < V; ++k) v[q][k] = t[k];
    } else if (ex > 0) {  // value from x - 1
      R left = __shfl_up_sync(0xffffffffu, t[V - 1], 1);
      if (lane == 0) left = to_r(base[xl]);
      v[q][0] = left;
#pragma unroll
      for (int k = 1; k < V; ++k) v[q][k] = t[k - 1];
    } else {  // value from x + 1
      R right = __shfl_down_sync(0xffffffffu, t[0], 1);
      if (lane == 31 && live) right = to_r(base[xr]);
#pragma unroll
      for (int k = 0; k < V - 1; ++k) v[q][k] = t[k + 1];
      v[q][V - 1] = right;
    }
  }

  R qv[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    R d[9], h[5];
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = v[q][k];
#pragma unroll
    for (int q = 0; q < 5; ++q) h[q] = v[9 + q][k];
    collide<R, VH, kHostK<S>>(c, d, h, qv[k]);
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q][k] = d[q];
#pragma unroll
    for (int q = 0; q < 5; ++q) v[9 + q][k] = h[q];
  }

  if (!live) return;
  S* out = dst + (long long)y * g.pitch + x0;
  if constexpr (MASKSTORE) {
    // a tile holding flagged nodes (solid, or fluid next to a wall) leaves them,
    // and the edge columns, to the boundary update of the same launch
    if (mixed) {
      const uint16_t* fp = g.flags + (long long)y * g.pitch + x0;
      uint32_t skip = 0;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int x = x0 + k;
        if (fp[k] != 0 || x == 0 || x == g.nx - 1) skip |= 1u << k;
      }
      if (skip) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
          if ((skip >> k) & 1u) continue;
          const int x = x0 + k;
          if constexpr (VH) out[14 * plane + k] = from_r<S, R>(qv[k]);
          const uint32_t key = sr_key(seed, (long long)(y + g.yoff) * g.pitch + (x & ~3));
#pragma unroll
          for (int q = 0; q < 14; ++q) st1<S, R>(out + q * plane + k, v[q][k], stochastic, key, q, x & 3);
        }
        return;
      }
    }
  }
  if constexpr (VH) {  // the viscous source of this step, read back with T (15th plane)
    if constexpr (SKIP_EDGES) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int x = x0 + k;
        if (x != 0 && x != g.nx - 1) out[14 * plane + k] = from_r<S, R>(qv[k]);
      }
    } else {
      stv<S, V>(out + 14 * plane, qv);
    }
  }
  if constexpr (SKIP_EDGES) {
    // leave the first and last column to the boundary update running alongside
    if (x0 == 0 || (x0 <= g.nx - 1 && g.nx - 1 < x0 + V)) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int x = x0 + k;
        if (x == 0 || x == g.nx - 1) continue;
        const uint32_t key = sr_key(seed, (long long)(y + g.yoff) * g.pitch + (x & ~3));
#pragma unroll
        for (int q = 0; q < 14; ++q) st1<S, R>(out + q * plane + k, v[q][k], stochastic, key, q, x & 3);
      }
      return;
    }
  }
  if constexpr (sizeof(S) == 2) {
    if (stochastic) {
      // x0 is a multiple of V (tiles start at multiples of 32 V nodes)
      const uint32_t key = sr_key(seed, (long long)(y + g.yoff) * g.pitch + (x0 & ~3));
#pragma unroll
      for (int q = 0; q < 14; ++q) {
        uint32_t r0, r1;
        sr_words(key, q, r0, r1);
        stv_sr<S, V>(out + q * plane, v[q], r0, r1, x0 & 3);
      }
      return;
    }
  }
#pragma unroll
  for (int q = 0; q < 14; ++q) stv<S, V>(out + q * plane, v[q]);
}

// Boundary update of node index i (pitch layout): pull with clamped indices,
// then the fix-up applies bounce-back, Eq. 26-28 and periodic wrapping.
template <typename S, bool MASK>
__device__ __forceinline__ void step_node(const DevGeom& g, const Co<typename Traits<S>::R>& c,
                                          const S* __restrict__ src, S* __restrict__ dst,
                                          long long i, uint32_t seed, int stochastic) {
  using R = typename Traits<S>::R;
  const int y = (int)(i / g.pitch), x = (int)(i - (long long)y * g.pitch);
  const long long plane = g.plane;
  R d[9], h[5];
#pragma unroll
  for (int q = 0; q < 14; ++q) {
    const int dir = q < 9 ? q : q - 9;
    int sx = x - ex_of(dir), sy = y - ey_of(dir);
    sx = sx < 0 ? 0 : (sx >= g.nx ? g.nx - 1 : sx);
    sy = sy < 0 ? 0 : (sy >= g.ny ? g.ny - 1 : sy);
    const R val = to_r(src[q * plane + (long long)sy * g.pitch + sx]);
    if (q < 9)
      d[q] = val;
    else
      h[q - 9] = val;
  }
  const uint16_t fl = MASK ? g.flags[i] : (uint16_t)0;
  fixup<S, MASK>(g, c, src, x, y, fl, d, h);
  R qv;
  const bool vh = c.vhc != R(0);
  collide_any<R, kHostK<S>>(c, vh, d, h, qv);
  if (vh) dst[14 * plane + i] = from_r<S, R>(qv);
  // global node index of the group of four (the pitch is a multiple of 4)
  const uint32_t key = sr_key(seed, i + (long long)g.yoff * g.pitch - (x & 3));
#pragma unroll
  for (int q = 0; q < 14; ++q) st1<S, R>(dst + q * plane + i, q < 9 ? d[q] : h[q - 9], stochastic, key, q, x & 3);
}

// Stochastic-rounding key of a step: from the host value, or from the device
// step counter when the launch is part of a replayed graph.
__device__ __forceinline__ uint32_t step_seed(const StepArgs& a) {
  if (!a.stochastic) return 0u;
  if (!a.tdev) return a.seed;
  const long long t = *a.tdev + a.tstep;
  return (uint32_t)(t * 0x9E3779B1ull) ^ (uint32_t)(t >> 32);
}

// One launch = the interior update of one time step of one lattice.
template <typename S, bool VH>
__global__ void __launch_bounds__(kStepThreads) step_kernel(const StepArgs a) {
  using R = typename Traits<S>::R;
  constexpr int V = Traits<S>::V;
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * (kStepThreads / 32) + (threadIdx.x >> 5);
  const int xw = warp * 32 * V;
  if (xw >= a.g.nx) return;  // whole warps only: the shuffles need all 32 lanes
  const int y = a.g.ylo + (a.reverse ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y);
  // a tile of solid nodes only: nothing reads them, so neither load nor store
  if (a.g.tile_fluid && !a.g.tile_fluid[(long long)y * a.g.tiles_per_row + warp]) return;
  const Co<R> c = make_co<R>(a.c);
  step_tile<S, V, false, VH, sizeof(S) != 2>(a.g, c, static_cast<const S*>(a.src),
                                             static_cast<S*>(a.dst), y, xw, lane, step_seed(a),
                                             a.stochastic);
}

// The boundary nodes of the same step (launched after step_kernel).
template <typename S, bool MASK>
__global__ void __launch_bounds__(kRedThreads) boundary_kernel(const StepArgs a) {
  using R = typename Traits<S>::R;
  const Co<R> c = make_co<R>(a.c);
  const uint32_t seed = step_seed(a);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.nb; k += gridDim.x * blockDim.x)
    step_node<S, MASK>(a.g, c, static_cast<const S*>(a.src), static_cast<S*>(a.dst), a.bnodes[k],
                       seed, a.stochastic);
}

// Box lattices (no mask): interior and boundary nodes are disjoint, so one
// launch does both.  The first nbb blocks update the boundary list (first and
// last column, first and last row of a non-periodic y axis); the others are
// interior tiles of rows that are not boundary rows, which skip the first and
// last column.  The latency-bound boundary work then overlaps the streaming
// interior work instead of following it.
// Blocks per SM the register budget is cut for: five (96 registers) where the
// step is memory-bound (FP32, FP64 storage); six (80 registers, a 44-byte
// spill) for 16-bit storage, which is bound by issue and memory latency and
// gains 2-6 % from the extra warps (measured A/B on one GB300).
template <typename S>
constexpr int kStepBlocks = sizeof(S) == 2 ? 6 : 5;

template <typename S, bool VH, bool MASKED = false>
__global__ void __launch_bounds__(kStepThreads, kStepBlocks<S>) step_fused_kernel(const StepArgs a, int nbb,
                                                                                int xblocks, int y0, int rows) {
  using R = typename Traits<S>::R;
  constexpr int V = Traits<S>::V;
  const Co<R> c = make_co<R>(a.c);
  if ((int)blockIdx.x < nbb) {
    const int k = blockIdx.x * kStepThreads + threadIdx.x;
    if (k < a.nb)
      step_node<S, MASKED>(a.g, c, static_cast<const S*>(a.src), static_cast<S*>(a.dst), a.bnodes[k],
                           step_seed(a), a.stochastic);
    return;
  }
  const int b = blockIdx.x - nbb;
  const int row = b / xblocks;
  const int y = y0 + (a.reverse ? rows - 1 - row : row);
  const int lane = threadIdx.x & 31;
  const int warp = (b % xblocks) * (kStepThreads / 32) + (threadIdx.x >> 5);
  const int xw = warp * 32 * V;
  if (xw >= a.g.nx) return;  // whole warps only
  if constexpr (MASKED) {  // tile classes: 0 no fluid, 1 unflagged fluid, 2 holds flagged nodes
    const uint8_t cls = a.g.tile_fluid[(long long)y * a.g.tiles_per_row + warp];
    if (!cls) return;
    step_tile<S, V, true, VH, sizeof(S) != 2, true>(a.g, c, static_cast<const S*>(a.src),
                                                    static_cast<S*>(a.dst), y, xw, lane, step_seed(a),
                                                    a.stochastic, cls == 2);
  } else {
    step_tile<S, V, true, VH, sizeof(S) != 2>(a.g, c, static_cast<const S*>(a.src),
                                              static_cast<S*>(a.dst), y, xw, lane, step_seed(a),
                                              a.stochastic);
  }
}

// ---------------------------------------------------------------------------
// Initialisation: equilibrium at the given fields, then one collision (the
// stored state is post-collision).
// ---------------------------------------------------------------------------
template <typename S>
__global__ void init_kernel(const DevGeom g, const DevCoef cf, S* __restrict__ dst,
                            const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, const double* __restrict__ T) {
  using R = typename Traits<S>::R;
  const Co<R> c = make_co<R>(cf);
  // one thread per column of the padded rows (every stored row, ghost rows too)
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.pitch) return;
  for (int y = (int)blockIdx.y; y < g.ny; y += (int)gridDim.y) {
    const long long i = (long long)y * g.pitch + x;
    R d[9], h[5];
    bool active = x < g.nx && y >= g.ylo && y < g.yhi;  // own rows (ghost rows: zero until exchanged)
    if (g.flags) active = active && !(g.flags[i] & kFlagSolid);
    if (active) {
      const long long k = (long long)(y - g.ylo) * g.nx + x;
      const R r = rho ? (R)rho[k] : c.rho0;
      const R u = ux ? (R)ux[k] : R(0);
      const R w = uy ? (R)uy[k] : R(0);
      const R t = T ? (R)T[k] : c.T0;
      equilibrium(c, r, u, w, t, d, h);
      R qv;
      collide_any<R, kHostK<S>>(c, cf.vh != 0, d, h, qv);
      if (cf.vh) dst[14 * g.plane + i] = from_r<S, R>(qv);
    } else {
      if (cf.vh) dst[14 * g.plane + i] = from_r<S, R>(R(0));
#pragma unroll
      for (int q = 0; q < 9; ++q) d[q] = R(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) h[q] = R(0);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) dst[q * g.plane + i] = from_r<S, R>(d[q]);
#pragma unroll
    for (int q = 0; q < 5; ++q) dst[(9 + q) * g.plane + i] = from_r<S, R>(h[q]);
  }
}

// ---------------------------------------------------------------------------
// Macroscopic fields from a post-collision state, in FP64:
//   rho = rho0 + sum d*, T = T0 + sum h* - Q/2, u = (sum d* e - F/2)/rho
// (the collision adds F to the first moments and Q to the zeroth thermal one).
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ void node_macros(const DevCoef& c, const S* __restrict__ b,
                                            long long plane, long long i, double& rho, double& ux,
                                            double& uy, double& T) {
  double f[9], s = 0.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) f[q] = (double)to_r(b[q * plane + i]);
#pragma unroll
  for (int q = 9; q < 14; ++q) s += (double)to_r(b[q * plane + i]);
  const double qv = c.vh ? (double)to_r(b[14 * plane + i]) : 0.0;
  T = c.T0 + s - 0.5 * (c.Q + qv);
  // the Boussinesq force uses T without the viscous source's half
  const double Fx = c.Fvx, Fy = c.Fvy + c.rho0 * c.gbeta * (T - 0.5 * qv - c.T0);
  const double dr = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  rho = c.rho0 + dr;
  const double jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const double jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  ux = (jx - 0.5 * Fx) / rho;
  uy = (jy - 0.5 * Fy) / rho;
}

// The same in the collision's arithmetic R (FP32 below FP64 storage).
template <typename S, typename R>
__device__ __forceinline__ void node_macros_r(const Co<R>& c, bool vh, const S* __restrict__ b,
                                              long long plane, long long i, R& rho, R& ux, R& uy,
                                              R& T) {
  R f[9], s = R(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) f[q] = (R)to_r(b[q * plane + i]);
#pragma unroll
  for (int q = 9; q < 14; ++q) s += (R)to_r(b[q * plane + i]);
  const R qv = vh ? (R)to_r(b[14 * plane + i]) : R(0);
  T = c.T0 + s - R(0.5) * (c.Q + qv);
  const R Fx = c.Fvx, Fy = c.Fvy + c.rgb * (T - R(0.5) * qv - c.T0);
  const R dr = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  rho = c.rho0 + dr;
  const R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const R jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const R inv = R(1) / rho;
  ux = (jx - R(0.5) * Fx) * inv;
  uy = (jy - R(0.5) * Fy) * inv;
}

// Sums of one node's stored deviations in the arithmetic R: the zeroth and
// first moments of d*, the zeroth moment of h* and the viscous source slot.
template <typename R>
struct NodeSums {
  R dr, jx, jy, s, qv;
};

template <typename R, typename S>
__device__ __forceinline__ NodeSums<R> node_sums(const S* __restrict__ b, long long plane,
                                                 long long i, bool vh) {
  R f[9];
  NodeSums<R> o;
  o.s = R(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) f[q] = (R)to_r(b[q * plane + i]);
#pragma unroll
  for (int q = 9; q < 14; ++q) o.s += (R)to_r(b[q * plane + i]);
  o.qv = vh ? (R)to_r(b[14 * plane + i]) : R(0);
  o.dr = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  o.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  o.jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  return o;
}

// The reported fields of one fluid node.  FP64 storage: all in FP64.  Below
// it the sums and the velocity take the collision's FP32 arithmetic (the
// precision the state carries) and only the offsets rho0 and T0 are added in
// FP64, so that the deviations of rho and T keep every bit the sums have.
// Fy uses T - qv/2 - T0 = sum h* - Q/2 - qv, without the cancellation of T0.
template <typename S>
__device__ __forceinline__ void node_fields(const DevCoef& c, const Co<typename Traits<S>::R>& co,
                                            const S* __restrict__ b, long long plane, long long i,
                                            double& rho, double& ux, double& uy, double& T) {
  using R = typename Traits<S>::R;
  if constexpr (std::is_same<R, double>::value) {
    node_macros(c, b, plane, i, rho, ux, uy, T);
  } else {
    const NodeSums<R> n = node_sums<R>(b, plane, i, c.vh != 0);
    const R Fy = co.Fvy + co.rgb * (n.s - R(0.5) * co.Q - n.qv);
    const R inv = R(1) / (co.rho0 + n.dr);
    ux = (double)((n.jx - R(0.5) * co.Fvx) * inv);
    uy = (double)((n.jy - R(0.5) * Fy) * inv);
    rho = c.rho0 + (double)n.dr;
    T = c.T0 + (double)(n.s - R(0.5) * (co.Q + n.qv));
  }
}

// One thread per column x of the own rows; the rows are strided over gridDim.y.
template <typename S>
__global__ void moments_kernel(const DevGeom g, const DevCoef c, const S* __restrict__ b,
                               double* __restrict__ rho, double* __restrict__ ux,
                               double* __restrict__ uy, double* __restrict__ T) {
  using R = typename Traits<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const Co<R> co = make_co<R>(c);
  for (int y = g.ylo + (int)blockIdx.y; y < g.yhi; y += (int)gridDim.y) {
    const long long i = (long long)y * g.pitch + x;
    const long long k = (long long)(y - g.ylo) * g.nx + x;  // own-row index
    double r = 0, u = 0, v = 0, t = 0;
    if (!g.flags || !(g.flags[i] & kFlagSolid)) node_fields<S>(c, co, b, g.plane, i, r, u, v, t);
    if (rho) rho[k] = r;
    if (ux) ux[k] = u;
    if (uy) uy[k] = v;
    if (T) T[k] = t;
  }
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions: each block writes its partial sums; a single
// block adds the partials in index order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int W>
__device__ __forceinline__ void block_sum_store(double (&acc)[W], double* out) {
  __shared__ double sh[kRedThreads / 32][W];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const double s = warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < W) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Squared one-step changes and squares of T, ux, uy at one fluid node, added
// to a[0..5] (a[6] counts a non-finite field).  FP64 storage: the fields of
// both states in FP64 and their differences.  Below it, in FP32 from the
// differences of the stored values, which are exact where the state barely
// moves (the differences of FP32 fields near rho0 and T0 would be rounded to
// their ulp):
//   dT = sum dh* - dqv/2,  du = (da - u(t-1) d(drho)) / rho(t),
// a = j - F/2 with dFy = rgb (sum dh* - dqv) (a(t) = a(t-1) + da, rho(t) =
// rho(t-1) + d(drho)).  Fields beyond ~1e19 overflow the FP32 squares and
// count as unstable, as a non-finite field does.
template <typename S, typename R>
__device__ __forceinline__ void residual_terms(const DevCoef& c, const Co<R>& co,
                                               const S* __restrict__ cur,
                                               const S* __restrict__ prev, long long plane,
                                               long long i, R (&a)[7]) {
  if constexpr (std::is_same<R, double>::value) {
    double r1, u1, v1, t1, r0, u0, v0, t0;
    node_macros(c, cur, plane, i, r1, u1, v1, t1);
    node_macros(c, prev, plane, i, r0, u0, v0, t0);
    a[0] += (t1 - t0) * (t1 - t0);
    a[1] += t1 * t1;
    a[2] += (u1 - u0) * (u1 - u0);
    a[3] += u1 * u1;
    a[4] += (v1 - v0) * (v1 - v0);
    a[5] += v1 * v1;
    if (!isfinite(r1) || !isfinite(u1) || !isfinite(v1) || !isfinite(t1)) a[6] += 1.0;
  } else {
    const bool vh = c.vh != 0;
    R f1[9], f0[9], df[9], s1 = R(0), s0 = R(0), ds = R(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      f1[q] = (R)to_r(cur[q * plane + i]);
      f0[q] = (R)to_r(prev[q * plane + i]);
      df[q] = f1[q] - f0[q];
    }
#pragma unroll
    for (int q = 9; q < 14; ++q) {
      const R h1 = (R)to_r(cur[q * plane + i]), h0 = (R)to_r(prev[q * plane + i]);
      s1 += h1;
      s0 += h0;
      ds += h1 - h0;
    }
    const R q1 = vh ? (R)to_r(cur[14 * plane + i]) : R(0);
    const R q0 = vh ? (R)to_r(prev[14 * plane + i]) : R(0);
    auto zeroth = [](const R* f) {
      return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    };
    auto first_x = [](const R* f) { return (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]); };
    auto first_y = [](const R* f) { return (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]); };
    const R dq = q1 - q0;
    const R t1 = co.T0 + (s1 - R(0.5) * (co.Q + q1));
    const R dT = ds - R(0.5) * dq;
    const R Fy1 = co.Fvy + co.rgb * (s1 - R(0.5) * co.Q - q1);
    const R Fy0 = co.Fvy + co.rgb * (s0 - R(0.5) * co.Q - q0);
    const R rho1 = co.rho0 + zeroth(f1), rho0 = co.rho0 + zeroth(f0), ddr = zeroth(df);
    const R inv1 = R(1) / rho1, inv0 = R(1) / rho0;
    const R u1 = (first_x(f1) - R(0.5) * co.Fvx) * inv1;
    const R v1 = (first_y(f1) - R(0.5) * Fy1) * inv1;
    const R u0 = (first_x(f0) - R(0.5) * co.Fvx) * inv0;
    const R v0 = (first_y(f0) - R(0.5) * Fy0) * inv0;
    const R dax = first_x(df), day = first_y(df) - R(0.5) * co.rgb * (ds - dq);
    const R du = (dax - u0 * ddr) * inv1, dv = (day - v0 * ddr) * inv1;
    a[0] += dT * dT;
    a[1] += t1 * t1;
    a[2] += du * du;
    a[3] += u1 * u1;
    a[4] += dv * dv;
    a[5] += v1 * v1;
    if (!isfinite(rho1) || !isfinite(u1) || !isfinite(v1) || !isfinite(t1)) a[6] += R(1);
  }
}

// Work items are (own row, span of kRedThreads * kResV columns); a thread
// sums its kResV nodes of an item in R and adds that to its FP64 sums.  The
// items' partial sums depend on the row and columns alone, so slabs of one
// lattice add the same numbers (in another order).
constexpr int kResV = 8;

template <typename S>
__global__ void __launch_bounds__(kRedThreads)
    residual_kernel(const DevGeom g, const DevCoef c, const S* __restrict__ cur,
                    const S* __restrict__ prev, double* __restrict__ partials) {
  using R = typename Traits<S>::R;
  const Co<R> co = make_co<R>(c);
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  constexpr int span = kRedThreads * kResV;
  const int xch = (g.nx + span - 1) / span;
  const long long items = (long long)(g.yhi - g.ylo) * xch;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int yr = (int)(it / xch);
    const int x0 = (int)(it - (long long)yr * xch) * span + (int)threadIdx.x;
    const long long row = (long long)(yr + g.ylo) * g.pitch;
    R a[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < kResV; ++j) {
      const int x = x0 + j * kRedThreads;
      if (x < g.nx && !(g.flags && (g.flags[row + x] & kFlagSolid)))
        residual_terms<S, R>(c, co, cur, prev, g.plane, row + x, a);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] += (double)a[q];
  }
  block_sum_store<8>(acc, partials + 8 * blockIdx.x);
}

// Conservation sums over the fluid nodes of the stored post-collision
// deviations, accumulated in FP64: Sum_i d_i, Sum_i d_i e_ix, Sum_i d_i e_iy,
// Sum_j h_j, the fluid-node count and the count of non-finite values.
template <typename S>
__global__ void __launch_bounds__(kRedThreads)
    totals_kernel(const DevGeom g, const S* __restrict__ b, double* __restrict__ partials) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long n = (long long)(g.yhi - g.ylo) * g.nx;  // own rows
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int yl = (int)(k / g.nx), x = (int)(k - (long long)yl * g.nx);
    const long long i = (long long)(yl + g.ylo) * g.pitch + x;
    if (g.flags && (g.flags[i] & kFlagSolid)) continue;
    double f[9], s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = (double)to_r(b[q * g.plane + i]);
#pragma unroll
    for (int q = 9; q < 14; ++q) s += (double)to_r(b[q * g.plane + i]);
    const double m = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const double jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const double jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    acc[0] += m;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += s;
    acc[4] += 1.0;
    if (!isfinite(m) || !isfinite(jx) || !isfinite(jy) || !isfinite(s)) acc[5] += 1.0;
  }
  block_sum_store<8>(acc, partials + 8 * blockIdx.x);
}

template <typename S>
__global__ void __launch_bounds__(kRedThreads)
    nusselt_kernel(const DevGeom g, const DevCoef c, const S* __restrict__ b,
                   const NuLink* __restrict__ links, int nlinks, double* __restrict__ partials) {
  double acc[2] = {0, 0};
  const Co<double> cd = make_co<double>(c);
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += gridDim.x * blockDim.x) {
    const NuLink L = links[l];
    const double T1 = node_T(b, g.plane, L.own, cd);
    const bool have2 = L.second >= 0;
    const double T2 = have2 ? node_T(b, g.plane, L.second, cd) : 0.0;
    double grad;
    if (L.q == 0.5) {
      const double Tw = wall_temperature(L.b1, L.b2, L.b3, L.ne, T1, T2, have2);
      grad = have2 ? (8.0 * Tw - 9.0 * T1 + T2) / (3.0 * L.ne)  // Eq. 27
                   : (Tw - T1) / (0.5 * L.ne);
    } else {  // wall off the link midpoint
      const double Tw = wall_temperature_q(L.b1, L.b2, L.b3, L.ne, L.q, T1, T2, have2);
      grad = wall_gradient_q(L.ne, L.q, Tw, T1, T2, have2);
    }
    acc[0] += grad;
    acc[1] += isfinite(grad) ? 0.0 : 1.0;
  }
  block_sum_store<2>(acc, partials + 2 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched solves: the step kernel walks a tile list with a persistent grid
// (each warp takes tiles w, w + #warps, ...), so the same launch serves any
// number of active lattices; the list is rebuilt on the device as lattices
// converge.
// ---------------------------------------------------------------------------
// Each warp takes one contiguous chunk of the tile list (tiles are ordered by
// lattice, row, x), so it stays on one lattice for many tiles; the lattice's
// descriptor is copied into a per-warp shared-memory slot when it changes and
// read from there, instead of chasing it through global memory on every tile.
// Tiles cover only the rows that are not boundary rows and skip the first and
// last column: those nodes belong to the boundary launch that follows.
template <typename S, int V, bool VH>
__global__ void __launch_bounds__(kStepThreads, 4)
    batch_step_kernel(const BatchLat* __restrict__ lats, const int4* __restrict__ tiles,
                      const int* __restrict__ count, int parity, const long long* __restrict__ tptr,
                      int tstep, int stochastic) {
  using R = typename Traits<S>::R;
  static_assert(sizeof(BatchLat) % 8 == 0, "descriptor is copied in 8-byte words");
  __shared__ BatchLat slot[kStepThreads / 32];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long n = *count;
  const long long nw = (long long)gridDim.x * (kStepThreads / 32);
  const long long chunk = (n + nw - 1) / nw;
  const long long begin = ((long long)blockIdx.x * (kStepThreads / 32) + wib) * chunk;
  const long long end = begin + chunk < n ? begin + chunk : n;
  uint32_t seed = 0;
  if (stochastic) {
    const long long t = *tptr + tstep;
    seed = (uint32_t)(t * 0x9E3779B1ull) ^ (uint32_t)(t >> 32);
  }
  BatchLat& L = slot[wib];
  int cur = -1;
  Co<R> c;
  for (long long w = begin; w < end; ++w) {
    const int4 tl = tiles[w];
    if (tl.x != cur) {
      __syncwarp();
      const unsigned long long* from = reinterpret_cast<const unsigned long long*>(lats + tl.x);
      unsigned long long* to = reinterpret_cast<unsigned long long*>(&L);
      for (int k = lane; k < (int)(sizeof(BatchLat) / 8); k += 32) to[k] = from[k];
      __syncwarp();
      cur = tl.x;
      c = make_co<R>(L.c);
    }
    step_tile<S, V, true, VH>(L.g, c, static_cast<const S*>(L.buf[parity]),
                              static_cast<S*>(L.buf[parity ^ 1]), tl.y, tl.z, lane, seed,
                              stochastic);
  }
}

// Boundary nodes of every active lattice of a batch: entries {lattice, node}.
template <typename S>
__global__ void __launch_bounds__(kRedThreads)
    batch_boundary_kernel(const BatchLat* __restrict__ lats, const int2* __restrict__ entries,
                          int n, const int* __restrict__ active, int parity,
                          const long long* __restrict__ tptr, int tstep, int stochastic) {
  using R = typename Traits<S>::R;
  uint32_t seed = 0;
  if (stochastic) {
    const long long t = *tptr + tstep;
    seed = (uint32_t)(t * 0x9E3779B1ull) ^ (uint32_t)(t >> 32);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 e = entries[k];
    if (!active[e.x]) continue;
    const BatchLat* L = lats + e.x;
    const Co<R> c = make_co<R>(L->c);
    const S* src = static_cast<const S*>(L->buf[parity]);
    S* dst = static_cast<S*>(L->buf[parity ^ 1]);
    if (L->g.flags)
      step_node<S, true>(L->g, c, src, dst, e.y, seed, stochastic);
    else
      step_node<S, false>(L->g, c, src, dst, e.y, seed, stochastic);
  }
}

// Convergence measure of every active lattice in FP64: max over (T, ux, uy) of
// ||phi(t) - phi(t - K)||_2 / (K ||phi(t)||_2), against the snapshot taken at
// the previous check, which is then replaced.  Comparing states K (even) steps
// apart is blind to the period-2 oscillation a closed cavity can keep at a
// small amplitude, which would otherwise hold a one-step residual above the
// tolerance.  Two deterministic stages: block (i, ch) sums chunk ch
// (kResChunk nodes) of lattice i into part[i][ch][0..7]; one thread per
// lattice then adds its chunks in order.
constexpr int kResChunk = 8192;

template <typename S>
__global__ void __launch_bounds__(kRedThreads)
    batch_residual_partial_kernel(const BatchLat* __restrict__ lats, const int* __restrict__ active,
                                  double* __restrict__ part, int maxchunks) {
  const int i = blockIdx.x, ch = blockIdx.y;
  if (!active[i]) return;
  const BatchLat* L = lats + i;
  const DevGeom& g = L->g;
  const long long n = (long long)g.ny * g.nx;
  const long long k0 = (long long)ch * kResChunk;
  if (k0 >= n) return;
  const long long k1 = k0 + kResChunk < n ? k0 + kResChunk : n;
  const S* cur = static_cast<const S*>(L->buf[0]);
  double* snap = L->snap;
  // per-node values and per-thread sums (at most kResChunk / blockDim nodes)
  // in the collision's arithmetic (FP32 below FP64 storage, where FP64 is
  // slow); block sums in FP64
  using R = typename Traits<S>::R;
  const Co<R> co = make_co<R>(L->c);
  const bool vh = L->c.vh != 0;
  R a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int y = (int)(k / g.nx), x = (int)(k - (long long)y * g.nx);
    const long long idx = (long long)y * g.pitch + x;
    if (g.flags && (g.flags[idx] & kFlagSolid)) continue;
    R r1, u1, v1, t1;
    node_macros_r(co, vh, cur, g.plane, idx, r1, u1, v1, t1);
    const R t0 = (R)snap[k], u0 = (R)snap[n + k], v0 = (R)snap[2 * n + k];
    a[0] += (t1 - t0) * (t1 - t0);
    a[1] += t1 * t1;
    a[2] += (u1 - u0) * (u1 - u0);
    a[3] += u1 * u1;
    a[4] += (v1 - v0) * (v1 - v0);
    a[5] += v1 * v1;
    if (!isfinite(r1) || !isfinite(u1) || !isfinite(v1) || !isfinite(t1)) a[6] += R(1);
    snap[k] = t1;
    snap[n + k] = u1;
    snap[2 * n + k] = v1;
  }
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = (double)a[q];
  __shared__ double tot[8];
  block_sum_store<8>(acc, tot);
  __syncthreads();
  if (threadIdx.x < 8) part[((long long)i * maxchunks + ch) * 8 + threadIdx.x] = tot[threadIdx.x];
}

template <typename S>
__global__ void batch_residual_final_kernel(const BatchLat* __restrict__ lats, const int* __restrict__ active,
                                            int* __restrict__ snap_valid, const double* __restrict__ part,
                                            int maxchunks, double* __restrict__ res, int n, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !active[i]) return;
  const DevGeom& g = lats[i].g;
  const long long nodes = (long long)g.ny * g.nx;
  const int nch = (int)((nodes + kResChunk - 1) / kResChunk);
  double tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int ch = 0; ch < nch; ++ch)
    for (int q = 0; q < 8; ++q) tot[q] += part[((long long)i * maxchunks + ch) * 8 + q];
  double best = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double den = sqrt(tot[2 * q + 1]) > 1e-30 ? sqrt(tot[2 * q + 1]) : 1e-30;
    const double v = sqrt(tot[2 * q]) / den;
    best = v > best ? v : best;
  }
  best /= (double)K;
  if (!snap_valid[i]) best = 1e300;
  if (tot[6] != 0.0 || !isfinite(best)) best = INFINITY;
  res[i] = best;
  snap_valid[i] = 1;
}

// a <- (a + b) / 2 over every stored value (both post-collision states of a
// lattice, one step apart): cancels any component that flips sign each step.
template <typename S>
__global__ void average_state_kernel(S* __restrict__ a, const S* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    using R = typename Traits<S>::R;
    const R v = R(0.5) * (to_r(a[i]) + to_r(b[i]));
    a[i] = from_r<S, R>(v);
  }
}

// ---------------------------------------------------------------------------
// Launchers for one storage type
// ---------------------------------------------------------------------------
template <typename S>
struct LaunchImpl {
  static constexpr int V = Traits<S>::V;

  static cudaError_t step(const StepArgs& a, cudaStream_t s) {
    const int nodes_per_block = kStepThreads * V;
    const int xblocks = (a.g.nx + nodes_per_block - 1) / nodes_per_block;
    // one fused launch: boundary nodes in the first blocks, interior tiles in the
    // rest (box lattices; masked ones with their tile classes, whose interior
    // tiles leave the listed nodes out)
    if (!a.g.flags || a.g.tile_fluid) {
      // interior tiles: the own rows that are not next to a box wall (those are
      // boundary rows, in the node list)
      const int y0 = a.g.ylo + a.g.ywlo;
      const int rows = std::max(0, a.g.yhi - a.g.ywhi - y0);
      const int nbb = (a.nb + kStepThreads - 1) / kStepThreads;
      const long long blocks = (long long)nbb + (long long)xblocks * rows;
      if (blocks > 0 && blocks < (1LL << 31)) {
        const unsigned nblk = (unsigned)blocks;
        if (a.g.flags) {
          if (a.c.vh)
            step_fused_kernel<S, true, true><<<nblk, kStepThreads, 0, s>>>(a, nbb, xblocks, y0, rows);
          else
            step_fused_kernel<S, false, true><<<nblk, kStepThreads, 0, s>>>(a, nbb, xblocks, y0, rows);
        } else {
          if (a.c.vh)
            step_fused_kernel<S, true><<<nblk, kStepThreads, 0, s>>>(a, nbb, xblocks, y0, rows);
          else
            step_fused_kernel<S, false><<<nblk, kStepThreads, 0, s>>>(a, nbb, xblocks, y0, rows);
        }
        return cudaGetLastError();
      }
    }
    dim3 grid(xblocks, a.g.yhi - a.g.ylo);
    if (a.c.vh)
      step_kernel<S, true><<<grid, kStepThreads, 0, s>>>(a);
    else
      step_kernel<S, false><<<grid, kStepThreads, 0, s>>>(a);
    if (a.nb > 0) {
      const int blocks = (a.nb + kRedThreads - 1) / kRedThreads;
      if (a.g.flags)
        boundary_kernel<S, true><<<blocks, kRedThreads, 0, s>>>(a);
      else
        boundary_kernel<S, false><<<blocks, kRedThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
  }

  static int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
  }

  static cudaError_t init(const DevGeom& g, const DevCoef& c, void* dst, const double* rho,
                          const double* ux, const double* uy, const double* T, cudaStream_t s) {
    if (g.ny <= 0 || g.pitch <= 0) return cudaSuccess;
    const dim3 grid((g.pitch + 255) / 256, g.ny < 65535 ? g.ny : 65535);
    init_kernel<S><<<grid, 256, 0, s>>>(g, c, static_cast<S*>(dst), rho, ux, uy, T);
    return cudaGetLastError();
  }

  static cudaError_t moments(const DevGeom& g, const DevCoef& c, const void* buf, double* rho,
                             double* ux, double* uy, double* T, cudaStream_t s) {
    const int rows = g.yhi - g.ylo;
    if (rows <= 0 || g.nx <= 0) return cudaSuccess;
    const int threads = g.nx >= 256 ? 256 : (g.nx + 31) / 32 * 32;
    const dim3 grid((g.nx + threads - 1) / threads, rows < 65535 ? rows : 65535);
    moments_kernel<S><<<grid, threads, 0, s>>>(g, c, static_cast<const S*>(buf), rho, ux, uy, T);
    return cudaGetLastError();
  }

  static cudaError_t residual(const DevGeom& g, const DevCoef& c, const void* cur,
                              const void* prev, double* partials, int nblocks, cudaStream_t s) {
    residual_kernel<S><<<nblocks, kRedThreads, 0, s>>>(g, c, static_cast<const S*>(cur),
                                                        static_cast<const S*>(prev), partials);
    return cudaGetLastError();
  }

  static cudaError_t totals(const DevGeom& g, const void* buf, double* partials, int nblocks,
                            cudaStream_t s) {
    totals_kernel<S><<<nblocks, kRedThreads, 0, s>>>(g, static_cast<const S*>(buf), partials);
    return cudaGetLastError();
  }

  static cudaError_t nusselt(const DevGeom& g, const DevCoef& c, const void* buf,
                             const NuLink* links, int nlinks, double* partials, int nblocks,
                             cudaStream_t s) {
    nusselt_kernel<S><<<nblocks, kRedThreads, 0, s>>>(g, c, static_cast<const S*>(buf), links,
                                                       nlinks, partials);
    return cudaGetLastError();
  }

  template <int VV>
  static cudaError_t batch_launch(const BatchLat* lats, const int4* tiles, const int* count,
                                  int parity, const long long* t, int tstep, int stochastic, int grid,
                                  cudaStream_t s) {
    // batches run without the viscous source (clbm_batch_create rejects it)
    batch_step_kernel<S, VV, false><<<grid, kStepThreads, 0, s>>>(lats, tiles, count, parity, t,
                                                                   tstep, stochastic);
    return cudaGetLastError();
  }

  static cudaError_t batch_step(int v, const BatchLat* lats, const int4* tiles, const int* count,
                                int parity, const long long* t, int tstep, int stochastic, int grid,
                                cudaStream_t s) {
    if (v == 1) return batch_launch<1>(lats, tiles, count, parity, t, tstep, stochastic, grid, s);
    if (v == 2) return batch_launch<2>(lats, tiles, count, parity, t, tstep, stochastic, grid, s);
    if constexpr (V >= 4) {
      if (v == 4) return batch_launch<4>(lats, tiles, count, parity, t, tstep, stochastic, grid, s);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t batch_boundary(const BatchLat* lats, const int2* entries, int n,
                                    const int* active, int parity, const long long* t, int tstep,
                                    int stochastic, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + kRedThreads - 1) / kRedThreads;
    if (blocks > 4096) blocks = 4096;
    batch_boundary_kernel<S><<<blocks, kRedThreads, 0, s>>>(lats, entries, n, active, parity, t,
                                                             tstep, stochastic);
    return cudaGetLastError();
  }

  template <int VV>
  static int grid_of() {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel<S, VV, false>,
                                                      kStepThreads, 0) != cudaSuccess)
      return 0;
    return sms * (per_sm > 0 ? per_sm : 1);
  }

  static int batch_grid(int v) {
    if (v == 1) return grid_of<1>();
    if (v == 2) return grid_of<2>();
    if constexpr (V >= 4) {
      if (v == 4) return grid_of<4>();
    }
    return 0;
  }

  static cudaError_t batch_residual(const BatchLat* lats, const int* active, int* snap_valid,
                                    double* res, int n, int K, double* part, int maxchunks,
                                    cudaStream_t s) {
    batch_residual_partial_kernel<S><<<dim3(n, maxchunks), kRedThreads, 0, s>>>(lats, active, part,
                                                                                maxchunks);
    batch_residual_final_kernel<S><<<(n + 255) / 256, 256, 0, s>>>(lats, active, snap_valid, part,
                                                                 maxchunks, res, n, K);
    return cudaGetLastError();
  }

  static cudaError_t average(void* a, const void* b, long long n, cudaStream_t s) {
    average_state_kernel<S><<<blocks_for(n, 256), 256, 0, s>>>(static_cast<S*>(a),
                                                                 static_cast<const S*>(b), n);
    return cudaGetLastError();
  }

  static Launchers table() {
    Launchers L;
    L.average = &average;
    L.batch_step = &batch_step;
    L.batch_boundary = &batch_boundary;
    L.batch_grid = &batch_grid;
    L.batch_residual = &batch_residual;
    L.residual_chunk = kResChunk;
    L.vec = V;
    L.step = &step;
    L.init = &init;
    L.moments = &moments;
    L.residual = &residual;
    L.nusselt = &nusselt;
    L.totals = &totals;
    L.elem_bytes = sizeof(S);
    return L;
  }
};

}  // namespace clbm
