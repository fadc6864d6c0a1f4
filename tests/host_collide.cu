// Test harness: the library's single-node collision (clbm::collide, the code
// every step kernel inlines) and its equilibrium (clbm::equilibrium, the
// initialisation) compiled for the host, so that CPU tests can set them
// against the FP64 oracle node by node.  Not part of the library; built by
// tests/test_collide_host.py.
#include "../paper_1801_04577_gb300/csrc/clbm_kernels.cuh"

namespace {

// rates: s_nu, s_b, s3, s4, l1, l2, rho0, T0, gbeta, Fvx, Fvy, Q, cT2 (s3 and
// l2 already resolved)
clbm::DevCoef coef_of(const double* r, int vh) {
  clbm::DevCoef k{};
  k.s_nu = r[0];
  k.s_b = r[1];
  k.s3 = r[2];
  k.s4 = r[3];
  k.l0 = 1.0;
  k.l1 = r[4];
  k.l2 = r[5];
  k.rho0 = r[6];
  k.T0 = r[7];
  k.gbeta = r[8];
  k.Fvx = r[9];
  k.Fvy = r[10];
  k.Q = r[11];
  k.cT2 = r[12];
  k.vh = vh;
  clbm::fill_f32(k);
  return k;
}

template <typename R, bool HK>
void run(const clbm::DevCoef& k, int vh, double* d, double* h, double* qv) {
  const clbm::Co<R> c = clbm::make_co<R>(k);
  R dd[9], hh[5], q = R(0);
  for (int i = 0; i < 9; ++i) dd[i] = (R)d[i];
  for (int i = 0; i < 5; ++i) hh[i] = (R)h[i];
  clbm::collide_any<R, HK>(c, vh != 0, dd, hh, q);
  for (int i = 0; i < 9; ++i) d[i] = (double)dd[i];
  for (int i = 0; i < 5; ++i) h[i] = (double)hh[i];
  *qv = (double)q;
}

}  // namespace

// d[9], h[5]: pre-collision deviations from the rest state in, post-collision
// deviations out.  form: 0 FP64 (host constants, the FP64 kernels), 1 FP32 with
// host constants (16-bit storage kernels), 2 FP32 with the constants formed in
// the collision (FP32-storage kernels).
extern "C" int host_collide(const double* rates, int vh, int form, double* d, double* h, double* qv) {
  const clbm::DevCoef k = coef_of(rates, vh);
  if (form == 0)
    run<double, true>(k, vh, d, h, qv);
  else if (form == 1)
    run<float, true>(k, vh, d, h, qv);
  else if (form == 2)
    run<float, false>(k, vh, d, h, qv);
  else
    return 1;
  return 0;
}

// d[9], h[5] out: equilibrium deviations from the rest state at (rho, ux, uy,
// T), in FP64.
extern "C" int host_equilibrium(const double* rates, double rho, double ux, double uy, double T, double* d,
                                double* h) {
  const clbm::DevCoef k = coef_of(rates, 0);
  const clbm::Co<double> c = clbm::make_co<double>(k);
  double dd[9], hh[5];
  clbm::equilibrium(c, rho, ux, uy, T, dd, hh);
  for (int i = 0; i < 9; ++i) d[i] = dd[i];
  for (int i = 0; i < 5; ++i) h[i] = hh[i];
  return 0;
}

// The wall rules of the fix-up (Eq. 28 and its off-midpoint form): which = 0
// wall_temperature, 1 wall_temperature_q, 2 midpoint_temperature_q; a[] holds
// the arguments in the functions' order; f32 != 0 evaluates in FP32.
extern "C" double host_wall(int which, int f32, const double* a) {
  if (f32) {
    float v[9];
    for (int i = 0; i < 9; ++i) v[i] = (float)a[i];
    if (which == 0) return clbm::wall_temperature(v[0], v[1], v[2], v[3], v[4], v[5], a[6] != 0);
    if (which == 1) return clbm::wall_temperature_q(v[0], v[1], v[2], v[3], v[4], v[5], v[6], a[7] != 0);
    return clbm::midpoint_temperature_q(v[0], v[1], v[2], v[3], a[4] != 0, v[5], a[6] != 0, a[7] != 0);
  }
  if (which == 0) return clbm::wall_temperature(a[0], a[1], a[2], a[3], a[4], a[5], a[6] != 0);
  if (which == 1) return clbm::wall_temperature_q(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7] != 0);
  return clbm::midpoint_temperature_q(a[0], a[1], a[2], a[3], a[4] != 0, a[5], a[6] != 0, a[7] != 0);
}
