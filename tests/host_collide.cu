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
