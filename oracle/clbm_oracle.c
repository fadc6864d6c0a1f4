/*
 * FP64 CPU oracle for the cascaded (central-moment) double-distribution
 * lattice Boltzmann method for incompressible thermal flows
 * (Fei & Luo, "Cascaded lattice Boltzmann method for incompressible thermal
 * flows with heat sources and general thermal boundary conditions").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal statement of the
 * scheme that the CUDA library is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * path never does.  It shares no code, header or table with the CUDA library.
 *
 * How it follows the paper:
 *   - every transform is an explicit matrix product: M (Eq. 6a), N(u) (Eq. 6b),
 *     S (Eq. 8), M_T (Eq. 16), N_T(u) (Eq. 17), S_T (Sec. 2.2);
 *   - M^-1 and M_T^-1 are obtained numerically (Gauss-Jordan) at start-up;
 *   - N^-1 and N_T^-1 are applied by forward substitution, since N(u) and
 *     N_T(u) as printed are unit lower-triangular;
 *   - one time step is: macroscopic fields (Eq. 25, Eq. 2, Eq. 12), collision
 *     in central-moment space (Eq. 7 with Eq. 9-10; Eq. 23 with Eq. 19, 24),
 *     back-transformation (Eq. 11 text, Eq. 20), push streaming (Eq. 11, 21),
 *     then the wall rules: half-way bounce-back for f (Sec. 3) and the general
 *     bounce-back of Eq. 26 with T_w from Eq. 28 for g.
 *
 * Walls off the link midpoint (beyond the paper, which places every wall
 * half-way along its links): a listed link may carry the fraction q of the
 * link from the fluid node to the wall.  Then f follows the linear
 * interpolated bounce-back of Bouzidi, Firdaouss and Lallemand (Phys. Fluids
 * 13, 2001), and g keeps Eq. 26 at the link midpoint with the temperature
 * that the wall condition implies there: T_w at the wall from the condition
 * with the gradient of the quadratic through the wall point and the fluid
 * nodes at distances q and 1 + q (Eq. 27-28 when q = 1/2), and that
 * quadratic evaluated at the midpoint.  With q = 1/2 every rule is the
 * paper's.
 *
 * The state held between steps is the pre-collision pair (f, g) at time t.
 * All arithmetic is double precision; the file is compiled with
 * -ffp-contract=off so that no fused multiply-add changes the rounding.
 *
 * Readings of points the paper leaves open (each is a choice of this oracle):
 *   - u = (sum_i f_i e_i + F/2)/rho with rho = sum_i f_i (Eq. 12 as printed).
 *   - The Boussinesq force enters as a force density rho0 g beta (T - T0)
 *     along +y plus the external force F_v (Eq. 2, gravity along -y).
 *   - T at time t feeds both the force and the wall temperature; T_1 = T(x_f),
 *     T_2 = T(x_f - e_i) with e_i pointing from the fluid node to the wall.
 *   - When x_f - e_i is not a fluid node, dT/dn is taken one-sided,
 *     (T_w - T_1)/(n.e_i/2), instead of Eq. 27 (thin fluid layers only).
 *   - Equilibrium initialisation: f, g are the distributions whose central
 *     moments are Eq. 9 and Eq. 19 at the given rho, u, T.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------- lattice (Eq. 3) ---------------- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* D2Q9 rest weights (the Eq. 9 equilibrium at rho = 1, u = 0); used only by
 * the moving-wall bounce-back, which is not part of the paper */
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static int opposite(int i) {
  for (int j = 0; j < 9; ++j)
    if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
  return -1;
}

/* ---------------- parameters ---------------- */
typedef struct {
  int32_t nx, ny, periodic_x, periodic_y;
  double s_nu, s_b, s_3, s_4, lambda0, lambda1, lambda2;
  double rho0, T0, gbeta, Fvx, Fvy, Q, cT2;
  int32_t viscous_heating, reserved1; /* 1: add the viscous dissipation source (Sec. 3.2) */
} oref_params;

/* ---------------- small dense linear algebra ---------------- */
static void matvec(int n, const double* A, const double* x, double* y) {
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
    y[r] = s;
  }
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(int n, const double* A, double* Ainv) {
  double a[81 * 2];
  const int w = 2 * n;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < w; ++c)
      a[r * w + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r * w + col]) > fabs(a[piv * w + col])) piv = r;
    if (fabs(a[piv * w + col]) < 1e-300) return -1;
    if (piv != col)
      for (int c = 0; c < w; ++c) {
        double t = a[col * w + c];
        a[col * w + c] = a[piv * w + c];
        a[piv * w + c] = t;
      }
    double d = a[col * w + col];
    for (int c = 0; c < w; ++c) a[col * w + c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double m = a[r * w + col];
      if (m == 0.0) continue;
      for (int c = 0; c < w; ++c) a[r * w + c] -= m * a[col * w + c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * w + n + c];
  return 0;
}

/* Solve L y = b for unit lower-triangular L (this is how N^-1 is applied). */
static void forward_subst(int n, const double* L, const double* b, double* y) {
  for (int r = 0; r < n; ++r) {
    double s = b[r];
    for (int c = 0; c < r; ++c) s -= L[r * n + c] * y[c];
    y[r] = s;
  }
}

/* ---------------- flow transforms (Sec. 2.1) ---------------- */
/* Eq. 6a, rows ordered as Eq. 5: k00,k10,k01,k20,k02,k11,k21,k12,k22. */
static const double M9[81] = {
    1, 1, 1, 1, 1, 1, 1, 1, 1,
    0, 1, 0, -1, 0, 1, -1, -1, 1,
    0, 0, 1, 0, -1, 1, 1, -1, -1,
    0, 1, 0, 1, 0, 1, 1, 1, 1,
    0, 0, 1, 0, 1, 1, 1, 1, 1,
    0, 0, 0, 0, 0, 1, -1, 1, -1,
    0, 0, 0, 0, 0, 1, 1, -1, -1,
    0, 0, 0, 0, 0, 1, -1, -1, 1,
    0, 0, 0, 0, 0, 1, 1, 1, 1};

/* Eq. 6b, the shift matrix N(u). */
static void shift9(double ux, double uy, double* N) {
  const double ux2 = ux * ux, uy2 = uy * uy;
  const double rows[81] = {
      1, 0, 0, 0, 0, 0, 0, 0, 0,
      -ux, 1, 0, 0, 0, 0, 0, 0, 0,
      -uy, 0, 1, 0, 0, 0, 0, 0, 0,
      ux2, -2 * ux, 0, 1, 0, 0, 0, 0, 0,
      uy2, 0, -2 * uy, 0, 1, 0, 0, 0, 0,
      ux * uy, -uy, -ux, 0, 0, 1, 0, 0, 0,
      -ux2 * uy, 2 * ux * uy, ux2, -uy, 0, -2 * ux, 1, 0, 0,
      -uy2 * ux, uy2, 2 * ux * uy, 0, -ux, -2 * uy, 0, 1, 0,
      ux2 * uy2, -2 * ux * uy2, -2 * uy * ux2, uy2, ux2, 4 * ux * uy, -2 * uy, -2 * ux, 1};
  memcpy(N, rows, sizeof(rows));
}

/* ---------------- thermal transforms (Sec. 2.2) ---------------- */
/* Eq. 16 */
static const double M5[25] = {
    1, 1, 1, 1, 1,
    0, 1, 0, -1, 0,
    0, 0, 1, 0, -1,
    0, 1, 0, 1, 0,
    0, 0, 1, 0, 1};

/* Eq. 17 */
static void shift5(double ux, double uy, double* N) {
  const double rows[25] = {
      1, 0, 0, 0, 0,
      -ux, 1, 0, 0, 0,
      -uy, 0, 1, 0, 0,
      ux * ux, -2 * ux, 0, 1, 0,
      uy * uy, 0, -2 * uy, 0, 1};
  memcpy(N, rows, sizeof(rows));
}

/* ---------------- solver state ---------------- */
typedef struct {
  oref_params p;
  double s3, lambda2;          /* resolved rates (Sec. 3 rules when <= 0)   */
  double Minv[81], MTinv[25];  /* numerical inverses of Eq. 6a and Eq. 16   */
  double S[81], ST[25];        /* Eq. 8 and diag(l0,l1,l1,l2,l2)            */
  int64_t n;                   /* nx*ny                                     */
  uint8_t* solid;              /* 1 = solid node                            */
  /* thermal wall data per (node, D2Q5 dir 1..4): tbc index or -1, and n.e  */
  int32_t* wtbc;
  double* wne;
  double* wq;                  /* per (node, dir 1..8): wall fraction q, 0.5 default */
  double *fs, *gs;             /* post-collision DFs of every node (one step)  */
  double* tbc;                 /* ntbc x (b1,b2,b3)                         */
  int32_t ntbc;
  double *f, *g, *fn, *gn;     /* pre-collision DFs at t, and at t+1        */
  double *T, *rho, *ux, *uy;   /* macroscopic fields at time t (of the last step) */
  double* Qn;                  /* total heat source per node at time t          */
  double uw[4][2];             /* velocity of each box side (x0, x1, y0, y1); 0 = at rest */
  int have_prev;
  int64_t steps;
} oref_ctx;

static int64_t idx(const oref_ctx* c, int x, int y) { return (int64_t)y * c->p.nx + x; }

/* Neighbour (x+dx, y+dy) after periodic wrapping; returns 0 if it is outside
 * the box (a box wall), 1 otherwise. */
static int neighbour(const oref_ctx* c, int x, int y, int dx, int dy, int* xo, int* yo, int* side) {
  int xn = x + dx, yn = y + dy;
  *side = -1;
  if (xn < 0 || xn >= c->p.nx) {
    if (c->p.periodic_x)
      xn = (xn + c->p.nx) % c->p.nx;
    else {
      *side = xn < 0 ? 0 : 1;
      return 0;
    }
  }
  if (yn < 0 || yn >= c->p.ny) {
    if (c->p.periodic_y)
      yn = (yn + c->p.ny) % c->p.ny;
    else {
      *side = yn < 0 ? 2 : 3;
      return 0;
    }
  }
  *xo = xn;
  *yo = yn;
  return 1;
}

static int is_fluid(const oref_ctx* c, int x, int y) {
  return c->solid == NULL || c->solid[idx(c, x, y)] == 0;
}

/* ---------------- node-level building blocks ---------------- */

/* Viscous dissipation source of Sec. 3.2, Q_v = nu (du/dy)^2 for the channel;
 * in general nu (D^2 + G^2) with D = dux/dx - duy/dy, G = duy/dx + dux/dy (the
 * dissipation 2 nu S:S of a divergence-free flow).  The strain rate is read
 * from the pre-collision non-equilibrium central moments: the stress
 * (1 - s/2) k~^neq equals rho nu times the strain with nu = (1/s_nu - 1/2)/3,
 * so G = -3 s_nu k~11 / rho and D = -3 s_nu (k~20 - k~02) / (2 rho). */
static double viscous_source(const oref_ctx* c, const double* f, double rho, double ux, double uy) {
  double N[81], k[9], kt[9];
  matvec(9, M9, f, k);
  shift9(ux, uy, N);
  matvec(9, N, k, kt); /* order of Eq. 5: kt[3] = k~20, kt[4] = k~02, kt[5] = k~11 */
  const double nu = (1.0 / c->p.s_nu - 0.5) / 3.0;
  const double G = -3.0 * c->p.s_nu * kt[5] / rho;
  const double D = -1.5 * c->p.s_nu * (kt[3] - kt[4]) / rho;
  return nu * (D * D + G * G);
}

/* Macroscopic fields of one node from its pre-collision DFs (Eq. 25, 2, 12);
 * *Q receives the total heat source at the node.  With viscous heating the
 * Boussinesq force uses T without the viscous source's half (the source needs
 * u, which needs the force). */
static void macros(const oref_ctx* c, const double* f, const double* g, double* rho, double* ux,
                   double* uy, double* T, double* Fx, double* Fy, double* Q) {
  double t = 0.0;
  for (int i = 0; i < 5; ++i) t += g[i];
  t += 0.5 * c->p.Q; /* Eq. 25 */
  double fx = c->p.Fvx;
  double fy = c->p.Fvy + c->p.rho0 * c->p.gbeta * (t - c->p.T0); /* Eq. 2 */
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    r += f[i];
    jx += f[i] * EX[i];
    jy += f[i] * EY[i];
  }
  *rho = r;
  *ux = (jx + 0.5 * fx) / r; /* Eq. 12 */
  *uy = (jy + 0.5 * fy) / r;
  double q = c->p.Q;
  if (c->p.viscous_heating) {
    const double qv = viscous_source(c, f, r, *ux, *uy);
    q += qv;
    t += 0.5 * qv; /* Eq. 25 with the total source */
  }
  *T = t;
  *Fx = fx;
  *Fy = fy;
  if (Q) *Q = q;
}

/* Flow collision (Eq. 6-10) and back-transformation (text after Eq. 11). */
static void collide_flow(const oref_ctx* c, const double* f, double rho, double ux, double uy,
                         double Fx, double Fy, double* fs) {
  double N[81], k[9], kt[9], keq[9], C[9], ks[9], a[9], b[9], raw[9];
  const double cs2 = 1.0 / 3.0;
  matvec(9, M9, f, k);    /* Gamma = M f          */
  shift9(ux, uy, N);
  matvec(9, N, k, kt);    /* Gamma~ = N Gamma     */
  /* Eq. 9 */
  const double eq[9] = {rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2};
  /* Eq. 10 */
  const double cf[9] = {0, Fx, Fy, 0, 0, 0, cs2 * Fy, cs2 * Fx, 0};
  memcpy(keq, eq, sizeof(eq));
  memcpy(C, cf, sizeof(cf));
  /* Eq. 7: (I - S) kt + S keq + (I - S/2) C */
  double ImS[81], ImS2[81];
  for (int r = 0; r < 9; ++r)
    for (int q = 0; q < 9; ++q) {
      double id = r == q ? 1.0 : 0.0;
      ImS[r * 9 + q] = id - c->S[r * 9 + q];
      ImS2[r * 9 + q] = id - 0.5 * c->S[r * 9 + q];
    }
  matvec(9, ImS, kt, a);
  matvec(9, c->S, keq, b);
  double cc[9];
  matvec(9, ImS2, C, cc);
  for (int r = 0; r < 9; ++r) ks[r] = a[r] + b[r] + cc[r];
  /* f* = M^-1 N^-1 Gamma~* */
  forward_subst(9, N, ks, raw);
  matvec(9, c->Minv, raw, fs);
}

/* Thermal collision with source Q (Eq. 15, 19, 23, 24) and Eq. 20. */
static void collide_thermal(const oref_ctx* c, const double* g, double ux, double uy, double T,
                            double Q, double* gs) {
  double N[25], k[5], kt[5], a[5], b[5], r5[5], ks[5], raw[5];
  const double cT2 = c->p.cT2;
  matvec(5, M5, g, k);
  shift5(ux, uy, N);
  matvec(5, N, k, kt);
  const double eq[5] = {T, 0, 0, T * cT2, T * cT2};  /* Eq. 19 */
  const double R[5] = {Q, 0, 0, Q * cT2, Q * cT2};   /* Eq. 24 */
  double ImS[25], ImS2[25];
  for (int r = 0; r < 5; ++r)
    for (int q = 0; q < 5; ++q) {
      double id = r == q ? 1.0 : 0.0;
      ImS[r * 5 + q] = id - c->ST[r * 5 + q];
      ImS2[r * 5 + q] = id - 0.5 * c->ST[r * 5 + q];
    }
  matvec(5, ImS, kt, a);
  matvec(5, c->ST, eq, b);
  matvec(5, ImS2, R, r5);
  for (int r = 0; r < 5; ++r) ks[r] = a[r] + b[r] + r5[r];
  forward_subst(5, N, ks, raw);
  matvec(5, c->MTinv, raw, gs);
}

/* Eq. 28: wall temperature of b1 dT/dn + b2 T = b3 with the second-order
 * gradient of Eq. 27; falls back to a one-sided gradient when T_2 is absent. */
double oref_wall_temperature(double b1, double b2, double b3, double ne, double T1, double T2,
                             int have_T2) {
  if (have_T2) return (9.0 * b1 * T1 - b1 * T2 + 3.0 * ne * b3) / (8.0 * b1 + 3.0 * ne * b2);
  /* b1 (Tw - T1)/(ne/2) + b2 Tw = b3 */
  return (2.0 * b1 * T1 + ne * b3) / (2.0 * b1 + ne * b2);
}

/* Walls at the fraction q of the link (beyond the paper).  With s the
 * distance from the wall along the link into the fluid, T(s) is the quadratic
 * through (0, T_w), (q, T_1), (1 + q, T_2), so
 *   dT/ds(0) = -(1+2q)/(q(1+q)) T_w + (1+q)/q T_1 - q/(1+q) T_2
 * and dT/dn = -dT/ds(0) / (n.e_i).  b1 dT/dn + b2 T_w = b3 is solved for T_w.
 * Without T_2 the profile is the line through (0, T_w), (q, T_1).  For q = 1/2
 * these are Eq. 27-28 and their one-sided fallback. */
double oref_wall_temperature_q(double b1, double b2, double b3, double ne, double q, double T1,
                               double T2, int have_T2) {
  if (have_T2) {
    const double a = (1.0 + 2.0 * q) / (q * (1.0 + q));
    const double c1 = (1.0 + q) / q, c2 = q / (1.0 + q);
    return (b3 * ne + b1 * (c1 * T1 - c2 * T2)) / (b1 * a + b2 * ne);
  }
  return (b3 * q * ne + b1 * T1) / (b1 + b2 * q * ne);
}

/* dT/dn at a wall at the fraction q of the link (same profile). */
static double wall_gradient_q(double ne, double q, double Tw, double T1, double T2, int have_T2) {
  if (have_T2)
    return ((1.0 + 2.0 * q) / (q * (1.0 + q)) * Tw - (1.0 + q) / q * T1 + q / (1.0 + q) * T2) / ne;
  return (Tw - T1) / (q * ne);
}

/* Value at s of the quadratic through (0, v0), (s1, v1), (s2, v2). */
static double quad_at(double s, double s1, double s2, double v0, double v1, double v2) {
  const double l0 = (s - s1) * (s - s2) / (s1 * s2);
  const double l1 = s * (s - s2) / (s1 * (s1 - s2));
  const double l2 = s * (s - s1) / (s2 * (s2 - s1));
  return l0 * v0 + l1 * v1 + l2 * v2;
}

/* The wall profile at the link midpoint s = q - 1/2, the temperature that
 * Eq. 26 imposes there.  q >= 1/2: the midpoint lies between the wall and
 * x_f, and the quadratic through (0, T_w), (q, T_1), (1 + q, T_2) is
 * interpolated.  q < 1/2: it lies beyond the wall; the quadratic through
 * (0, T_w), (1 + q, T_2), (2 + q, T_3) is extrapolated instead, which keeps
 * the weights bounded as q -> 0 and leaves out T_1 (a large weight on the
 * node's own temperature feeds back into the node and is unstable).  Both are
 * exact for quadratic profiles.  Fallbacks for thin fluid layers: lines
 * through the available points, else T_w. */
double oref_midpoint_temperature_q(double q, double Tw, double T1, double T2, int have_T2, double T3,
                                   int have_T3, int dirichlet) {
  const double s = q - 0.5;
  if (q >= 0.5 || !dirichlet) {
    if (have_T2) return quad_at(s, q, 1.0 + q, Tw, T1, T2);
    return Tw + (T1 - Tw) * s / q;
  }
  if (have_T2 && have_T3) return quad_at(s, 1.0 + q, 2.0 + q, Tw, T2, T3);
  if (have_T2) return Tw + (T2 - Tw) * s / (1.0 + q);
  return Tw;
}

/* Eq. 27 (or its one-sided fallback). */
static double wall_gradient(double ne, double Tw, double T1, double T2, int have_T2) {
  if (have_T2) return (8.0 * Tw - 9.0 * T1 + T2) / (3.0 * ne);
  return (Tw - T1) / (0.5 * ne);
}

/* ---------------- public API ---------------- */
enum { OREF_OK = 0, OREF_EINVAL = 1, OREF_ENOMEM = 2 };

static double resolved_s3(const oref_params* p) {
  if (p->s_3 > 0) return p->s_3;
  return (16.0 - 8.0 * p->s_nu) / (8.0 - p->s_nu); /* non-slip rule, Sec. 3 */
}

static double resolved_lambda2(const oref_params* p) {
  if (p->lambda2 > 0) return p->lambda2;
  return 12.0 * (p->lambda1 - 2.0) / (p->lambda1 - 12.0); /* Sec. 3.1 */
}

static void build_relaxation(oref_ctx* c) {
  const oref_params* p = &c->p;
  memset(c->S, 0, sizeof(c->S));
  const double sp = 0.5 * (p->s_b + p->s_nu), sm = 0.5 * (p->s_b - p->s_nu); /* Eq. 8 */
  c->S[3 * 9 + 3] = sp;
  c->S[3 * 9 + 4] = sm;
  c->S[4 * 9 + 3] = sm;
  c->S[4 * 9 + 4] = sp;
  c->S[5 * 9 + 5] = p->s_nu;
  c->S[6 * 9 + 6] = c->s3;
  c->S[7 * 9 + 7] = c->s3;
  c->S[8 * 9 + 8] = p->s_4;
  memset(c->ST, 0, sizeof(c->ST));
  c->ST[0] = p->lambda0;
  c->ST[1 * 5 + 1] = p->lambda1;
  c->ST[2 * 5 + 2] = p->lambda1;
  c->ST[3 * 5 + 3] = c->lambda2;
  c->ST[4 * 5 + 4] = c->lambda2;
}

void oref_destroy(void* h) {
  oref_ctx* c = (oref_ctx*)h;
  if (!c) return;
  free(c->solid);
  free(c->wtbc);
  free(c->wne);
  free(c->wq);
  free(c->fs);
  free(c->gs);
  free(c->tbc);
  free(c->f);
  free(c->g);
  free(c->fn);
  free(c->gn);
  free(c->T);
  free(c->rho);
  free(c->ux);
  free(c->uy);
  free(c->Qn);
  free(c);
}

/* Links: node, dir (1..8, from the fluid node towards the wall), n.e_i and
 * condition index (D2Q5 directions 1..4 only; ignored for 5..8), and the wall
 * fraction q in (0, 1] (lq NULL: 1/2 for every link). */
int oref_create(const oref_params* p, const uint8_t* solid, const double* tbc, int32_t ntbc,
                const int32_t* side_tbc, const int32_t* lnode, const int32_t* ldir,
                const double* lne, const int32_t* ltbc, const double* lq, int32_t nlinks,
                void** out) {
  *out = NULL;
  if (p->nx < 1 || p->ny < 1) return OREF_EINVAL;
  oref_ctx* c = (oref_ctx*)calloc(1, sizeof(oref_ctx));
  if (!c) return OREF_ENOMEM;
  c->p = *p;
  c->n = (int64_t)p->nx * p->ny;
  c->s3 = resolved_s3(p);
  c->lambda2 = resolved_lambda2(p);
  build_relaxation(c);
  if (invert(9, M9, c->Minv) || invert(5, M5, c->MTinv)) {
    oref_destroy(c);
    return OREF_EINVAL;
  }
  const int64_t n = c->n;
  c->f = (double*)calloc(9 * n, sizeof(double));
  c->g = (double*)calloc(5 * n, sizeof(double));
  c->fn = (double*)calloc(9 * n, sizeof(double));
  c->gn = (double*)calloc(5 * n, sizeof(double));
  c->T = (double*)calloc(n, sizeof(double));
  c->rho = (double*)calloc(n, sizeof(double));
  c->ux = (double*)calloc(n, sizeof(double));
  c->uy = (double*)calloc(n, sizeof(double));
  c->Qn = (double*)calloc(n, sizeof(double));
  c->solid = (uint8_t*)calloc(n, 1);
  c->wtbc = (int32_t*)malloc(5 * n * sizeof(int32_t));
  c->wne = (double*)calloc(5 * n, sizeof(double));
  c->wq = (double*)malloc(9 * n * sizeof(double));
  c->fs = (double*)calloc(9 * n, sizeof(double));
  c->gs = (double*)calloc(5 * n, sizeof(double));
  c->tbc = (double*)calloc(3 * (ntbc > 0 ? ntbc : 1), sizeof(double));
  if (!c->f || !c->g || !c->fn || !c->gn || !c->T || !c->rho || !c->ux || !c->uy || !c->Qn || !c->solid ||
      !c->wtbc || !c->wne || !c->wq || !c->fs || !c->gs || !c->tbc) {
    oref_destroy(c);
    return OREF_ENOMEM;
  }
  if (solid) memcpy(c->solid, solid, n);
  c->ntbc = ntbc;
  if (ntbc > 0) memcpy(c->tbc, tbc, 3 * ntbc * sizeof(double));
  for (int64_t k = 0; k < 5 * n; ++k) c->wtbc[k] = -1;
  for (int64_t k = 0; k < 9 * n; ++k) c->wq[k] = 0.5;
  /* Box sides: axis-aligned links, n.e_i = 1. */
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      if (!is_fluid(c, x, y)) continue;
      for (int i = 1; i < 5; ++i) {
        int xo, yo, side;
        if (!neighbour(c, x, y, EX[i], EY[i], &xo, &yo, &side)) {
          int t = side_tbc[side];
          if (t < 0 || t >= ntbc) {
            oref_destroy(c);
            return OREF_EINVAL;
          }
          c->wtbc[5 * idx(c, x, y) + i] = t;
          c->wne[5 * idx(c, x, y) + i] = 1.0;
        }
      }
    }
  /* Listed links into solid nodes. */
  for (int32_t l = 0; l < nlinks; ++l) {
    const double q = lq ? lq[l] : 0.5;
    const int axis = ldir[l] >= 1 && ldir[l] <= 4;
    if (lnode[l] < 0 || lnode[l] >= n || ldir[l] < 1 || ldir[l] > 8 || !(q > 0.0 && q <= 1.0) ||
        (axis && (ltbc[l] < 0 || ltbc[l] >= ntbc || !(lne[l] > 0)))) {
      oref_destroy(c);
      return OREF_EINVAL;
    }
    if (axis) {
      c->wtbc[5 * (int64_t)lnode[l] + ldir[l]] = ltbc[l];
      c->wne[5 * (int64_t)lnode[l] + ldir[l]] = lne[l];
    }
    c->wq[9 * (int64_t)lnode[l] + ldir[l]] = q;
  }
  /* Every D2Q5 link from a fluid node into a solid node needs a condition. */
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      if (!is_fluid(c, x, y)) continue;
      for (int i = 1; i < 5; ++i) {
        int xo, yo, side;
        if (neighbour(c, x, y, EX[i], EY[i], &xo, &yo, &side) && !is_fluid(c, xo, yo) &&
            c->wtbc[5 * idx(c, x, y) + i] < 0) {
          oref_destroy(c);
          return OREF_EINVAL;
        }
      }
    }
  *out = c;
  return OREF_OK;
}

/* Equilibrium DFs: central moments given by Eq. 9 and Eq. 19 at (rho, u, T). */
void oref_equilibrium(void* h, double rho, double ux, double uy, double T, double* f, double* g) {
  oref_ctx* c = (oref_ctx*)h;
  const double cs2 = 1.0 / 3.0, cT2 = c->p.cT2;
  double N[81], raw[9], N5[25], raw5[5];
  const double eq[9] = {rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2};
  shift9(ux, uy, N);
  forward_subst(9, N, eq, raw);
  matvec(9, c->Minv, raw, f);
  const double eq5[5] = {T, 0, 0, T * cT2, T * cT2};
  shift5(ux, uy, N5);
  forward_subst(5, N5, eq5, raw5);
  matvec(5, c->MTinv, raw5, g);
}

int oref_init(void* h, const double* rho, const double* ux, const double* uy, const double* T) {
  oref_ctx* c = (oref_ctx*)h;
  for (int64_t k = 0; k < c->n; ++k) {
    double r = rho ? rho[k] : c->p.rho0;
    double u = ux ? ux[k] : 0.0, v = uy ? uy[k] : 0.0;
    double t = T ? T[k] : c->p.T0;
    if (c->solid[k]) {
      r = c->p.rho0;
      u = v = 0.0;
      t = c->p.T0;
    }
    oref_equilibrium(c, r, u, v, t, c->f + 9 * k, c->g + 5 * k);
  }
  c->have_prev = 0;
  c->steps = 0;
  return OREF_OK;
}

/* One time step in the paper's order. */
static void step_once(oref_ctx* c) {
  const int nx = c->p.nx, ny = c->p.ny;
  const double cT2 = c->p.cT2;
  int opp[9];
  for (int i = 0; i < 9; ++i) opp[i] = opposite(i);
  /* macroscopic fields at time t (needed by Eq. 28 at every wall link) */
#pragma omp parallel for schedule(static) if (c->n >= 2048)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int64_t k = idx(c, x, y);
      double Fx, Fy;
      if (!is_fluid(c, x, y)) {
        c->rho[k] = c->ux[k] = c->uy[k] = c->T[k] = c->Qn[k] = 0.0;
        continue;
      }
      macros(c, c->f + 9 * k, c->g + 5 * k, &c->rho[k], &c->ux[k], &c->uy[k], &c->T[k], &Fx, &Fy,
             &c->Qn[k]);
    }
  /* collide every fluid node (Eq. 7-11, Eq. 18-23) */
#pragma omp parallel for schedule(static) if (c->n >= 2048)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int64_t k = idx(c, x, y);
      if (!is_fluid(c, x, y)) continue;
      const double Fx = c->p.Fvx;
      /* force temperature: T without the viscous source's half (see macros) */
      const double Tf = c->T[k] - 0.5 * (c->Qn[k] - c->p.Q);
      const double Fy = c->p.Fvy + c->p.rho0 * c->p.gbeta * (Tf - c->p.T0);
      collide_flow(c, c->f + 9 * k, c->rho[k], c->ux[k], c->uy[k], Fx, Fy, c->fs + 9 * k);
      collide_thermal(c, c->g + 5 * k, c->ux[k], c->uy[k], c->T[k], c->Qn[k], c->gs + 5 * k);
    }
  /* stream (Eq. 11, 21) and apply the wall rules */
#pragma omp parallel for schedule(static) if (c->n >= 2048)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int64_t k = idx(c, x, y);
      if (!is_fluid(c, x, y)) {
        for (int i = 0; i < 9; ++i) c->fn[9 * k + i] = 0.0;
        for (int i = 0; i < 5; ++i) c->gn[5 * k + i] = 0.0;
        continue;
      }
      const double* fs = c->fs + 9 * k;
      const double* gs = c->gs + 5 * k;
      for (int i = 0; i < 9; ++i) {
        int xo, yo, side;
        if (neighbour(c, x, y, EX[i], EY[i], &xo, &yo, &side) && is_fluid(c, xo, yo)) {
          c->fn[9 * idx(c, xo, yo) + i] = fs[i];
          continue;
        }
        const double q = c->wq[9 * k + i];
        int xb, yb, sb;
        const int have_b = neighbour(c, x, y, -EX[i], -EY[i], &xb, &yb, &sb) && is_fluid(c, xb, yb);
        if (q == 0.5 || (q < 0.5 && !have_b)) {
          /* half-way bounce-back: the DF returns to x_f reversed */
          c->fn[9 * k + opp[i]] = fs[i];
          if (side >= 0) {
            /* a moving box side (not in the paper; the bounce-back of Ladd,
             * J. Fluid Mech. 271, 1994): the reflected DF gains
             * -2 w_i rho0 (e_i . u_w) / cs^2 */
            const double eu = EX[i] * c->uw[side][0] + EY[i] * c->uw[side][1];
            c->fn[9 * k + opp[i]] -= 6.0 * W9[i] * c->p.rho0 * eu;
          }
        } else if (q < 0.5) {
          /* f_i* interpolated to the point 1 - 2q behind x_f, which reaches x_f reflected */
          c->fn[9 * k + opp[i]] = 2.0 * q * fs[i] + (1.0 - 2.0 * q) * c->fs[9 * idx(c, xb, yb) + i];
        } else {
          /* the reflected DF lands 2q - 1 beyond x_f: interpolate with f_ibar* at x_f */
          c->fn[9 * k + opp[i]] = fs[i] / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fs[opp[i]];
        }
      }
      for (int i = 0; i < 5; ++i) {
        int xo, yo, side;
        if (neighbour(c, x, y, EX[i], EY[i], &xo, &yo, &side) && is_fluid(c, xo, yo)) {
          c->gn[5 * idx(c, xo, yo) + i] = gs[i];
          continue;
        }
        /* Eq. 26-28 with e_i pointing into the wall */
        const int t = c->wtbc[5 * k + i];
        const double ne = c->wne[5 * k + i];
        const double* b = c->tbc + 3 * t;
        const double q = c->wq[9 * k + i];
        int x2, y2, s2;
        int have2 = neighbour(c, x, y, -EX[i], -EY[i], &x2, &y2, &s2) && is_fluid(c, x2, y2);
        const double T2 = have2 ? c->T[idx(c, x2, y2)] : 0.0;
        double Tm;
        if (q == 0.5) {
          Tm = oref_wall_temperature(b[0], b[1], b[2], ne, c->T[k], T2, have2);
        } else {
          int x3 = 0, y3 = 0, s3 = 0;
          const int have3 = have2 && neighbour(c, x2, y2, -EX[i], -EY[i], &x3, &y3, &s3) && is_fluid(c, x3, y3);
          const double T3 = have3 ? c->T[idx(c, x3, y3)] : 0.0;
          const double Tw = oref_wall_temperature_q(b[0], b[1], b[2], ne, q, c->T[k], T2, have2);
          Tm = oref_midpoint_temperature_q(q, Tw, c->T[k], T2, have2, T3, have3, b[0] == 0.0);
        }
        c->gn[5 * k + opp[i]] = -gs[i] + cT2 * Tm;
      }
    }
  double* t;
  t = c->f; c->f = c->fn; c->fn = t;
  t = c->g; c->g = c->gn; c->gn = t;
  c->have_prev = 1;
  c->steps += 1;
}

int oref_step(void* h, int64_t nsteps) {
  oref_ctx* c = (oref_ctx*)h;
  if (nsteps < 0) return OREF_EINVAL;
  for (int64_t s = 0; s < nsteps; ++s) step_once(c);
  return OREF_OK;
}

/* rho, u, T at the current time (solid nodes report 0). */
int oref_moments(void* h, double* rho, double* ux, double* uy, double* T) {
  oref_ctx* c = (oref_ctx*)h;
  for (int64_t k = 0; k < c->n; ++k) {
    double r = 0, u = 0, v = 0, t = 0, Fx, Fy;
    if (!c->solid[k]) macros(c, c->f + 9 * k, c->g + 5 * k, &r, &u, &v, &t, &Fx, &Fy, NULL);
    if (rho) rho[k] = r;
    if (ux) ux[k] = u;
    if (uy) uy[k] = v;
    if (T) T[k] = t;
  }
  return OREF_OK;
}

int oref_get_dfs(void* h, double* f, double* g) {
  oref_ctx* c = (oref_ctx*)h;
  if (f) memcpy(f, c->f, 9 * c->n * sizeof(double));
  if (g) memcpy(g, c->g, 5 * c->n * sizeof(double));
  return OREF_OK;
}

int oref_set_dfs(void* h, const double* f, const double* g) {
  oref_ctx* c = (oref_ctx*)h;
  if (f) memcpy(c->f, f, 9 * c->n * sizeof(double));
  if (g) memcpy(c->g, g, 5 * c->n * sizeof(double));
  c->have_prev = 0;
  return OREF_OK;
}

/* Nusselt number of a wall: (length/dT) * mean over its D2Q5 wall links of
 * dT/dn (Eq. 27, n out of the fluid), i.e. positive where heat enters the
 * fluid.  which = 0..3 selects a box side (x0, x1, y0, y1); which = 4 + k
 * selects the listed links with condition k. */
int oref_nusselt(void* h, int32_t which, double length, double dT, double* nu) {
  oref_ctx* c = (oref_ctx*)h;
  const int nx = c->p.nx, ny = c->p.ny;
  double* T = (double*)malloc(c->n * sizeof(double));
  if (!T) return OREF_ENOMEM;
  oref_moments(c, NULL, NULL, NULL, T);
  double sum = 0.0;
  int64_t cnt = 0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (!is_fluid(c, x, y)) continue;
      int64_t k = idx(c, x, y);
      for (int i = 1; i < 5; ++i) {
        int t = c->wtbc[5 * k + i];
        if (t < 0) continue;
        int xo, yo, side;
        int inbox = neighbour(c, x, y, EX[i], EY[i], &xo, &yo, &side);
        int match = which < 4 ? (!inbox && side == which) : (inbox && t == which - 4);
        if (!match) continue;
        const double ne = c->wne[5 * k + i];
        const double* b = c->tbc + 3 * t;
        int x2, y2, s2;
        int have2 = neighbour(c, x, y, -EX[i], -EY[i], &x2, &y2, &s2) && is_fluid(c, x2, y2);
        const double T2 = have2 ? T[idx(c, x2, y2)] : 0.0;
        const double q = c->wq[9 * k + i];
        if (q == 0.5) {
          const double Tw = oref_wall_temperature(b[0], b[1], b[2], ne, T[k], T2, have2);
          sum += wall_gradient(ne, Tw, T[k], T2, have2);
        } else {
          const double Tw = oref_wall_temperature_q(b[0], b[1], b[2], ne, q, T[k], T2, have2);
          sum += wall_gradient_q(ne, q, Tw, T[k], T2, have2);
        }
        cnt += 1;
      }
    }
  free(T);
  if (cnt == 0) return OREF_EINVAL;
  *nu = length / dT * (sum / (double)cnt);
  return OREF_OK;
}

/* Relative change of (T, ux, uy) over the last step: the largest of
 * ||phi(t) - phi(t-1)||_2 / max(||phi(t)||_2, 1e-30) over fluid nodes. */
int oref_residual(void* h, double* r) {
  oref_ctx* c = (oref_ctx*)h;
  if (!c->have_prev) return OREF_EINVAL;
  double d[3] = {0, 0, 0}, s[3] = {0, 0, 0};
  for (int64_t k = 0; k < c->n; ++k) {
    if (c->solid[k]) continue;
    double rr, u, v, t, Fx, Fy;
    macros(c, c->f + 9 * k, c->g + 5 * k, &rr, &u, &v, &t, &Fx, &Fy, NULL);
    const double now[3] = {t, u, v}, prev[3] = {c->T[k], c->ux[k], c->uy[k]};
    for (int q = 0; q < 3; ++q) {
      d[q] += (now[q] - prev[q]) * (now[q] - prev[q]);
      s[q] += now[q] * now[q];
    }
  }
  double best = 0.0;
  for (int q = 0; q < 3; ++q) {
    double v = sqrt(d[q]) / fmax(sqrt(s[q]), 1e-30);
    if (v > best) best = v;
  }
  *r = best;
  return OREF_OK;
}

/* ---------------- node-level entry points used by the pin tests ---------------- */
void oref_moment_matrix(double* M) { memcpy(M, M9, sizeof(M9)); }
void oref_shift_matrix(double ux, double uy, double* N) { shift9(ux, uy, N); }
void oref_thermal_moment_matrix(double* M) { memcpy(M, M5, sizeof(M5)); }
void oref_thermal_shift_matrix(double ux, double uy, double* N) { shift5(ux, uy, N); }

/* Central moments N(u) M f of nine DFs (Eq. 4b via Eq. 6). */
void oref_central_moments(const double* f, double ux, double uy, double* out) {
  double N[81], k[9];
  matvec(9, M9, f, k);
  shift9(ux, uy, N);
  matvec(9, N, k, out);
}

/* Inverse: DFs from central moments, M^-1 N^-1 kt. */
void oref_from_central(void* h, const double* kt, double ux, double uy, double* f) {
  oref_ctx* c = (oref_ctx*)h;
  double N[81], raw[9];
  shift9(ux, uy, N);
  forward_subst(9, N, kt, raw);
  matvec(9, c->Minv, raw, f);
}

void oref_thermal_central_moments(const double* g, double ux, double uy, double* out) {
  double N[25], k[5];
  matvec(5, M5, g, k);
  shift5(ux, uy, N);
  matvec(5, N, k, out);
}

void oref_thermal_from_central(void* h, const double* kt, double ux, double uy, double* g) {
  oref_ctx* c = (oref_ctx*)h;
  double N[25], raw[5];
  shift5(ux, uy, N);
  forward_subst(5, N, kt, raw);
  matvec(5, c->MTinv, raw, g);
}

/* One collision at one node: macros in mac[4] = (rho, ux, uy, T). */
void oref_collide_node(void* h, const double* f, const double* g, double* fs, double* gs,
                       double* mac) {
  oref_ctx* c = (oref_ctx*)h;
  double rho, ux, uy, T, Fx, Fy, Q;
  macros(c, f, g, &rho, &ux, &uy, &T, &Fx, &Fy, &Q);
  collide_flow(c, f, rho, ux, uy, Fx, Fy, fs);
  collide_thermal(c, g, ux, uy, T, Q, gs);
  mac[0] = rho;
  mac[1] = ux;
  mac[2] = uy;
  mac[3] = T;
}

void oref_rates(void* h, double* out) {
  oref_ctx* c = (oref_ctx*)h;
  out[0] = c->s3;
  out[1] = c->lambda2;
}

void oref_inverse_matrices(void* h, double* Minv, double* MTinv) {
  oref_ctx* c = (oref_ctx*)h;
  memcpy(Minv, c->Minv, sizeof(c->Minv));
  memcpy(MTinv, c->MTinv, sizeof(c->MTinv));
}

int oref_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Velocity of box side `side` (0 = x0, 1 = x1, 2 = y0, 3 = y1) for the
 * moving-wall bounce-back (not in the paper; used for thermal Couette flow). */
int oref_set_wall_velocity(void* h, int32_t side, double ux, double uy) {
  oref_ctx* c = (oref_ctx*)h;
  if (side < 0 || side > 3) return OREF_EINVAL;
  c->uw[side][0] = ux;
  c->uw[side][1] = uy;
  return OREF_OK;
}

void oref_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
