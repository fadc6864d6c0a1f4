"""The library's single-node collision, compiled for the host, against the FP64
oracle's collision (Eq. 2-10 and 15-24 with explicit matrices) on random
near-equilibrium states.

The step kernels inline `clbm::collide`, whose moment transforms are
tensor-product 1-D forms with the relaxation rates combined into scaled
constants (halved and quartered moments, regrouped sums); the oracle uses the
paper's matrices literally.  Here both collide the same pre-collision
populations, so a wrong sign, a dropped term or a mis-scaled constant in the
regrouped algebra shows up without a GPU.  Tolerances: FP64 to 2e-15
(rounding of some two hundred operations on values below 1; measured 2.8e-16);
the FP32 forms to 3e-7 absolute on populations of order 0.1 (FP32 rounding of
the same operations, the density and temperature carried as deviations;
measured up to 8e-8), far below any dropped term (the smallest, the force
Fx/2, is 1e-5 here)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1801_04577_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host_collide") / "host_collide.so")
    cmd = [nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-std=c++17", "--expt-relaxed-constexpr",
           f"-I{os.path.join(ROOT, 'include')}", "-gencode", "arch=compute_103a,code=sm_103a",
           "-o", out, os.path.join(HERE, "host_collide.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    L.host_collide.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp]
    L.host_collide.restype = C.c_int
    L.host_equilibrium.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
    L.host_equilibrium.restype = C.c_int
    L.host_wall.argtypes = [C.c_int, C.c_int, dp]
    L.host_wall.restype = C.c_double
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


CASES = {
    # name: Params overrides
    "cavity": dict(s_nu=1.511, s_b=1.0, s_4=1.0, lambda1=1.4495, T0=0.5, gbeta=1.5625e-4),
    "rb_source": dict(s_nu=0.98, s_b=1.2, s_4=1.3, lambda1=0.903, T0=0.5, gbeta=4.88e-6, Q=1e-4),
    "forced_rates": dict(s_nu=1.6, s_b=1.1, s_3=0.9, s_4=1.2, lambda1=0.6, lambda2=1.7, rho0=1.05,
                         T0=0.3, gbeta=0.01, Fvx=2e-5, Fvy=-3e-5, Q=2e-4),
    "viscous_heating": dict(s_nu=1.8, s_b=1.0, s_4=1.0, lambda1=1.2, T0=0.0, gbeta=1e-3, Q=0.0,
                            viscous_heating=1),
}


def _setup(name):
    p = I.Params(nx=4, ny=4, periodic_x=1, periodic_y=1, **CASES[name])
    g = I.Geometry(tbc=[I.dirichlet(0.0)], side_tbc=(-1, -1, -1, -1))
    o = oracle.Oracle(p, g)
    s3, l2 = o.rates()
    rates = np.array([p.s_nu, p.s_b, s3, p.s_4, p.lambda1, l2, p.rho0, p.T0, p.gbeta, p.Fvx, p.Fvy,
                      p.Q, p.cT2])
    f_rest, g_rest = o.equilibrium(p.rho0, 0.0, 0.0, p.T0)
    return p, o, rates, f_rest, g_rest


def _states(p, o, n, seed):
    """n pre-collision states: equilibria at random (rho, u, T) plus random
    non-equilibrium parts of a few percent of each weight."""
    r = I.splitmix64_uniform(seed, n * 18).reshape(n, 18)
    out = []
    for k in range(n):
        rho = p.rho0 * (1 + 0.03 * (2 * r[k, 0] - 1))
        ux, uy = 0.08 * (2 * r[k, 1] - 1), 0.08 * (2 * r[k, 2] - 1)
        T = p.T0 + 0.4 * (2 * r[k, 3] - 1)
        f, g = o.equilibrium(rho, ux, uy, T)
        w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        f = f + 0.03 * w9 * (2 * r[k, 4:13] - 1)
        g = g + 0.01 * (2 * r[k, 13:18] - 1)
        out.append((f, g))
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("form,tol", [(0, 2e-15), (1, 3e-7), (2, 3e-7)])
def test_host_collision_matches_oracle(harness, name, form, tol):
    p, o, rates, f_rest, g_rest = _setup(name)
    worst = 0.0
    for f, g in _states(p, o, 64, seed=1000 + form):
        fs, gs, _ = o.collide_node(f, g)
        d = np.ascontiguousarray(f - f_rest)
        h = np.ascontiguousarray(g - g_rest)
        qv = np.zeros(1)
        assert harness.host_collide(_dp(rates), int(p.viscous_heating), form, _dp(d), _dp(h), _dp(qv)) == 0
        err = max(np.abs(d + f_rest - fs).max(), np.abs(h + g_rest - gs).max())
        worst = max(worst, err)
    assert worst <= tol, (name, form, worst)


def test_harness_detects_a_mis_scaled_rate(harness):
    """The comparison is sharp enough to see a 1 % change of one rate (s_nu),
    the size of a wrong constant in the combined rates."""
    p, o, rates, f_rest, g_rest = _setup("cavity")
    f, g = _states(p, o, 1, seed=7)[0]
    fs, gs, _ = o.collide_node(f, g)
    bad = rates.copy()
    bad[0] *= 1.01
    d = np.ascontiguousarray(f - f_rest)
    h = np.ascontiguousarray(g - g_rest)
    qv = np.zeros(1)
    harness.host_collide(_dp(bad), 0, 0, _dp(d), _dp(h), _dp(qv))
    assert np.abs(d + f_rest - fs).max() > 1e-6


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_equilibrium_matches_oracle(harness, name):
    """The initialisation's equilibrium (Eq. 9 and Eq. 19 through the
    tensor-product inverse transforms, as deviations from the rest state)
    against the oracle's, which inverts the paper's matrices."""
    p, o, rates, f_rest, g_rest = _setup(name)
    r = I.splitmix64_uniform(31, 64 * 4).reshape(64, 4)
    worst = 0.0
    for a in r:
        rho = p.rho0 * (1 + 0.05 * (2 * a[0] - 1))
        ux, uy = 0.1 * (2 * a[1] - 1), 0.1 * (2 * a[2] - 1)
        T = p.T0 + 0.5 * (2 * a[3] - 1)
        f, g = o.equilibrium(rho, ux, uy, T)
        d, h = np.zeros(9), np.zeros(5)
        assert harness.host_equilibrium(_dp(rates), rho, ux, uy, T, _dp(d), _dp(h)) == 0
        worst = max(worst, np.abs(d + f_rest - f).max(), np.abs(h + g_rest - g).max())
    assert worst <= 2e-15, (name, worst)


@pytest.mark.parametrize("f32,tol", [(0, 4e-15), (1, 2e-6)])
def test_host_wall_rules_match_oracle(harness, f32, tol):
    """The fix-up's wall temperature (Eq. 28, one- and two-point), its form for
    walls off the link midpoint, and the midpoint value Eq. 26 imposes there,
    against the oracle's own implementations, on random conditions (Dirichlet,
    Neumann, Robin), link fractions and temperatures; relative to the scale of
    the temperatures involved (measured 3.3e-16 in FP64, 3.2e-7 in FP32)."""
    r = I.splitmix64_uniform(57, 400 * 8).reshape(400, 8)
    worst = 0.0
    for k, a in enumerate(r):
        kind = k % 3  # Dirichlet (b1 = 0), Neumann (b2 = 0), Robin
        b1 = 0.0 if kind == 0 else 0.5 + a[0]
        b2 = 0.0 if kind == 1 else 0.5 + a[1]
        b3 = 2 * a[2] - 1
        ne = [1.0, 0.7071067811865476, 0.55][k % 3]
        q = 0.05 + 0.95 * a[3]
        T1, T2, T3 = 2 * a[4] - 1, 2 * a[5] - 1, 2 * a[6] - 1
        have2 = a[7] > 0.2
        have3 = a[7] > 0.4
        scale = 1 + abs(b3) / max(b2, 1e-3) + abs(T1) + abs(T2) + abs(T3)
        got = harness.host_wall(0, f32, _dp(np.array([b1, b2, b3, ne, T1, T2, float(have2), 0, 0])))
        want = oracle.wall_temperature(b1, b2, b3, ne, T1, T2, have2)
        worst = max(worst, abs(got - want) / scale)
        got = harness.host_wall(1, f32, _dp(np.array([b1, b2, b3, ne, q, T1, T2, float(have2), 0])))
        want = oracle.wall_temperature_q(b1, b2, b3, ne, q, T1, T2, have2)
        worst = max(worst, abs(got - want) / scale)
        Tw = want
        got = harness.host_wall(2, f32, _dp(np.array([q, Tw, T1, T2, float(have2), T3, float(have3),
                                                      float(kind == 0), 0])))
        want = oracle.midpoint_temperature_q(q, Tw, T1, T2, T3, have2, have3, kind == 0)
        worst = max(worst, abs(got - want) / (scale + abs(Tw)))
    assert worst <= tol, worst
