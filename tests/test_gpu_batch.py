"""Batched solves (many lattices per launch) against single-lattice runs and the oracle."""
import numpy as np
import pytest

import oracle
from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

from _parity import TOL, compare

pytestmark = pytest.mark.gpu


def mixed_workloads():
    return [I.obstacle_channel(), I.natural_convection_cavity(48, 1e4),
            I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2), I.diffusion_channel(0.1, nx=4),
            I.periodic_box(133, 37), I.annulus(64, 2.6, Ra=1e4),
            I.natural_convection_cavity(20, 1e3)]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_lattice_runs(precision, autotune):
    """tol = 0: no lattice retires, so every lattice takes exactly max_steps steps
    and must reproduce its own single-lattice run."""
    ws = mixed_workloads()
    b = clbm.Batch(ws, precision, autotune=autotune)
    conv, res, steps = b.solve(0.0, 200, check_every=100)
    assert steps == 200
    assert (conv == -1).all()
    for i, w in enumerate(ws):
        s = clbm.from_workload(w, precision)
        s.step(200)
        ref = s.moments()
        got = b.moments(i)
        errs = compare(w, got, ref)
        assert max(errs.values()) <= (1e-13 if precision == "f64" else 1e-6), (i, w.name, errs)
        assert b.tile_width(i) in (32, 64, 128)
    b.close()


@pytest.mark.parametrize("precision,rounding", [("bf16", 0), ("bf16", 1), ("f16", 0), ("f16", 1)])
def test_batch_16bit_storage_matches_single_lattice_runs(precision, rounding):
    """16-bit storage of deviations, FP32 collision, in the batch: every lattice
    reproduces its own single-lattice run at the same storage format and
    rounding mode (the stochastic-rounding bits depend on the step and the
    lattice-local node only, so they are the same in both)."""
    ws = mixed_workloads()
    b = clbm.Batch(ws, precision, rounding=rounding)
    conv, res, steps = b.solve(0.0, 200, check_every=100)
    assert steps == 200 and (conv == -1).all()
    for i, w in enumerate(ws):
        s = clbm.from_workload(w, precision, rounding=rounding)
        s.step(200)
        errs = compare(w, b.moments(i), s.moments())
        print(precision, rounding, w.name, errs)
        assert max(errs.values()) <= 1e-6, (i, w.name, errs)
    b.close()


def test_batch_against_oracle_f64():
    ws = mixed_workloads()[:3]
    ws[2].init = I.random_fields(300, 70, seed=19, amp=0.02)  # every field O(1e-2)
    b = clbm.Batch(ws, "f64")
    b.solve(0.0, 300, check_every=150)
    for i, w in enumerate(ws):
        o = oracle.from_workload(w)
        o.step(300)
        errs = compare(w, b.moments(i), o.moments())
        assert max(errs.values()) <= TOL["f64"], (w.name, errs)
    b.close()


def test_batch_against_oracle_f32():
    """FP32 lattices of a batch (random initial fields with walls, obstacle and
    source; a cavity from rest; a noisy Rayleigh-Benard cell with a periodic
    seam) against the FP64 oracle, every field against its own largest value."""
    ws = [I.obstacle_channel(), I.natural_convection_cavity(48, 1e4),
          I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2)]
    ws[1].init = I.random_fields(48, 48, seed=17, amp=0.02)
    ws[2].init = I.random_fields(300, 70, seed=19, amp=0.02)
    b = clbm.Batch(ws, "f32")
    b.solve(0.0, 300, check_every=150)
    for i, w in enumerate(ws):
        o = oracle.from_workload(w)
        o.step(300)
        errs = compare(w, b.moments(i), o.moments())
        assert max(errs.values()) <= TOL["f32"], (w.name, errs)
    b.close()


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_batch_16bit_stochastic_against_oracle(precision):
    """The precision of batched solves (16-bit deviation storage, stochastic
    rounding, FP32 collision) against the FP64 oracle: the 64^2 Ra = 1e4
    cavity, solved inside a batch for 10,000 steps beside two other lattices,
    meets the single-lattice tolerances of the same format (field L2 of u_x,
    u_y, T and the cold-wall Nusselt number)."""
    from test_gpu_precision import CAVITY_TOL
    ws = [I.natural_convection_cavity(40, 1e3), I.natural_convection_cavity(64, 1e4),
          I.obstacle_channel()]
    b = clbm.Batch(ws, precision, rounding=1)
    conv, _, steps = b.solve(0.0, 10000, check_every=200)
    assert steps == 10000 and (conv == -1).all()
    w = ws[1]
    o = oracle.from_workload(w)
    o.step(10000)
    ref = o.moments()
    got = b.moments(1)
    l2 = [float(np.linalg.norm(a - r) / np.linalg.norm(r)) for a, r in zip(got[1:], ref[1:])]
    nu, nu_ref = -b.nusselt(1, 1, 64, 1.0), -o.nusselt(1, 64, 1.0)
    tol_l2, tol_nu = CAVITY_TOL[(precision, 1)]
    assert max(l2) < tol_l2, (precision, l2)
    assert abs(nu - nu_ref) / abs(nu_ref) < tol_nu, (precision, nu, nu_ref)
    b.close()


def test_batch_convergence_and_retirement():
    """Cavities reach the tolerance at different times; each converged lattice
    stops at its own step count with its residual below tol.  (The per-step
    residual of a closed cavity levels off at a small floor that shrinks with
    the size -- about 1e-6 at 16^2, 5e-8 at 32^2 in the oracle too -- so the
    cases are 32^2 and larger.)"""
    ws = [I.natural_convection_cavity(H, Ra) for H, Ra in ((32, 1e3), (40, 1e3), (32, 1e4))]
    ws[2].params.lambda1 = 1.0 / (0.12 / 0.4 + 0.5)
    b = clbm.Batch(ws, "f64")
    tol = 2e-7
    conv, res, steps = b.solve(tol, 40000, check_every=50)
    assert (conv > 0).all(), conv
    assert (res < tol).all()
    assert steps == conv.max()
    assert (conv % 50 == 0).all() and (conv >= 100).all()  # the first check only takes a snapshot
    for i, w in enumerate(ws):
        v = b.view(i)
        assert clbm.clbm_time(v) == conv[i]
        # the frozen state is the single-lattice state after the same number of steps
        s = clbm.from_workload(w, "f64")
        s.step(int(conv[i]))
        errs = compare(w, b.moments(i), s.moments())
        assert max(errs.values()) <= 1e-13
    b.close()


def test_batch_flags_diverged_lattice():
    ws = [I.natural_convection_cavity(24, 1e3), I.obstacle_channel()]
    T = np.full((24, 24), 0.5)
    T[3, 4] = np.nan
    ws[0].init = I.Fields(T=T)
    b = clbm.Batch(ws, "f32")
    conv, res, steps = b.solve(1e-30, 400, check_every=100)
    assert conv[0] == -2 and not np.isfinite(res[0])
    assert conv[1] == -1 and np.isfinite(res[1]) and res[1] < 1.0
    assert steps == 400
    b.close()


def test_batch_with_walls_off_the_link_midpoint():
    """Lattices with interpolated walls inside a batch reproduce their own
    single-lattice runs."""
    ws = [I.annulus(48, 2.6, Ra=1e4, interpolated=True),
          I.offset_channel(12, 0.3, 0.8, 0.1, 0.1, 1e-5, top_tbc=(1.0, 0.2, 0.0), Q=1e-3),
          I.natural_convection_cavity(24, 1e4)]
    b = clbm.Batch(ws, "f64", autotune=False)
    b.solve(0.0, 200, check_every=100)
    for i, w in enumerate(ws):
        s = clbm.from_workload(w, "f64")
        s.step(200)
        errs = compare(w, b.moments(i), s.moments())
        assert max(errs.values()) <= 1e-13, (w.name, errs)
    b.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_config4_generator_cavities_against_oracle(precision):
    """Cavities of the 512-cavity generator (uneven sides, both orientations,
    mixed Dirichlet / Neumann / Robin sides, heat sources, Ra up to 1e6; sides
    32..40 here so the oracle stays quick) in one batch, each started from
    seeded random rho, u, T (so that every field is O(1e-2) from the first
    step: from rest the velocity of these cavities is still far below U after a
    few hundred steps) and compared with the FP64 oracle after 100 steps, every
    field against its own largest value.  (Several of these cavities have
    s_nu above 1.9 -- small H at Ra ~ 1e5 -- and barely damp the random start:
    after 300 steps their rounding differences reach 1.3e-12 in FP64 and 2.1e-5
    in FP32, relative, so the comparison is made earlier.)"""
    ws = I.random_cavities(6, hmax=40)
    for k, w in enumerate(ws):
        w.init = I.random_fields(w.params.nx, w.params.ny, seed=400 + k, amp=0.02)
    b = clbm.Batch(ws, precision, autotune=True)
    conv, _, steps = b.solve(0.0, 100, check_every=50)
    assert steps == 100 and (conv == -1).all()
    for i, w in enumerate(ws):
        o = oracle.from_workload(w)
        o.step(100)
        errs = compare(w, b.moments(i), o.moments())
        assert max(errs.values()) <= TOL[precision], (w.name, errs)
    b.close()
