"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: FP64 storage/collision within 1e-12 of the oracle and FP32 within
1e-5, per field, as max-norm relative to the field's largest value (the
density as rho - rho0 relative to rho0).  Cases cover several warp tiles, ragged
row lengths, both kinds of walls, periodic seams, masks with listed links,
curved walls, the heat source and the body force.
"""
import copy

import numpy as np
import pytest

import oracle
from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

from _parity import TOL, compare, rel_inf, run_pair

pytestmark = pytest.mark.gpu


def _assert_within(errs, tol, label):
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, f"{label}: errors {errs} exceed {tol}"


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_cavity_64_ra1e4_10000_steps(precision):
    """Differentially heated cavity, 64^2, Ra = 1e4, 10,000 steps (Sec. 3.3 setup)."""
    w = I.natural_convection_cavity(64, 1e4)
    errs, (s, o) = run_pair(w, 10000, precision)
    _assert_within(errs, TOL[precision], f"cavity {precision}")
    tol_nu = 1e-11 if precision == "f64" else 1e-4
    for side in (0, 1, 2, 3):
        a = s.nusselt(side, 64, 1.0)
        b = o.nusselt(side, 64, 1.0)
        assert abs(a - b) <= tol_nu * max(1.0, abs(b)), (side, a, b)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ragged_mask_links_mixed_walls(precision):
    """37 x 19 box: walls on all sides with Dirichlet/Robin/Neumann conditions,
    a solid obstacle with listed links, a source and a body force."""
    w = I.obstacle_channel()
    errs, _ = run_pair(w, 400, precision)
    _assert_within(errs, TOL[precision], f"obstacle {precision}")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_periodic_x_several_tiles(precision):
    """Rayleigh-Benard setup on 300 x 70 (ragged against the 128/64-node warp
    tiles, periodic seam inside a tile) with a source, started from seeded
    random rho, u, T so that every field is O(1e-2) throughout."""
    w = I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2)
    w.init = I.random_fields(300, 70, seed=23, amp=0.02)
    errs, _ = run_pair(w, 300, precision)
    _assert_within(errs, TOL[precision], f"rb {precision}")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_doubly_periodic_box(precision):
    w = I.periodic_box(133, 37)
    errs, _ = run_pair(w, 200, precision)
    _assert_within(errs, TOL[precision], f"periodic {precision}")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_annulus_curved_walls(precision):
    """Annulus with curved Dirichlet (inner) and Robin (outer) walls."""
    w = I.annulus(96, 2.6, Ra=1e4)
    errs, _ = run_pair(w, 300, precision)
    _assert_within(errs, TOL[precision], f"annulus {precision}")


def test_annulus_nusselt_and_residual_f64():
    w = I.annulus(64, 2.6, Ra=1e4)
    s = clbm.from_workload(w, "f64")
    o = oracle.from_workload(w)
    s.step(500)
    o.step(500)
    for which in (4, 5):
        a, b = s.nusselt(which, w.length, 1.0), o.nusselt(which, w.length, 1.0)
        assert a == pytest.approx(b, rel=1e-11, abs=1e-13)
    assert s.residual() == pytest.approx(o.residual(), rel=1e-8)


@pytest.mark.parametrize("nx", [1, 4, 130])
def test_diffusion_with_source_exact_gpu(nx, paper_values):
    """Sec. 3.1 on the GPU, including a single-column lattice (nx = 1)."""
    pv = paper_values["diffusion_with_source"]
    for case in pv["cases"]:
        w = I.diffusion_channel(case["alpha"], L=pv["L"], nx=nx)
        s = clbm.from_workload(w, "f64")
        s.step(6000)
        T = s.moments()[3]
        Ta = I.diffusion_exact(pv["L"])
        E2 = np.sqrt(((T - Ta[:, None]) ** 2).sum(axis=0) / (Ta ** 2).sum())
        assert E2.max() < 1e-12


def test_poiseuille_exact_gpu():
    ny, nu, Fx = 8, 0.1, 1e-5
    w = I.poiseuille_channel(ny, nu, Fx, nx=64)
    s = clbm.from_workload(w, "f64")
    s.step(8000)
    ux = s.moments()[1]
    ua = I.poiseuille_exact(ny, nu, Fx)
    assert np.abs(ux - ua[:, None]).max() / ua.max() < 1e-10


def test_residual_and_nusselt_match_oracle_cavity():
    w = I.natural_convection_cavity(48, 1e4)
    s = clbm.from_workload(w, "f64")
    o = oracle.from_workload(w)
    s.step(700)
    o.step(700)
    assert s.residual() == pytest.approx(o.residual(), rel=1e-9)
    assert s.time == 700


def test_zero_steps_is_identity():
    w = I.obstacle_channel()
    s = clbm.from_workload(w, "f64")
    before = s.moments()
    s.step(0)
    after = s.moments()
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


def test_nan_is_reported_unstable():
    """A NaN placed in the initial temperature (host input) is caught by the
    residual check as CLBM_EUNSTABLE."""
    w = I.obstacle_channel()
    T = np.full((w.params.ny, w.params.nx), 0.5)
    T[5, 7] = np.nan
    w.init = I.Fields(T=T)
    s = clbm.from_workload(w, "f32")
    s.step(2)
    with pytest.raises(clbm.ClbmError) as ei:
        s.residual()
    assert ei.value.status == clbm.CLBM_EUNSTABLE


def test_invalid_arguments_gpu():
    w = I.natural_convection_cavity(16, 1e4)
    s = clbm.Solver(w.params, None, "f32")
    with pytest.raises(clbm.ClbmError) as ei:
        s.step(1)  # walls not described yet
    assert ei.value.status == clbm.CLBM_EINVAL
    with pytest.raises(clbm.ClbmError):
        clbm.clbm_set_boundaries(s.ctx, None, w.geom.tbc, (0, 1, 2, 7))
    with pytest.raises(clbm.ClbmError):
        s.residual()  # no step since initialisation


def test_full_size_rayleigh_benard_f32_against_oracle():
    """The benchmark lattice itself (4096 x 2048, FP32, the launch
    configuration the benchmark times), started from seeded random rho, u and
    T (amplitude 0.02 around rest, T in 0.25..0.75) so that every field is
    O(1e-2) from the first step: five steps (a replayed 4-step graph and one
    single launch) compared node by node with the FP64 oracle, every field
    against its own largest value."""
    w = I.rayleigh_benard(4096, 2048)
    w.init = I.random_fields(4096, 2048, seed=1801045771, amp=0.02)
    s = clbm.from_workload(w, "f32")
    o = oracle.from_workload(w)
    s.step(5)
    o.step(5)
    errs = compare(w, s.moments(), o.moments())
    _assert_within(errs, TOL["f32"], "rb4096 f32")


@pytest.mark.parametrize("precision,rounding", [("f32", 0), ("bf16", 1), ("f64", 0)])
@pytest.mark.parametrize("name", ["cavity", "obstacle"])
def test_graph_replay_matches_single_launches(precision, rounding, name):
    """clbm_step(n >= 32) replays a captured 32-step graph (device-side step
    counter for the stochastic-rounding key); the result is bit-identical to n
    single-step calls."""
    w = I.natural_convection_cavity(48, 1e4) if name == "cavity" else I.obstacle_channel()
    a = clbm.from_workload(w, precision, rounding=rounding)
    b = clbm.from_workload(w, precision, rounding=rounding)
    a.step(3)
    b.step(3)  # odd start: exercises the graph keyed on an odd step and buffer 1
    a.step(70)
    for _ in range(70):
        b.step(1)
    assert a.time == b.time == 73
    for x, y in zip(a.moments(), b.moments()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", ["cavity", "obstacle"])
def test_viscous_heating_matches_oracle(precision, name):
    """Viscous dissipation source (Sec. 3.2) on a box lattice (fused launch) and
    on a masked one with source, force and mixed walls."""
    w = I.natural_convection_cavity(48, 1e4) if name == "cavity" else I.obstacle_channel()
    w.params.viscous_heating = 1
    if name == "cavity":
        w.params.Fvx = 2e-5  # stronger shear so the source matters
    errs, (s, o) = run_pair(w, 600, precision)
    _assert_within(errs, TOL[precision], f"viscous {name} {precision}")
    a, b = s.nusselt(0, w.length, 1.0), o.nusselt(0, w.length, 1.0)
    assert abs(a - b) <= (1e-11 if precision == "f64" else 1e-4) * max(1.0, abs(b))


def test_viscous_heating_channel_profile_gpu():
    """Sec. 3.2 on the GPU: the steady channel temperature matches the exact
    quartic profile as closely as the oracle does (E2 ~ 7e-3 at L = 16)."""
    L, nu, alpha, Fx = 16, 0.1, 0.1, 1e-5
    w = I.dissipation_channel(L, nu, alpha, Fx, nx=64)
    s = clbm.from_workload(w, "f64")
    s.step(int(20 * L * L / alpha) + 2000)
    T = s.moments()[3]
    Ta = I.dissipation_exact(L, nu, alpha, Fx)
    E2 = np.sqrt(((T - Ta[:, None]) ** 2).sum(axis=0) / (Ta ** 2).sum())
    assert E2.max() < 1e-2
    o = oracle.from_workload(I.dissipation_channel(L, nu, alpha, Fx, nx=1))
    o.step(int(20 * L * L / alpha) + 2000)
    np.testing.assert_allclose(T[:, 0], o.moments()[3][:, 0], rtol=1e-10, atol=1e-18)


def _offset_channel_convective():
    """Walls at fractions 0.3 / 0.8 of a link, Robin top wall, heat source,
    body force (peak velocity ~0.02, so FP32 rounding of the state stays well
    below the tolerance): every off-midpoint rule is active."""
    return I.offset_channel(12, 0.3, 0.8, 0.1, 0.1, 1e-4, top_tbc=(1.0, 0.2, 0.0), Q=1e-3)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", ["annulus", "channel", "channel_small_q"])
def test_walls_off_the_link_midpoint_match_oracle(precision, name):
    """Interpolated walls (no counterpart in the paper): the curved annulus with
    every link's crossing fraction (diagonals included, convection on), and
    offset channels, against the oracle."""
    if name == "annulus":
        w, steps = I.annulus(64, 2.6, Ra=1e4, interpolated=True), 400
    elif name == "channel":
        w, steps = _offset_channel_convective(), 3000
    else:  # Dirichlet walls close to the nodes: the far-node extrapolation
        w, steps = I.offset_channel(10, 0.05, 0.1, 0.1, 0.1, 1e-4, Q=1e-3), 3000
    # u_y and rho - rho0 vanish in the exact channel flow: compared against U and rho0
    errs, (s, o) = run_pair(w, steps, precision,
                            vanishing=() if name == "annulus" else ("rho", "uy"))
    _assert_within(errs, TOL[precision], f"{name} {precision}")
    which = 4 if name == "annulus" else 5
    a, b = s.nusselt(which, w.length, 1.0), o.nusselt(which, w.length, 1.0)
    assert abs(a - b) <= (1e-11 if precision == "f64" else 1e-4) * max(1.0, abs(b))


def test_offset_channel_steady_temperature_gpu():
    """The steady parabola between offset walls (Robin top, source) on the GPU
    in FP64, to rounding, as in the oracle."""
    nu, alpha = 0.1, 0.1
    w = I.offset_channel(8, 0.3, 0.2, nu, alpha, 1e-5, top_tbc=(1.0, 0.2, 0.0), Q=1e-3)
    s = clbm.from_workload(w, "f64")
    s.step(int(40 * 81 / alpha) + 2000)
    T = s.moments()[3][:, 0]
    _, Ta = I.offset_channel_exact(w, nu, alpha)
    assert np.abs(T[1:-1] - Ta[1:-1]).max() < 1e-11


def test_half_fraction_links_are_the_half_way_walls_gpu():
    """Listing every link with q = 1/2 changes nothing, bit for bit."""
    a = I.annulus(48, 2.6, Ra=1e4)
    b = I.annulus(48, 2.6, Ra=1e4, interpolated=True)
    b.geom.link_q = np.full(b.geom.n_links, 0.5)
    sa, sb = clbm.from_workload(a, "f32"), clbm.from_workload(b, "f32")
    sa.step(200)
    sb.step(200)
    for x, y in zip(sa.moments(), sb.moments()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", ["row", "column", "two_rows", "single_node"])
def test_degenerate_lattices_match_oracle(precision, case):
    """Degenerate shapes: one periodic row (every pull in y wraps onto the
    node itself), one periodic column, a two-row walled channel (every node is
    a boundary node, with both walls on each column) and a single node."""
    if case == "row":
        w = I.periodic_box(200, 1)
    elif case == "column":
        w = I.periodic_box(1, 77)
    elif case == "two_rows":
        w = I.poiseuille_channel(2, 0.1, 1e-4, nx=9)
    else:
        w = I.periodic_box(1, 1)
    # the two-row channel flow has u_y = 0 and rho = rho0 exactly: compared against U and rho0
    errs, _ = run_pair(w, 150, precision, vanishing=("rho", "uy") if case == "two_rows" else ())
    _assert_within(errs, TOL[precision], f"{case} {precision}")


@pytest.mark.parametrize("precision,rounding", [("f64", 0), ("f32", 0), ("bf16", 1)])
@pytest.mark.parametrize("name", ["cavity", "rb_periodic_x", "periodic_box", "viscous"])
def test_all_fluid_mask_is_bit_identical_to_the_box(precision, rounding, name):
    """A mask with no solid node makes the lattice 'masked': flags, the three-class
    tile table, and the fused launch whose flagged tiles store node by node and
    leave the listed nodes to the boundary blocks.  The walls are the same, so
    every value must equal the unmasked run's bit for bit."""
    if name == "cavity":
        w = I.natural_convection_cavity(150, 1e4)
    elif name == "rb_periodic_x":
        w = I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2)
    elif name == "periodic_box":
        w = I.periodic_box(133, 37)
    else:  # the viscous dissipation source (a 15th plane stored by the tiles)
        w = I.natural_convection_cavity(70, 1e5)
        w.params.viscous_heating = 1
    m = copy.deepcopy(w)
    m.geom.solid = np.zeros((w.params.ny, w.params.nx), np.uint8)
    a = clbm.from_workload(w, precision, rounding=rounding)
    b = clbm.from_workload(m, precision, rounding=rounding)
    a.step(41)
    b.step(41)
    for x, y in zip(a.moments(), b.moments()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("vh", [0, 1])
def test_thermal_couette_matches_oracle(precision, vh):
    """Thermal Couette flow (moving top wall, not in the paper) against the
    oracle while the profiles develop (2,000 steps), and, in FP64, the steady
    profiles against the closed form as the oracle pin states them."""
    nu, alpha, H, Uw = 0.1, 0.08, 16, 0.05
    w = I.couette_channel(H, Uw, nu, alpha, viscous_heating=vh)
    # u_y and rho - rho0 vanish in the exact Couette flow: compared against U and rho0
    errs, _ = run_pair(w, 2000, precision, vanishing=("rho", "uy"))
    _assert_within(errs, TOL[precision], f"couette vh={vh} {precision}")
    if precision == "f64":
        s = clbm.from_workload(w, "f64")
        s.step(int(40 * H * H / min(nu, alpha)))
        _, ux, _, T = s.moments()
        u_ex, T_ex = I.couette_exact(w, nu, alpha)
        assert np.abs(ux[:, 0] - u_ex).max() < 1e-12 * Uw
        lin = 1 - (np.arange(H) + 0.5) / H
        tol = 1e-5 * (T_ex - lin).max() if vh else 1e-11
        assert np.abs(T[:, 0] - T_ex).max() < tol


def test_moving_wall_velocity_rejects_bad_side():
    w = I.couette_channel()
    s = clbm.from_workload(w, "f32")
    with pytest.raises(clbm.ClbmError) as ei:
        clbm.clbm_set_wall_velocity(s.ctx, 4, 0.1)
    assert ei.value.status == clbm.CLBM_EINVAL
