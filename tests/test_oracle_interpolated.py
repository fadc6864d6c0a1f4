"""Pins of the oracle's walls off the link midpoint (no counterpart in the paper,
which puts every wall half-way along its links).

The flow follows the linear interpolated bounce-back of Bouzidi, Firdaouss and
Lallemand; the temperature keeps Eq. 26 at the link midpoint with the value of
the wall profile there.  Pinned by: the wall formulas on exact quadratic
profiles; q = 1/2 reproducing the paper's scheme bit for bit; channels whose
walls sit at arbitrary fractions of a link, where the steady temperature
(linear, or parabolic with a heat source; Dirichlet and Robin walls) is
reproduced to rounding and the Poiseuille velocity converges at second order;
and the annulus, where the interpolated walls beat the staircase."""
import math

import numpy as np
import pytest

import oracle
from paper_1801_04577_gb300 import inputs as I


def _quadratic(seed):
    r = I.splitmix64_uniform(seed, 8)
    a0, a1, a2 = 2 * r[0] - 1, 2 * r[1] - 1, 2 * r[2] - 1
    return (lambda s: a0 + a1 * s + a2 * s * s), (lambda s: a1 + 2 * a2 * s), r[3:]


@pytest.mark.parametrize("seed", range(12))
def test_wall_formulas_exact_for_quadratic_profiles(seed):
    """T(s) quadratic along the link, s measured from the wall into the fluid:
    T_w recovered from (T(q), T(1+q)) and the condition b1 dT/dn + b2 T_w = b3
    with dT/dn = -T'(0)/(n.e); the midpoint value T(q - 1/2) recovered by
    every branch (q below and above 1/2, flux and Dirichlet walls)."""
    T, dT, r = _quadratic(1000 + seed)
    q = 0.02 + 0.98 * r[0]
    ne = 0.2 + 0.8 * r[1]
    b1, b2 = r[2], 0.1 + r[3]
    b3 = b1 * (-dT(0.0) / ne) + b2 * T(0.0)
    Tw = oracle.wall_temperature_q(b1, b2, b3, ne, q, T(q), T(1 + q))
    assert Tw == pytest.approx(T(0.0), abs=1e-12)
    for dirichlet in (False, True):
        Tm = oracle.midpoint_temperature_q(q, T(0.0), T(q), T(1 + q), T(2 + q), dirichlet=dirichlet)
        assert Tm == pytest.approx(T(q - 0.5), abs=1e-11)
    # Dirichlet wall (b1 = 0): T_w = b3
    assert oracle.wall_temperature_q(0.0, 1.0, 0.37, ne, q, T(q), T(1 + q)) == pytest.approx(0.37, abs=1e-15)


def test_wall_formulas_one_sided_exact_for_lines():
    lin = lambda s: 0.3 - 0.7 * s  # noqa: E731
    for q in (0.1, 0.5, 0.9):
        b1, b2, ne = 1.0, 0.4, 0.8
        b3 = b1 * (0.7 / ne) + b2 * lin(0.0)
        Tw = oracle.wall_temperature_q(b1, b2, b3, ne, q, lin(q), 0.0, have_T2=False)
        assert Tw == pytest.approx(lin(0.0), abs=1e-14)


@pytest.mark.parametrize("have2", [True, False])
def test_wall_temperature_at_half_is_eq28(have2):
    for (b1, b2, b3, ne, T1, T2) in [(1, 1, 0.2, 0.8, 0.5, 0.4), (0, 1, 0.3, 1, 0.2, 0.9), (1, 0, 0.05, 0.6, 0.1, 0.3)]:
        a = oracle.wall_temperature(b1, b2, b3, ne, T1, T2, have2)
        b = oracle.wall_temperature_q(b1, b2, b3, ne, 0.5, T1, T2, have2)
        assert b == pytest.approx(a, rel=1e-14, abs=1e-15)


def test_half_fraction_is_the_papers_scheme():
    """Every link listed (diagonals included) with q = 1/2: the same numbers as
    the half-way walls, bit for bit, with convection."""
    a = I.annulus(32, 2.6, Ra=1e4)
    b = I.annulus(32, 2.6, Ra=1e4, interpolated=True)
    b.geom.link_q = np.full(b.geom.n_links, 0.5)
    oa, ob = oracle.from_workload(a), oracle.from_workload(b)
    oa.step(300)
    ob.step(300)
    for x, y in zip(oa.moments(), ob.moments()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("N,qb,qt,top,Q", [
    (8, 0.3, 0.8, None, 0.0),                # linear, Dirichlet
    (8, 0.3, 0.8, (1.0, 0.2, 0.0), 1e-3),    # parabola, Robin top (q >= 1/2)
    (16, 0.3, 0.2, (1.0, 0.1, 0.0), 1e-3),   # parabola, Robin top (q < 1/2)
    (8, 0.7, 0.1, None, 1e-3),               # parabola, Dirichlet, small q
    (8, 0.05, 0.02, (1.0, 0.2, 0.1), 1e-3),  # both walls very close to the nodes
])
def test_offset_walls_temperature_exact(N, qb, qt, top, Q):
    """Walls at y = 1 - qb and y = N + qt: the steady temperature (linear, or
    the parabola of a uniform source) is reproduced to rounding."""
    nu, alpha = 0.1, 0.1
    w = I.offset_channel(N, qb, qt, nu, alpha, 1e-5, top_tbc=top, Q=Q)
    o = oracle.from_workload(w)
    o.step(int(40 * (N + 1) ** 2 / alpha) + 2000)
    T = o.moments()[3][:, 0]
    _, Ta = I.offset_channel_exact(w, nu, alpha)
    assert np.abs(T[1:-1] - Ta[1:-1]).max() < 1e-11


def test_offset_walls_poiseuille_second_order():
    """Interpolated bounce-back: the Poiseuille velocity between walls at
    fractions 0.3 and 0.8 converges at second order (the half-way walls of the
    paper reproduce it exactly, but only at q = 1/2)."""
    nu, alpha, Fx = 0.1, 0.1, 1e-5
    errs = []
    for N in (8, 16):
        w = I.offset_channel(N, 0.3, 0.8, nu, alpha, Fx)
        o = oracle.from_workload(w)
        o.step(int(40 * (N + 1) ** 2 / nu) + 2000)
        ux = o.moments()[1][:, 0]
        ua, _ = I.offset_channel_exact(w, nu, alpha)
        errs.append(np.abs(ux[1:-1] - ua[1:-1]).max() / ua.max())
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 3.5


def _annulus_conduction_E2(n, interpolated):
    w = I.annulus(n, 2.6, gravity=False, alpha=0.1, interpolated=interpolated)
    o = oracle.from_workload(w)
    o.step(int(17000 * (n / 64) ** 2))
    T = o.moments()[3]
    ro = n / 2 - 1
    ri = ro / 2.6
    H = ro - ri
    c = (n - 1) / 2
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - c, yy - c)
    A, B = np.linalg.solve([[1, math.log(ri)], [1 / H, 1 / ro + math.log(ro) / H]], [1, 0])
    Ta = A + B * np.log(r)
    fl = w.geom.solid == 0
    return math.sqrt(((T[fl] - Ta[fl]) ** 2).sum() / (Ta[fl] ** 2).sum())


def test_annulus_interpolated_walls_beat_the_staircase():
    """Steady conduction in the annulus (Dirichlet inside, Robin outside)
    against T = A + B ln r: the interpolated walls are at least three times
    more accurate than the half-way staircase at 32^2 and 64^2, and improve
    with the grid."""
    e32 = (_annulus_conduction_E2(32, False), _annulus_conduction_E2(32, True))
    e64 = (_annulus_conduction_E2(64, False), _annulus_conduction_E2(64, True))
    assert e32[1] < e32[0] / 3
    assert e64[1] < e64[0] / 3
    assert e64[1] < 0.5 * e32[1]
    assert e64[1] < 1.2e-3


@pytest.mark.parametrize("N,qb,qt,top,Q", [
    (8, 0.3, 0.8, None, 0.0),                # linear; bottom q < 1/2, top q > 1/2; Dirichlet
    (8, 0.7, 0.2, (1.0, 0.5, 0.1), 0.0),     # linear; bottom q > 1/2, top q < 1/2; Robin top
    (8, 0.3, 0.8, (1.0, 0.2, 0.0), 1e-3),    # parabola, Robin top (q >= 1/2)
    (16, 0.3, 0.2, (1.0, 0.1, 0.0), 1e-3),   # parabola, Robin top (q < 1/2)
    (8, 0.7, 0.1, None, 1e-3),               # parabola, Dirichlet, small q
])
def test_offset_walls_nusselt_is_the_exact_wall_flux(N, qb, qt, top, Q):
    """The wall gradient off the link midpoint, through the Nusselt number of
    the listed links: with walls at y_b = 1 - qb and y_t = N + qt, the steady
    profile T = T_b + s x + Q/(2 alpha) x (L - x) (x = y - y_b) has the exact
    outward gradients dT/dn = -(s + Q L/(2 alpha)) at the bottom wall and
    s - Q L/(2 alpha) at the top wall.  oref_nusselt(4 + k) with length = dT = 1
    is the mean of dT/dn over the links of condition k, so it must return these
    fluxes (to the rounding of the steady state).  A slip in the gradient's
    weights, in its sign or in the q used (for instance q where 1 - q belongs)
    moves it by O(1)."""
    nu, alpha = 0.1, 0.1
    w = I.offset_channel(N, qb, qt, nu, alpha, 1e-5, top_tbc=top, Q=Q)
    o = oracle.from_workload(w)
    o.step(int(40 * (N + 1) ** 2 / alpha) + 2000)
    ny = w.params.ny
    yb, yt = 1.0 - qb, (ny - 2) + qt
    L = yt - yb
    b1, b2, b3 = w.geom.tbc[1]
    c = Q / (2.0 * alpha)
    s = (b3 - b2 * 1.0 + b1 * c * L) / (b1 + b2 * L)
    assert o.nusselt(4, 1.0, 1.0) == pytest.approx(-(s + c * L), abs=1e-9)
    assert o.nusselt(5, 1.0, 1.0) == pytest.approx(s - c * L, abs=1e-9)
    # the fluxes are O(1/L); the tolerance is far below any formula slip
    assert min(abs(s + c * L), abs(s - c * L)) > 1e-2 or abs(s) > 1e-2
