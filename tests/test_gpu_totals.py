"""Conservation sums on the GPU (clbm_totals): FP64 sums of the stored
post-collision distributions over the fluid nodes.

Checked against the oracle's moments (sum f = sum rho, sum f e = sum (rho u +
F/2), sum g = sum (T + Q/2): the post-collision conserved moments of Eq. 7 and
the zeroth thermal moment of Eq. 23) and against the conservation laws on a
lattice without walls."""
import numpy as np
import pytest

import oracle
from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _expected(w, moments):
    p = w.params
    rho, ux, uy, T = moments
    fl = np.ones_like(rho, bool) if w.geom.solid is None else w.geom.solid == 0
    n = fl.sum()
    Fy = p.Fvy + p.rho0 * p.gbeta * (T - p.T0)
    return np.array([rho[fl].sum(), (rho * ux)[fl].sum() + 0.5 * n * p.Fvx,
                     (rho * uy + 0.5 * Fy)[fl].sum(), T[fl].sum() + 0.5 * n * p.Q]), n


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("name", ["obstacle", "rb", "cavity", "annulus"])
def test_totals_match_oracle(precision, tol, name):
    w = {"obstacle": lambda: I.obstacle_channel(),
         "rb": lambda: I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2),
         "cavity": lambda: I.natural_convection_cavity(48, 1e4),
         "annulus": lambda: I.annulus(64, 2.6, Ra=1e4)}[name]()
    s = clbm.from_workload(w, precision)
    o = oracle.from_workload(w)
    s.step(37)
    o.step(37)
    got = s.totals()
    ref, n = _expected(w, o.moments())
    scale = np.array([w.params.rho0, w.u_scale, w.u_scale, max(abs(w.params.T0), w.dT)]) * n
    assert np.all(np.abs(got - ref) <= tol * scale), (got, ref, np.abs(got - ref) / scale)
    # the same state gives the same sums (fixed-order reduction)
    np.testing.assert_array_equal(s.totals(), got)


def test_totals_conservation_without_walls():
    """Doubly periodic box with a body force, buoyancy and a heat source: the
    mass is constant, the momentum grows by the summed force of each step and
    sum g by N Q."""
    w = I.periodic_box(133, 37)
    p = w.params
    s = clbm.from_workload(w, "f64")
    n = p.nx * p.ny
    prev = s.totals()
    for _ in range(40):
        s.step(1)
        cur = s.totals()
        rho, ux, uy, T = s.moments()
        Fy = (p.Fvy + p.rho0 * p.gbeta * (T - p.T0)).sum()
        assert cur[0] == pytest.approx(prev[0], rel=1e-14)
        assert cur[1] - prev[1] == pytest.approx(n * p.Fvx, rel=1e-8, abs=1e-13)
        assert cur[2] - prev[2] == pytest.approx(Fy, rel=1e-8, abs=1e-13)
        assert cur[3] - prev[3] == pytest.approx(n * p.Q, rel=1e-8)
        prev = cur
