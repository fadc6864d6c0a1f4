"""clbm_damp_period2 removes the neutral period-2 component that a restart
from non-equilibrium fields excites (see the oracle characterisation test)."""
import numpy as np
import pytest

from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _alternation(s):
    a = s.nusselt(0, 32, 1.0)
    s.step(1)
    b = s.nusselt(0, 32, 1.0)
    return abs(a - b), 0.5 * (a + b)


@pytest.mark.parametrize("presteps", [2, 32])
def test_damp_period2_removes_alternation(presteps):
    """The filter cancels the period-2 component present when it is applied
    (measured: the step-to-step Nusselt alternation drops about six-fold; what
    is left is fed by the slowly decaying perturbation itself) and leaves the
    slow evolution of the two-step mean unchanged."""
    w = I.natural_convection_cavity(32, 1e4)
    s = clbm.from_workload(w, "f64")
    s.step(40000)
    rho, ux, uy, T = s.moments()
    nu_ref = s.nusselt(0, 32, 1.0)
    yy, xx = np.mgrid[0:32, 0:32]
    f = I.Fields(ux=ux, uy=uy, T=T + 2e-2 * np.sin(np.pi * (xx + 0.5) / 32))
    plain = clbm.Solver(w.params, w.geom, "f64", init=f)
    damped = clbm.Solver(w.params, w.geom, "f64", init=f)
    damped.step(presteps)
    clbm.clbm_damp_period2(damped.ctx)
    plain.step(presteps)
    plain.step(6000)
    damped.step(6000)
    amp_plain, mean_plain = _alternation(plain)
    amp_damped, mean_damped = _alternation(damped)
    assert amp_plain > 1e-5
    assert amp_damped < 0.3 * amp_plain
    assert abs(mean_damped - mean_plain) < 1e-4 * abs(nu_ref)
    assert abs(mean_plain - nu_ref) < 5e-3 * abs(nu_ref)


def test_damp_period2_needs_a_step():
    w = I.natural_convection_cavity(16, 1e4)
    s = clbm.from_workload(w, "f32")
    with pytest.raises(clbm.ClbmError):
        clbm.clbm_damp_period2(s.ctx)
