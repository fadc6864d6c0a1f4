"""Table 1 of the paper (Sec. 3.3) reproduced at the paper's grids.

The four natural-convection cavities (Ra = 1e3, 1e4, 1e5, 1e6 on 128^2, 192^2,
192^2, 256^2, Pr = 0.71, U = 0.1) are solved together as one batch to steady
state; the midline velocity maxima, their locations and the cold-wall Nusselt
number are compared with the paper's CLBM column."""
import numpy as np
import pytest

from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

from _table1 import table1_quantities

pytestmark = pytest.mark.gpu


def test_table1_at_paper_grids(paper_values):
    t1 = paper_values["table1_clbm"]
    ws = [I.natural_convection_cavity(G, Ra, Pr=t1["Pr"], U=t1["U"]) for G, Ra in zip(t1["grid"], t1["Ra"])]
    b = clbm.Batch(ws, "f32")
    conv, res, steps = b.solve(2e-9, 2_000_000, check_every=1000)
    assert (conv > 0).all(), (conv, res)
    for k, (w, G) in enumerate(zip(ws, t1["grid"])):
        rho, ux, uy, T = b.moments(k)
        alpha = (1.0 / w.params.lambda1 - 0.5) * w.params.cT2
        u_max, y_max, v_max, x_max = table1_quantities(ux, uy, G, alpha)
        nu = -b.nusselt(k, 1, float(G), 1.0)
        got = dict(u_max=u_max, y_max=y_max, v_max=v_max, x_max=x_max, Nu=nu)
        print(f"Ra={t1['Ra'][k]:g} G={G} steps={conv[k]}", {n: round(float(v), 4) for n, v in got.items()})
        for name in ("u_max", "v_max", "Nu"):
            assert got[name] == pytest.approx(t1[name][k], rel=0.01), (name, k)
        for name in ("y_max", "x_max"):
            assert got[name] == pytest.approx(t1[name][k], abs=0.01), (name, k)
    b.close()
