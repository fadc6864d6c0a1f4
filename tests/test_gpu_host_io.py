"""Host fields in and out through the C ABI: a raw address of pinned host
memory, a pinned CPU tensor and a numpy array initialise the same state, and
moments written to raw pinned addresses equal those read into numpy arrays,
bit for bit (the library copies exactly nx * ny doubles per field)."""
import numpy as np
import pytest

from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_host_fields_by_address_tensor_and_array_agree(precision):
    torch = pytest.importorskip("torch")
    w = I.rayleigh_benard(70, 33, Ra=1e5, noise=1e-2)
    w.init = I.random_fields(70, 33, seed=5, amp=0.02)
    n = 70 * 33
    s = clbm.from_workload(w, precision)  # numpy arrays
    ref = s.moments()
    host = [torch.from_numpy(np.array(np.broadcast_to(a, (33, 70)), np.float64).ravel()).pin_memory()
            for a in (w.init.rho, w.init.ux, w.init.uy, w.init.T)]
    for form in ("address", "tensor"):
        args = [h.data_ptr() for h in host] if form == "address" else host
        clbm.clbm_init_fields(s.ctx, *args, on_device=False)
        got = s.moments()
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b, err_msg=form)
    s.step(25)
    want = s.moments()
    outs = [torch.full((n,), np.nan, dtype=torch.float64).pin_memory() for _ in range(4)]
    clbm.clbm_moments(s.ctx, *[o.data_ptr() for o in outs], on_device=False)
    for o, b in zip(outs, want):
        np.testing.assert_array_equal(o.numpy().reshape(33, 70), b)
