"""The allocation-free residual entry point, through the C ABI.

clbm_residual_fields_noalloc serves callers that cannot allocate device
memory (their own pool owns all of it, or they cannot afford the
synchronisation of cudaFree): it keeps its reduction scratch in a fixed device
array of the library.  This test checks it against clbm_residual on the same
state, on two calls in a row (the second call reuses the scratch the first one
left behind), with and without a solid mask.  It allocates its own device
buffers with torch; the entry point itself allocates nothing.
"""
import numpy as np
import pytest

from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.mark.parametrize("name", ["cavity", "obstacle"])
def test_noalloc_residual_matches_clbm_residual_twice(name):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    w = I.natural_convection_cavity(48, 1e4) if name == "cavity" else I.obstacle_channel()
    ny, nx = w.params.ny, w.params.nx
    n = nx * ny
    s = clbm.from_workload(w, "f64", stream=stream.cuda_stream)
    solid = None
    if w.geom.solid is not None:
        solid = torch.from_numpy(np.ascontiguousarray(w.geom.solid, np.uint8).ravel()).to(dev)
    prev = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3)]
    now = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3)]
    s.step(50)
    for call in range(2):
        # T, ux, uy at t-1 and at t, both left on the device
        clbm.clbm_moments(s.ctx, None, prev[1], prev[2], prev[0], on_device=True)
        s.step(1)
        clbm.clbm_moments(s.ctx, None, now[1], now[2], now[0], on_device=True)
        r_ref = s.residual()  # existing entry point (synchronises the stream)
        r = clbm.clbm_residual_fields_noalloc(now[0], now[1], now[2], prev[0], prev[1], prev[2],
                                              solid, n, stream=stream.cuda_stream)
        assert r > 0
        assert r == pytest.approx(r_ref, rel=REL_TOL), (call, r, r_ref)
        s.step(25 + 10 * call)
    s.close()


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    for n in (0, -5, (1 << 31) + 1):
        with pytest.raises(clbm.ClbmError) as ei:
            clbm.clbm_residual_fields_noalloc(a, a, a, a, a, a, None, n)
        assert ei.value.status == clbm.CLBM_EINVAL
