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


def test_noalloc_large_fields_against_numpy():
    """n = 1024 x 512 > 1024 blocks x 256 threads: the grid is clamped to the
    scratch's 1024 blocks, every thread loops over several nodes and the final
    pass adds all 1024 partial rows.  Random fields with a random solid mask,
    checked against the definition evaluated in FP64 with numpy, twice in a
    row (the second call reads only what it wrote itself)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    nx, ny = 1024, 512
    n = nx * ny
    for call in range(2):
        r = I.splitmix64_uniform(90210 + call, 7 * n).reshape(7, n)
        now = [0.5 + 0.3 * (2 * r[0] - 1), 0.02 * (2 * r[1] - 1), 0.02 * (2 * r[2] - 1)]
        prev = [now[k] + 1e-4 * (2 * r[3 + k] - 1) for k in range(3)]
        solid = (r[6] < 0.2).astype(np.uint8)
        fluid = solid == 0
        want = max(np.linalg.norm((a - b)[fluid]) / np.linalg.norm(a[fluid]) for a, b in zip(now, prev))
        d = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in now + prev]
        got = clbm.clbm_residual_fields_noalloc(*d, torch.from_numpy(solid).to(dev), n)
        assert got == pytest.approx(want, rel=REL_TOL), (call, got, want)


def test_noalloc_reports_nonfinite_values():
    """A NaN in the current temperature: CLBM_EUNSTABLE (the binding raises)."""
    torch = pytest.importorskip("torch")
    n = 5000
    a = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    b = a.clone()
    b[1234] = float("nan")
    with pytest.raises(clbm.ClbmError) as ei:
        clbm.clbm_residual_fields_noalloc(b, a, a, a, a, a, None, n)
    assert ei.value.status == clbm.CLBM_EUNSTABLE


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    for n in (0, -5, (1 << 31) + 1):
        with pytest.raises(clbm.ClbmError) as ei:
            clbm.clbm_residual_fields_noalloc(a, a, a, a, a, a, None, n)
        assert ei.value.status == clbm.CLBM_EINVAL
