"""CPU checks of the C ABI library: it builds for sm_103a, loads, exports every
entry point declared in include/clbm.h, and rejects invalid descriptions
before touching the GPU (no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

from paper_1801_04577_gb300 import build, clbm, net
from paper_1801_04577_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "clbm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|clbm_status)\s+(clbm_\w+)\s*\(", src, re.M)))


def test_library_builds_and_exports_all_declared_symbols():
    path = build.build()
    assert os.path.exists(path)
    lib = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(clbm.EXPORTS) | set(net.NET_EXPORTS)


def test_net_create_rejects_bad_config():
    L = net.load()
    import ctypes as C
    h = C.c_void_p()
    for cfg in [(30, 5, 3, 8, 3, 4),   # grid not divisible by 2^(levels-1)
                (32, 5, 3, 8, 1, 4),   # too few levels
                (32, 0, 3, 8, 3, 4),   # no input channels
                (32, 5, 3, 8, 3, 4, 7)]:  # unknown convolution arithmetic
        c = net.clbm_net_config(*cfg)
        assert L.clbm_net_create(C.byref(c), 1, None, C.byref(h)) == clbm.CLBM_EINVAL


def test_status_strings():
    L = clbm.load()
    assert L.clbm_status_string(0) == b"CLBM_OK"
    assert L.clbm_status_string(4) == b"CLBM_EUNSTABLE"


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -3), ("s_nu", 2.5), ("lambda1", 0.0),
                                         ("rho0", -1.0), ("cT2", 0.7), ("precision", 9)])
def test_create_rejects_invalid_params(field, value):
    p = clbm.make_params(I.natural_convection_cavity(16).params, "f32")
    setattr(p, field, value)
    L = clbm.load()
    ctx = C.c_void_p()
    st = L.clbm_create(C.byref(p), None, C.byref(ctx))
    assert st == clbm.CLBM_EINVAL
    assert not ctx.value


def test_null_arguments():
    L = clbm.load()
    assert L.clbm_create(None, None, None) == clbm.CLBM_EINVAL
    assert L.clbm_destroy(None) == clbm.CLBM_OK
    assert L.clbm_step(None, 1) == clbm.CLBM_EINVAL
    assert L.clbm_last_error(None) == b""
    out = (C.c_double * 4)()
    assert L.clbm_totals(None, out) == clbm.CLBM_EINVAL
    assert L.clbm_residual(None, out) == clbm.CLBM_EINVAL
    assert L.clbm_nusselt(None, 0, 1.0, 1.0, out) == clbm.CLBM_EINVAL


def test_host_field_addresses_pass_through_unchanged(monkeypatch):
    """clbm_init_fields with host fields: a raw address (int) and a contiguous
    FP64 CPU tensor reach the library as the caller's own address; only
    array-likes are converted.  (A raw address once became the address of a
    one-element array, and the library copied nx * ny doubles from it.)"""
    import numpy as np
    import torch

    seen = []

    class Fake:
        def clbm_init_fields(self, ctx, *args):
            seen.append(args)
            return clbm.CLBM_OK

        def clbm_field_shape(self, ctx, nx, rows):
            nx._obj.value, rows._obj.value = 4, 3
            return clbm.CLBM_OK

    monkeypatch.setattr(clbm, "load", lambda: Fake())
    t = torch.arange(12, dtype=torch.float64)
    a = np.arange(12, dtype=np.float32)
    clbm.clbm_init_fields(None, None, 0x7F00_0000_1000, t, a, on_device=False)
    rho, ux, uy, T, dev = seen[-1]
    assert rho is None and ux == 0x7F00_0000_1000 and uy == t.data_ptr() and dev == 0
    assert T not in (None, a.ctypes.data)  # converted to a new FP64 array
    with pytest.raises(ValueError):
        clbm.clbm_init_fields(None, t.float(), on_device=False)
    with pytest.raises(ValueError):
        clbm.clbm_init_fields(None, t[::2], on_device=False)
    with pytest.raises(ValueError):  # 13 values for a 3 x 4 field
        clbm.clbm_init_fields(None, np.zeros(13), on_device=False)
    with pytest.raises(ValueError):  # a host tensor where device fields are asked for
        clbm.clbm_init_fields(None, t, on_device=True)
    clbm.clbm_init_fields(None, 1234, 5678, on_device=True)
    assert seen[-1][:2] == (1234, 5678) and seen[-1][4] == 1


def test_mask_and_sums_of_the_wrong_size_are_refused_before_the_library():
    """The library copies ny * nx mask bytes and eight sums: shorter inputs are
    refused by the binding (no GPU needed: the checks come first)."""
    import numpy as np
    w = I.natural_convection_cavity(12, 1e4)
    w.geom.solid = np.zeros((11, 12), np.uint8)
    with pytest.raises(ValueError):
        clbm.Solver(w.params, w.geom)
    with pytest.raises(ValueError):
        clbm.Slab(w.params, 0, 6, w.geom)
    with pytest.raises(ValueError):
        clbm.Batch([w])
    with pytest.raises(ValueError):
        clbm.clbm_finish_sums(None, 0, np.zeros(7))
