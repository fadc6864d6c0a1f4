"""ctypes binding of the surrogate-network entry points of libclbm.so
(clbm_net_*, declared in include/clbm.h).  Argument marshalling only: the
forward pass, the backward pass and the optimizer run in the library's CUDA
kernels.  Device tensors are torch CUDA float32 tensors."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import clbm as _clbm


class clbm_net_config(C.Structure):
    _fields_ = [("grid", C.c_int32), ("in_ch", C.c_int32), ("out_ch", C.c_int32),
                ("base", C.c_int32), ("levels", C.c_int32), ("max_batch", C.c_int32),
                ("math", C.c_int32)]


MATH = {"tensor": 0, "fp32": 1}  # CLBM_NET_TENSOR, CLBM_NET_FP32


NET_EXPORTS = ["clbm_net_create", "clbm_net_param_count", "clbm_net_get_params",
               "clbm_net_set_params", "clbm_net_forward", "clbm_net_gradients",
               "clbm_net_train_step", "clbm_net_destroy", "clbm_net_last_error"]

_done = False


def load():
    global _done
    L = _clbm.load()
    if not _done:
        vp, fp, dp = C.c_void_p, C.c_void_p, C.POINTER(C.c_double)
        L.clbm_net_create.argtypes = [C.POINTER(clbm_net_config), C.c_uint64, vp, C.POINTER(vp)]
        L.clbm_net_param_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.clbm_net_get_params.argtypes = [vp, fp, C.c_int32]
        L.clbm_net_set_params.argtypes = [vp, fp, C.c_int32]
        L.clbm_net_forward.argtypes = [vp, fp, C.c_int32, fp]
        L.clbm_net_gradients.argtypes = [vp, fp, fp, fp, C.c_int32, fp, dp]
        L.clbm_net_train_step.argtypes = [vp, fp, fp, fp, C.c_int32, C.c_float, dp]
        L.clbm_net_destroy.argtypes = [vp]
        L.clbm_net_last_error.argtypes = [vp]
        L.clbm_net_last_error.restype = C.c_char_p
        for n in NET_EXPORTS[:-1]:
            getattr(L, n).restype = C.c_int
        _done = True
    return L


def _check(st, net, what):
    if st != 0:
        L = load()
        msg = L.clbm_status_string(st).decode()
        if net is not None and net.value:
            d = L.clbm_net_last_error(net).decode()
            if d:
                msg += ": " + d
        raise _clbm.ClbmError(st, f"{what}: {msg}")


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _check_dev(t, shape, name):
    """A device tensor the library reads or writes in full: refuse a wrong shape,
    dtype or layout here rather than let a kernel run past its end.  Raw
    addresses (int) are the caller's responsibility."""
    if t is None or isinstance(t, int):
        return
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if str(getattr(t, "dtype", "")) != "torch.float32" or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{name}: a contiguous float32 CUDA tensor is expected")


class Net:
    """U-Net surrogate; see clbm_net_create for the architecture."""

    def __init__(self, grid: int, in_ch: int, out_ch: int, base: int, levels: int, max_batch: int,
                 seed: int = 1, stream: Optional[int] = None, math: str = "tensor"):
        self.math = math
        self.cfg = clbm_net_config(grid, in_ch, out_ch, base, levels, max_batch, MATH[math])
        self.h = C.c_void_p()
        _check(load().clbm_net_create(C.byref(self.cfg), seed, stream, C.byref(self.h)), None,
               "clbm_net_create")
        n = C.c_int64()
        _check(load().clbm_net_param_count(self.h, C.byref(n)), self.h, "clbm_net_param_count")
        self.nparam = n.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().clbm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        _check(load().clbm_net_get_params(self.h, out.ctypes.data, 0), self.h, "get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32).ravel()
        if p.size != self.nparam:
            raise ValueError(f"{p.size} parameters for a network of {self.nparam}")
        _check(load().clbm_net_set_params(self.h, p.ctypes.data, 0), self.h, "set_params")

    def _check_batch(self, x, target=None, mask=None, y=None):
        G, N = self.cfg.grid, int(x.shape[0])
        _check_dev(x, (N, self.cfg.in_ch, G, G), "x")
        _check_dev(target, (N, self.cfg.out_ch, G, G), "target")
        _check_dev(y, (N, self.cfg.out_ch, G, G), "y")
        _check_dev(mask, (N, G, G), "mask")

    def forward(self, x, y):
        """x, y: torch CUDA float32 tensors [N, C, G, G] (async on the net's stream)."""
        self._check_batch(x, y=y)
        _check(load().clbm_net_forward(self.h, _ptr(x), int(x.shape[0]), _ptr(y)), self.h, "forward")

    def gradients(self, x, target, mask=None):
        self._check_batch(x, target, mask)
        g = np.empty(self.nparam, np.float32)
        loss = C.c_double()
        _check(load().clbm_net_gradients(self.h, _ptr(x), _ptr(target), _ptr(mask), int(x.shape[0]),
                                         g.ctypes.data, C.byref(loss)), self.h, "gradients")
        return loss.value, g

    def train_step(self, x, target, mask, lr: float) -> float:
        self._check_batch(x, target, mask)
        loss = C.c_double()
        _check(load().clbm_net_train_step(self.h, _ptr(x), _ptr(target), _ptr(mask), int(x.shape[0]),
                                          float(lr), C.byref(loss)), self.h, "train_step")
        return loss.value


def layer_shapes(grid: int, in_ch: int, out_ch: int, base: int, levels: int):
    """(ci, co, k) of every convolution in parameter order (weights then bias each)."""
    L, B = levels, base
    out = []
    for l in range(L - 1):
        out.append((in_ch if l == 0 else B << (l - 1), B << l, 3))
        out.append((B << l, B << l, 3))
    out.append((B << (L - 2), B << (L - 1), 3))
    out.append((B << (L - 1), B << (L - 1), 3))
    for l in range(L - 2, -1, -1):
        out.append(((B << (l + 1)) + (B << l), B << l, 3))
        out.append((B << l, B << l, 3))
    out.append((B, out_ch, 1))
    return out


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and back to float32."""
    a = np.ascontiguousarray(a, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def weights_as_used(params: np.ndarray, shapes) -> np.ndarray:
    """The parameter vector as the kernels see it: weights rounded to BF16, biases FP32."""
    out = params.astype(np.float32).copy()
    off = 0
    for ci, co, k in shapes:
        nw = co * ci * k * k
        out[off:off + nw] = bf16_round(out[off:off + nw])
        off += nw + co
    return out
