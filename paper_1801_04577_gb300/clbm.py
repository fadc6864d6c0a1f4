"""Thin ctypes binding of libclbm.so (declared in include/clbm.h).

The functions below carry the C names and only marshal arguments: every step
of the method runs in the library's CUDA kernels.  There is no CPU fallback;
if the library cannot be loaded, or no CUDA device is present, the calls raise.

Device buffers may be passed as ``torch.Tensor`` (float64, contiguous, on the
context's device) or as raw integer addresses; host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

CLBM_OK, CLBM_EINVAL, CLBM_ENOMEM, CLBM_ECUDA, CLBM_EUNSTABLE, CLBM_ETIMEOUT, CLBM_ENOTCONV = range(7)
CLBM_F64, CLBM_F32, CLBM_F16DEV, CLBM_BF16DEV = range(4)
PRECISIONS = {"f64": CLBM_F64, "f32": CLBM_F32, "f16": CLBM_F16DEV, "bf16": CLBM_BF16DEV}


class clbm_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32), ("precision", C.c_int32), ("rounding", C.c_int32),
                ("s_nu", C.c_double), ("s_b", C.c_double), ("s_3", C.c_double), ("s_4", C.c_double),
                ("lambda0", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("rho0", C.c_double), ("T0", C.c_double), ("gbeta", C.c_double),
                ("Fvx", C.c_double), ("Fvy", C.c_double), ("Q", C.c_double), ("cT2", C.c_double),
                ("viscous_heating", C.c_int32), ("reserved1", C.c_int32)]


class clbm_tbc(C.Structure):
    _fields_ = [("b1", C.c_double), ("b2", C.c_double), ("b3", C.c_double)]


class clbm_link(C.Structure):
    _fields_ = [("node", C.c_int32), ("dir", C.c_int32), ("n_dot_e", C.c_double),
                ("tbc", C.c_int32), ("reserved", C.c_int32), ("q", C.c_double)]


class clbm_batch_item(C.Structure):
    _fields_ = [("params", clbm_params), ("solid", C.c_void_p), ("tbc", C.POINTER(clbm_tbc)),
                ("n_tbc", C.c_int32), ("side_tbc", C.c_int32 * 4), ("n_links", C.c_int32),
                ("links", C.POINTER(clbm_link)), ("rho", C.c_void_p), ("ux", C.c_void_p),
                ("uy", C.c_void_p), ("T", C.c_void_p)]


EXPORTS = ["clbm_create", "clbm_set_boundaries", "clbm_init_fields", "clbm_step", "clbm_moments",
           "clbm_nusselt", "clbm_residual", "clbm_totals", "clbm_residual_fields_noalloc", "clbm_batch_create",
           "clbm_batch_solve", "clbm_batch_lattice", "clbm_batch_tile_width", "clbm_batch_destroy",
           "clbm_damp_period2", "clbm_batch_damp_period2",
           "clbm_set_wall_velocity", "clbm_create_slab", "clbm_halo_bytes", "clbm_halo_pack", "clbm_halo_unpack", "clbm_halo_copy",
           "clbm_slabs_exchange", "clbm_slabs_step", "clbm_reduce_sums", "clbm_finish_sums",
           "clbm_batch_last_error", "clbm_time", "clbm_field_shape", "clbm_destroy", "clbm_last_error",
           "clbm_status_string"]

_lib = None


class ClbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libclbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.clbm_create.argtypes = [C.POINTER(clbm_params), vp, C.POINTER(vp)]
    L.clbm_set_boundaries.argtypes = [vp, vp, C.POINTER(clbm_tbc), C.c_int32, C.POINTER(C.c_int32),
                                      C.POINTER(clbm_link), C.c_int32]
    L.clbm_init_fields.argtypes = [vp, vp, vp, vp, vp, C.c_int32]
    L.clbm_step.argtypes = [vp, C.c_int64]
    L.clbm_moments.argtypes = [vp, vp, vp, vp, vp, C.c_int32]
    L.clbm_nusselt.argtypes = [vp, C.c_int32, C.c_double, C.c_double, dp]
    L.clbm_residual.argtypes = [vp, dp]
    L.clbm_totals.argtypes = [vp, dp]
    L.clbm_residual_fields_noalloc.argtypes = [vp] * 7 + [C.c_int64, vp, dp]
    L.clbm_time.argtypes = [vp, C.POINTER(C.c_int64)]
    L.clbm_field_shape.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.clbm_destroy.argtypes = [vp]
    L.clbm_last_error.argtypes = [vp]
    L.clbm_last_error.restype = C.c_char_p
    L.clbm_status_string.argtypes = [C.c_int]
    L.clbm_status_string.restype = C.c_char_p
    L.clbm_batch_create.argtypes = [C.POINTER(clbm_batch_item), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
    L.clbm_batch_solve.argtypes = [vp, C.c_double, C.c_int64, C.c_int32, C.POINTER(C.c_int64), dp,
                                   C.POINTER(C.c_int64)]
    L.clbm_batch_lattice.argtypes = [vp, C.c_int32, C.POINTER(vp)]
    L.clbm_batch_tile_width.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    L.clbm_batch_destroy.argtypes = [vp]
    L.clbm_damp_period2.argtypes = [vp]
    L.clbm_batch_damp_period2.argtypes = [vp]
    L.clbm_set_wall_velocity.argtypes = [vp, C.c_int32, C.c_double, C.c_double]
    L.clbm_create_slab.argtypes = [C.POINTER(clbm_params), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
    L.clbm_halo_bytes.argtypes = [vp, C.POINTER(C.c_int64)]
    L.clbm_halo_pack.argtypes = [vp, C.c_int32, vp]
    L.clbm_halo_unpack.argtypes = [vp, C.c_int32, vp]
    L.clbm_halo_copy.argtypes = [vp, C.c_int32, vp]
    L.clbm_slabs_exchange.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32]
    L.clbm_slabs_step.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32, C.c_int64]
    L.clbm_reduce_sums.argtypes = [vp, C.c_int32, C.c_int32, dp]
    L.clbm_finish_sums.argtypes = [vp, C.c_int32, dp, C.c_double, C.c_double, dp]
    L.clbm_batch_last_error.argtypes = [vp]
    L.clbm_batch_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("clbm_last_error", "clbm_status_string", "clbm_batch_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st: int, ctx=None, what: str = ""):
    if st != CLBM_OK:
        L = load()
        msg = L.clbm_status_string(st).decode()
        if ctx is not None:
            detail = L.clbm_last_error(ctx).decode()
            if detail:
                msg += ": " + detail
        raise ClbmError(st, f"{what}: {msg}" if what else msg)


def _addr(a) -> Optional[int]:
    """Address of a torch tensor, numpy array or raw pointer (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def make_params(p, precision="f32", rounding: int = 0) -> clbm_params:
    """rounding: 0 = nearest even, 1 = stochastic (16-bit storage only)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return clbm_params(p.nx, p.ny, p.periodic_x, p.periodic_y, prec, int(rounding), p.s_nu, p.s_b, p.s_3,
                       p.s_4, p.lambda0, p.lambda1, p.lambda2, p.rho0, p.T0, p.gbeta, p.Fvx,
                       p.Fvy, p.Q, p.cT2, int(getattr(p, "viscous_heating", 0)), 0)


# --------------------------------------------------------------------------
# The C entry points, one Python function each
# --------------------------------------------------------------------------
def clbm_create(params: clbm_params, stream: Optional[int] = None) -> C.c_void_p:
    L = load()
    ctx = C.c_void_p()
    _check(L.clbm_create(C.byref(params), stream, C.byref(ctx)), None, "clbm_create")
    return ctx


def clbm_set_boundaries(ctx, solid: Optional[np.ndarray], tbc: Sequence, side_tbc: Sequence[int],
                        link_node=None, link_dir=None, link_ne=None, link_tbc=None, link_q=None):
    L = load()
    n_tbc = len(tbc)
    tarr = (clbm_tbc * max(n_tbc, 1))(*[clbm_tbc(*map(float, t)) for t in tbc])
    sides = (C.c_int32 * 4)(*[int(s) for s in side_tbc])
    n_links = 0 if link_node is None else int(len(link_node))
    larr = (clbm_link * max(n_links, 1))()
    for k in range(n_links):
        larr[k] = clbm_link(int(link_node[k]), int(link_dir[k]), float(link_ne[k]), int(link_tbc[k]), 0,
                            0.5 if link_q is None else float(link_q[k]))
    sol = None
    if solid is not None:  # a raw host address passes through; arrays become uint8
        sol = solid if isinstance(solid, int) else np.ascontiguousarray(solid, dtype=np.uint8)
    _check(L.clbm_set_boundaries(ctx, _addr(sol), tarr, n_tbc, sides, larr, n_links), ctx,
           "clbm_set_boundaries")


def _host_f64(b):
    """A host field for the library: a raw address (int) or a contiguous FP64
    CPU tensor passes through as it is; anything else becomes a contiguous
    FP64 numpy array."""
    if b is None or isinstance(b, int):
        return b
    if hasattr(b, "data_ptr"):
        if getattr(b, "is_cuda", False):
            raise ValueError("device tensor passed as a host field (use on_device=True)")
        if str(b.dtype) != "torch.float64" or not b.is_contiguous():
            raise ValueError("host tensors must be contiguous float64")
        return b
    return np.ascontiguousarray(b, dtype=np.float64)


def clbm_field_shape(ctx):
    """(nx, rows) of the fields of a context: each field holds nx * rows doubles."""
    nx, rows = C.c_int64(), C.c_int64()
    _check(load().clbm_field_shape(ctx, C.byref(nx), C.byref(rows)), ctx, "clbm_field_shape")
    return nx.value, rows.value


def _check_fields(ctx, bufs, on_device, what):
    """Every field array (not a raw address) must hold nx * rows FP64 values on
    the side `on_device` names: the library reads or writes all of them."""
    if all(b is None or isinstance(b, int) for b in bufs):
        return
    nx, rows = clbm_field_shape(ctx)
    for b in bufs:
        if b is None or isinstance(b, int):
            continue
        if hasattr(b, "data_ptr"):
            ok = (b.numel() == nx * rows and str(b.dtype) == "torch.float64" and b.is_contiguous()
                  and bool(b.is_cuda) == bool(on_device))
        else:
            ok = (not on_device and isinstance(b, np.ndarray) and b.size == nx * rows
                  and b.dtype == np.float64 and b.flags["C_CONTIGUOUS"])
        if not ok:
            raise ValueError(f"{what}: each field must be {rows} x {nx} contiguous float64 "
                             f"{'device' if on_device else 'host'} values")


def clbm_init_fields(ctx, rho=None, ux=None, uy=None, T=None, on_device: bool = False):
    L = load()
    bufs = [rho, ux, uy, T]
    if not on_device:
        bufs = [_host_f64(b) for b in bufs]
    _check_fields(ctx, bufs, on_device, "clbm_init_fields")
    _check(L.clbm_init_fields(ctx, *[_addr(b) for b in bufs], int(on_device)), ctx,
           "clbm_init_fields")


def clbm_step(ctx, nsteps: int):
    _check(load().clbm_step(ctx, int(nsteps)), ctx, "clbm_step")


def clbm_moments(ctx, rho=None, ux=None, uy=None, T=None, on_device: bool = False):
    _check_fields(ctx, (rho, ux, uy, T), on_device, "clbm_moments")
    _check(load().clbm_moments(ctx, *[_addr(b) for b in (rho, ux, uy, T)], int(on_device)), ctx,
           "clbm_moments")


def clbm_nusselt(ctx, which: int, length: float, dT: float) -> float:
    out = C.c_double()
    _check(load().clbm_nusselt(ctx, int(which), float(length), float(dT), C.byref(out)), ctx,
           "clbm_nusselt")
    return out.value


def clbm_residual(ctx) -> float:
    out = C.c_double()
    _check(load().clbm_residual(ctx, C.byref(out)), ctx, "clbm_residual")
    return out.value


def clbm_totals(ctx) -> np.ndarray:
    """(sum f_i, sum f_i e_ix, sum f_i e_iy, sum g_j) over the fluid nodes, FP64."""
    out = np.zeros(4, np.float64)
    _check(load().clbm_totals(ctx, out.ctypes.data_as(C.POINTER(C.c_double))), ctx, "clbm_totals")
    return out


def clbm_residual_fields_noalloc(T_now, ux_now, uy_now, T_prev, ux_prev, uy_prev, solid, n: int,
                                 stream: Optional[int] = None) -> float:
    """Residual from caller-owned device fields, without device allocation."""
    out = C.c_double()
    args = [_addr(b) for b in (T_now, ux_now, uy_now, T_prev, ux_prev, uy_prev, solid)]
    _check(load().clbm_residual_fields_noalloc(*args, int(n), stream, C.byref(out)), None,
           "clbm_residual_fields_noalloc")
    return out.value


def clbm_set_wall_velocity(ctx, side: int, ux: float, uy: float = 0.0):
    _check(load().clbm_set_wall_velocity(ctx, int(side), float(ux), float(uy)), ctx, "clbm_set_wall_velocity")


def _apply_side_velocities(ctx, geom):
    for side, (ux, uy) in enumerate(getattr(geom, "side_u", None) or ()):
        if ux or uy:
            clbm_set_wall_velocity(ctx, side, ux, uy)


def clbm_create_slab(params: clbm_params, y0: int, rows: int, stream: Optional[int] = None) -> C.c_void_p:
    L = load()
    ctx = C.c_void_p()
    _check(L.clbm_create_slab(C.byref(params), int(y0), int(rows), stream, C.byref(ctx)), None,
           "clbm_create_slab")
    return ctx


def clbm_halo_bytes(ctx) -> int:
    out = C.c_int64()
    _check(load().clbm_halo_bytes(ctx, C.byref(out)), ctx, "clbm_halo_bytes")
    return out.value


def _check_halo_buffer(ctx, buf, what):
    """A device tensor given as a halo buffer must hold clbm_halo_bytes bytes
    (the library writes or reads all of them); raw addresses pass unchecked."""
    if isinstance(buf, int) or not hasattr(buf, "data_ptr"):
        return
    have = buf.numel() * buf.element_size()
    need = clbm_halo_bytes(ctx)
    if have < need or not buf.is_contiguous() or not buf.is_cuda:
        raise ValueError(f"{what}: a contiguous CUDA buffer of {need} bytes is needed, got {have}")


def clbm_halo_pack(ctx, side: int, dst):
    _check_halo_buffer(ctx, dst, "clbm_halo_pack")
    _check(load().clbm_halo_pack(ctx, int(side), _addr(dst)), ctx, "clbm_halo_pack")


def clbm_halo_unpack(ctx, side: int, src):
    _check_halo_buffer(ctx, src, "clbm_halo_unpack")
    _check(load().clbm_halo_unpack(ctx, int(side), _addr(src)), ctx, "clbm_halo_unpack")


def clbm_halo_copy(src_ctx, side: int, dst_ctx):
    _check(load().clbm_halo_copy(src_ctx, int(side), dst_ctx), dst_ctx, "clbm_halo_copy")


def _ctx_array(ctxs):
    return (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])


def clbm_slabs_exchange(ctxs, periodic: bool):
    _check(load().clbm_slabs_exchange(_ctx_array(ctxs), len(ctxs), int(periodic)), None,
           "clbm_slabs_exchange")


def clbm_slabs_step(ctxs, periodic: bool, nsteps: int):
    _check(load().clbm_slabs_step(_ctx_array(ctxs), len(ctxs), int(periodic), int(nsteps)), None,
           "clbm_slabs_step")


REDUCE_RESIDUAL, REDUCE_NUSSELT, REDUCE_TOTALS = 0, 1, 2


def clbm_reduce_sums(ctx, what: int, which: int = 0) -> np.ndarray:
    out = np.zeros(8, np.float64)
    _check(load().clbm_reduce_sums(ctx, int(what), int(which), out.ctypes.data_as(C.POINTER(C.c_double))),
           ctx, "clbm_reduce_sums")
    return out


def clbm_finish_sums(ctx, what: int, sums, length: float = 0.0, dT: float = 1.0) -> np.ndarray:
    h = np.ascontiguousarray(sums, np.float64).ravel()
    if h.size < 8:
        raise ValueError("clbm_finish_sums takes the eight sums of clbm_reduce_sums")
    out = np.zeros(4, np.float64)
    _check(load().clbm_finish_sums(ctx, int(what), h.ctypes.data_as(C.POINTER(C.c_double)), float(length),
                                   float(dT), out.ctypes.data_as(C.POINTER(C.c_double))), None,
           "clbm_finish_sums")
    return out


def clbm_damp_period2(ctx):
    _check(load().clbm_damp_period2(ctx), ctx, "clbm_damp_period2")


def clbm_time(ctx) -> int:
    out = C.c_int64()
    _check(load().clbm_time(ctx, C.byref(out)), ctx, "clbm_time")
    return out.value


def clbm_destroy(ctx):
    if ctx is not None and ctx.value:
        load().clbm_destroy(ctx)


def clbm_last_error(ctx) -> str:
    return load().clbm_last_error(ctx).decode()


# --------------------------------------------------------------------------
# Convenience wrapper around one context
# --------------------------------------------------------------------------
def _check_solid_shape(geom, params):
    """The library copies ny * nx mask bytes: a mask of any other shape is refused here."""
    solid = None if geom is None else geom.solid
    if solid is not None and np.shape(solid) != (params.ny, params.nx):
        raise ValueError(f"solid mask of shape {np.shape(solid)} for a {params.ny} x {params.nx} lattice")


class Solver:
    """One lattice on the GPU, described by ``inputs.Params`` / ``inputs.Geometry``."""

    def __init__(self, params, geom=None, precision="f32", stream: Optional[int] = None, init=None,
                 rounding: int = 0):
        _check_solid_shape(geom, params)
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.precision = precision
        self.ctx = clbm_create(make_params(params, precision, rounding), stream)
        if geom is not None:
            clbm_set_boundaries(self.ctx, geom.solid, geom.tbc, geom.side_tbc, geom.link_node,
                                geom.link_dir, geom.link_ne, geom.link_tbc, geom.link_q_or_half())
            _apply_side_velocities(self.ctx, geom)
        if init is not None:
            self.init(init)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            clbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, fields=None):
        shape = (self.ny, self.nx)
        if fields is None:
            clbm_init_fields(self.ctx)
            return
        arrs = []
        for a in (fields.rho, fields.ux, fields.uy, fields.T):
            arrs.append(None if a is None else np.ascontiguousarray(np.broadcast_to(a, shape), np.float64))
        clbm_init_fields(self.ctx, *arrs)

    def step(self, n: int = 1):
        clbm_step(self.ctx, n)

    def moments(self):
        shape = (self.ny, self.nx)
        out = [np.empty(shape) for _ in range(4)]
        clbm_moments(self.ctx, *out)
        return tuple(out)

    def nusselt(self, which: int, length: float, dT: float) -> float:
        return clbm_nusselt(self.ctx, which, length, dT)

    def residual(self) -> float:
        return clbm_residual(self.ctx)

    def totals(self) -> np.ndarray:
        return clbm_totals(self.ctx)

    @property
    def time(self) -> int:
        return clbm_time(self.ctx)


class Slab(Solver):
    """Rows [y0, y0 + rows) of the lattice ``params`` describes, with a ghost
    row on each side (``clbm_create_slab``); walls and initial fields are given
    for the whole lattice and cut here."""

    def __init__(self, params, y0: int, rows: int, geom=None, precision="f32",
                 stream: Optional[int] = None, init=None, rounding: int = 0):
        self.params = params
        self.nx, self.ny = params.nx, rows
        self.y0, self.rows = y0, rows
        self.precision = precision
        _check_solid_shape(geom, params)
        self.ctx = clbm_create_slab(make_params(params, precision, rounding), y0, rows, stream)
        if geom is not None:
            clbm_set_boundaries(self.ctx, geom.solid, geom.tbc, geom.side_tbc, geom.link_node,
                                geom.link_dir, geom.link_ne, geom.link_tbc, geom.link_q_or_half())
            _apply_side_velocities(self.ctx, geom)
        if init is not None:
            self.init(init)

    def init(self, fields=None):
        if fields is None:
            clbm_init_fields(self.ctx)
            return
        full = (self.params.ny, self.nx)
        arrs = []
        for a in (fields.rho, fields.ux, fields.uy, fields.T):
            arrs.append(None if a is None else
                        np.ascontiguousarray(np.broadcast_to(a, full)[self.y0:self.y0 + self.rows], np.float64))
        clbm_init_fields(self.ctx, *arrs)

    def sums(self, what: int, which: int = 0) -> np.ndarray:
        return clbm_reduce_sums(self.ctx, what, which)


def from_workload(w, precision="f32", stream=None, rounding: int = 0) -> Solver:
    return Solver(w.params, w.geom, precision, stream, w.init, rounding)


# --------------------------------------------------------------------------
# Batched solves
# --------------------------------------------------------------------------
def _batch_check(st, b, what):
    if st != CLBM_OK:
        L = load()
        msg = L.clbm_status_string(st).decode()
        if b is not None and b.value:
            detail = L.clbm_batch_last_error(b).decode()
            if detail:
                msg += ": " + detail
        raise ClbmError(st, f"{what}: {msg}")


def clbm_batch_create(items, autotune: bool = True, stream: Optional[int] = None) -> C.c_void_p:
    arr = (clbm_batch_item * len(items))(*items)
    b = C.c_void_p()
    _batch_check(load().clbm_batch_create(arr, len(items), int(autotune), stream, C.byref(b)), None,
                 "clbm_batch_create")
    return b


def clbm_batch_solve(b, n: int, tol: float, max_steps: int, check_every: int = 100):
    conv = (C.c_int64 * n)()
    res = (C.c_double * n)()
    steps = C.c_int64()
    _batch_check(load().clbm_batch_solve(b, float(tol), int(max_steps), int(check_every), conv,
                                         res, C.byref(steps)), b, "clbm_batch_solve")
    return np.array(conv[:], dtype=np.int64), np.array(res[:]), steps.value


def clbm_batch_lattice(b, i: int) -> C.c_void_p:
    v = C.c_void_p()
    _batch_check(load().clbm_batch_lattice(b, int(i), C.byref(v)), b, "clbm_batch_lattice")
    return v


def clbm_batch_tile_width(b, i: int) -> int:
    w = C.c_int32()
    _batch_check(load().clbm_batch_tile_width(b, int(i), C.byref(w)), b, "clbm_batch_tile_width")
    return w.value


def clbm_batch_destroy(b):
    if b is not None and b.value:
        load().clbm_batch_destroy(b)


class Batch:
    """Many independent lattices (``inputs.Workload`` list) solved together."""

    def __init__(self, workloads, precision="f32", rounding: int = 0, autotune: bool = True,
                 stream: Optional[int] = None):
        self.workloads = list(workloads)
        keep = []
        items = []
        for w in self.workloads:
            p, g = w.params, w.geom
            if any(ux or uy for ux, uy in (getattr(g, "side_u", None) or ())):
                raise ValueError(f"{w.name}: batched lattices have walls at rest")
            shape = (p.ny, p.nx)
            _check_solid_shape(g, p)
            tbc = (clbm_tbc * max(len(g.tbc), 1))(*[clbm_tbc(*map(float, t)) for t in g.tbc])
            nl = g.n_links
            links = (clbm_link * max(nl, 1))()
            lq = g.link_q_or_half()
            for k in range(nl):
                links[k] = clbm_link(int(g.link_node[k]), int(g.link_dir[k]), float(g.link_ne[k]),
                                     int(g.link_tbc[k]), 0, float(lq[k]))
            solid = None if g.solid is None else np.ascontiguousarray(g.solid, np.uint8)
            fields = []
            for a in (w.init.rho, w.init.ux, w.init.uy, w.init.T):
                fields.append(None if a is None else
                              np.ascontiguousarray(np.broadcast_to(a, shape), np.float64))
            keep.append((tbc, links, solid, fields))
            it = clbm_batch_item()
            it.params = make_params(p, precision, rounding)
            it.solid = None if solid is None else solid.ctypes.data
            it.tbc = tbc
            it.n_tbc = len(g.tbc)
            it.side_tbc = (C.c_int32 * 4)(*[int(v) for v in g.side_tbc])
            it.n_links = nl
            it.links = links
            it.rho, it.ux, it.uy, it.T = [None if a is None else a.ctypes.data for a in fields]
            items.append(it)
        self.b = clbm_batch_create(items, autotune, stream)
        del keep

    def __len__(self):
        return len(self.workloads)

    def solve(self, tol: float, max_steps: int, check_every: int = 100):
        return clbm_batch_solve(self.b, len(self), tol, max_steps, check_every)

    def damp_period2(self):
        _batch_check(load().clbm_batch_damp_period2(self.b), self.b, "clbm_batch_damp_period2")

    def view(self, i: int) -> C.c_void_p:
        return clbm_batch_lattice(self.b, i)

    def moments(self, i: int):
        w = self.workloads[i]
        shape = (w.params.ny, w.params.nx)
        out = [np.empty(shape) for _ in range(4)]
        clbm_moments(self.view(i), *out)
        return tuple(out)

    def nusselt(self, i: int, which: int, length: float, dT: float) -> float:
        return clbm_nusselt(self.view(i), which, length, dT)

    def tile_width(self, i: int) -> int:
        return clbm_batch_tile_width(self.b, i)

    def close(self):
        if getattr(self, "b", None) is not None:
            clbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
