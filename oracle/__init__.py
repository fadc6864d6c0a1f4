"""FP64 CPU oracle for the cascaded thermal lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY: this package is the judge the CUDA library is checked
against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA library; both are driven by the
input descriptions in ``paper_1801_04577_gb300.inputs``.

Every function here follows a passage of the paper (see ``clbm_oracle.c``).
Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libclbm_oracle.so")
_lock = threading.Lock()
_lib = None


class OrefParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32),
                ("s_nu", C.c_double), ("s_b", C.c_double), ("s_3", C.c_double),
                ("s_4", C.c_double), ("lambda0", C.c_double), ("lambda1", C.c_double),
                ("lambda2", C.c_double), ("rho0", C.c_double), ("T0", C.c_double),
                ("gbeta", C.c_double), ("Fvx", C.c_double), ("Fvy", C.c_double),
                ("Q", C.c_double), ("cT2", C.c_double), ("viscous_heating", C.c_int32),
                ("reserved1", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        vp = C.c_void_p
        L.oref_create.argtypes = [C.POINTER(OrefParams), C.c_void_p, dp, C.c_int32, ip, ip, ip,
                                  dp, ip, dp, C.c_int32, C.POINTER(C.c_void_p)]
        L.oref_create.restype = C.c_int
        L.oref_destroy.argtypes = [vp]
        L.oref_init.argtypes = [vp, dp, dp, dp, dp]
        L.oref_step.argtypes = [vp, C.c_int64]
        L.oref_moments.argtypes = [vp, dp, dp, dp, dp]
        L.oref_get_dfs.argtypes = [vp, dp, dp]
        L.oref_set_dfs.argtypes = [vp, dp, dp]
        L.oref_nusselt.argtypes = [vp, C.c_int32, C.c_double, C.c_double, dp]
        L.oref_residual.argtypes = [vp, dp]
        L.oref_wall_temperature.argtypes = [C.c_double] * 6 + [C.c_int]
        L.oref_wall_temperature.restype = C.c_double
        L.oref_wall_temperature_q.argtypes = [C.c_double] * 7 + [C.c_int]
        L.oref_wall_temperature_q.restype = C.c_double
        L.oref_midpoint_temperature_q.argtypes = [C.c_double] * 4 + [C.c_int, C.c_double, C.c_int, C.c_int]
        L.oref_midpoint_temperature_q.restype = C.c_double
        L.oref_moment_matrix.argtypes = [dp]
        L.oref_shift_matrix.argtypes = [C.c_double, C.c_double, dp]
        L.oref_thermal_moment_matrix.argtypes = [dp]
        L.oref_thermal_shift_matrix.argtypes = [C.c_double, C.c_double, dp]
        L.oref_central_moments.argtypes = [dp, C.c_double, C.c_double, dp]
        L.oref_from_central.argtypes = [vp, dp, C.c_double, C.c_double, dp]
        L.oref_thermal_central_moments.argtypes = [dp, C.c_double, C.c_double, dp]
        L.oref_thermal_from_central.argtypes = [vp, dp, C.c_double, C.c_double, dp]
        L.oref_collide_node.argtypes = [vp, dp, dp, dp, dp, dp]
        L.oref_equilibrium.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
        L.oref_rates.argtypes = [vp, dp]
        L.oref_inverse_matrices.argtypes = [vp, dp, dp]
        L.oref_set_wall_velocity.argtypes = [vp, C.c_int32, C.c_double, C.c_double]
        L.oref_set_wall_velocity.restype = C.c_int
        L.oref_threads.restype = C.c_int
        L.oref_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = np.ascontiguousarray(np.broadcast_to(a, shape))
    return a


def make_params(p) -> OrefParams:
    return OrefParams(p.nx, p.ny, p.periodic_x, p.periodic_y, p.s_nu, p.s_b, p.s_3, p.s_4,
                      p.lambda0, p.lambda1, p.lambda2, p.rho0, p.T0, p.gbeta, p.Fvx, p.Fvy,
                      p.Q, p.cT2, int(getattr(p, "viscous_heating", 0)), 0)


class Oracle:
    """FP64 reference solver for one lattice (``inputs.Params`` + ``inputs.Geometry``)."""

    def __init__(self, params, geom, init=None):
        L = lib()
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self._p = make_params(params)
        tbc = np.ascontiguousarray(np.asarray(geom.tbc, np.float64).reshape(-1, 3))
        side = np.ascontiguousarray(np.asarray(geom.side_tbc, np.int32))
        solid = None if geom.solid is None else np.ascontiguousarray(geom.solid, np.uint8)
        ln = np.ascontiguousarray(geom.link_node, np.int32)
        ld = np.ascontiguousarray(geom.link_dir, np.int32)
        le = np.ascontiguousarray(geom.link_ne, np.float64)
        lt = np.ascontiguousarray(geom.link_tbc, np.int32)
        lq = getattr(geom, "link_q", None)
        lq = None if lq is None else np.ascontiguousarray(lq, np.float64)
        self.solid = solid
        h = C.c_void_p()
        st = L.oref_create(C.byref(self._p), None if solid is None else solid.ctypes.data,
                           _dp(tbc), tbc.shape[0], _ip(side), _ip(ln), _ip(ld), _dp(le), _ip(lt),
                           _dp(lq), ln.shape[0], C.byref(h))
        if st != 0:
            raise ValueError(f"oracle rejected the problem description (status {st})")
        self._h = h
        for side, (ux, uy) in enumerate(getattr(geom, "side_u", None) or ()):
            if ux or uy:
                self.set_wall_velocity(side, ux, uy)
        self.init(init)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oref_destroy(h)
            self._h = None

    def init(self, fields=None):
        shape = (self.ny, self.nx)
        rho = ux = uy = T = None
        if fields is not None:
            rho, ux, uy, T = (_f64(fields.rho, shape), _f64(fields.ux, shape),
                              _f64(fields.uy, shape), _f64(fields.T, shape))
        lib().oref_init(self._h, _dp(rho), _dp(ux), _dp(uy), _dp(T))
        self._keep = (rho, ux, uy, T)

    def step(self, n: int = 1):
        if lib().oref_step(self._h, int(n)) != 0:
            raise ValueError("bad step count")

    def moments(self):
        shape = (self.ny, self.nx)
        out = [np.empty(shape) for _ in range(4)]
        lib().oref_moments(self._h, *[_dp(a) for a in out])
        return tuple(out)  # rho, ux, uy, T

    def dfs(self):
        n = self.nx * self.ny
        f = np.empty((n, 9))
        g = np.empty((n, 5))
        lib().oref_get_dfs(self._h, _dp(f), _dp(g))
        return f.reshape(self.ny, self.nx, 9), g.reshape(self.ny, self.nx, 5)

    def set_dfs(self, f, g):
        f = _f64(f)
        g = _f64(g)
        lib().oref_set_dfs(self._h, _dp(f), _dp(g))

    def nusselt(self, which: int, length: float, dT: float) -> float:
        out = C.c_double()
        if lib().oref_nusselt(self._h, which, length, dT, C.byref(out)) != 0:
            raise ValueError("no wall links for this selection")
        return out.value

    def residual(self) -> float:
        out = C.c_double()
        if lib().oref_residual(self._h, C.byref(out)) != 0:
            raise ValueError("residual needs at least one step")
        return out.value

    def set_wall_velocity(self, side: int, ux: float, uy: float = 0.0):
        """Velocity of a box side for the moving-wall bounce-back (not in the paper)."""
        if lib().oref_set_wall_velocity(self._h, int(side), float(ux), float(uy)) != 0:
            raise ValueError("bad side")

    def collide_node(self, f, g):
        f = _f64(f)
        g = _f64(g)
        fs = np.empty(9)
        gs = np.empty(5)
        mac = np.empty(4)
        lib().oref_collide_node(self._h, _dp(f), _dp(g), _dp(fs), _dp(gs), _dp(mac))
        return fs, gs, mac

    def equilibrium(self, rho, ux, uy, T):
        f = np.empty(9)
        g = np.empty(5)
        lib().oref_equilibrium(self._h, rho, ux, uy, T, _dp(f), _dp(g))
        return f, g

    def from_central(self, kt, ux, uy):
        kt = _f64(kt)
        f = np.empty(9)
        lib().oref_from_central(self._h, _dp(kt), ux, uy, _dp(f))
        return f

    def thermal_from_central(self, kt, ux, uy):
        kt = _f64(kt)
        g = np.empty(5)
        lib().oref_thermal_from_central(self._h, _dp(kt), ux, uy, _dp(g))
        return g

    def rates(self):
        out = np.empty(2)
        lib().oref_rates(self._h, _dp(out))
        return float(out[0]), float(out[1])  # s3, lambda2

    def inverse_matrices(self):
        a = np.empty(81)
        b = np.empty(25)
        lib().oref_inverse_matrices(self._h, _dp(a), _dp(b))
        return a.reshape(9, 9), b.reshape(5, 5)


def central_moments(f, ux, uy):
    f = _f64(f)
    out = np.empty(9)
    lib().oref_central_moments(_dp(f), ux, uy, _dp(out))
    return out


def thermal_central_moments(g, ux, uy):
    g = _f64(g)
    out = np.empty(5)
    lib().oref_thermal_central_moments(_dp(g), ux, uy, _dp(out))
    return out


def moment_matrix():
    M = np.empty(81)
    lib().oref_moment_matrix(_dp(M))
    return M.reshape(9, 9)


def shift_matrix(ux, uy):
    N = np.empty(81)
    lib().oref_shift_matrix(ux, uy, _dp(N))
    return N.reshape(9, 9)


def thermal_moment_matrix():
    M = np.empty(25)
    lib().oref_thermal_moment_matrix(_dp(M))
    return M.reshape(5, 5)


def thermal_shift_matrix(ux, uy):
    N = np.empty(25)
    lib().oref_thermal_shift_matrix(ux, uy, _dp(N))
    return N.reshape(5, 5)


def wall_temperature(b1, b2, b3, ne, T1, T2, have_T2=True):
    return lib().oref_wall_temperature(b1, b2, b3, ne, T1, T2, int(have_T2))


def wall_temperature_q(b1, b2, b3, ne, q, T1, T2, have_T2=True):
    """T_w of a wall at the fraction q of the link."""
    return lib().oref_wall_temperature_q(b1, b2, b3, ne, q, T1, T2, int(have_T2))


def midpoint_temperature_q(q, Tw, T1, T2, T3=0.0, have_T2=True, have_T3=True, dirichlet=False):
    """The wall profile at the link midpoint, the value Eq. 26 imposes there."""
    return lib().oref_midpoint_temperature_q(q, Tw, T1, T2, int(have_T2), T3, int(have_T3),
                                             int(dirichlet))


def threads() -> int:
    return lib().oref_threads()


def set_threads(n: int):
    lib().oref_set_threads(int(n))


def from_workload(w) -> Oracle:
    return Oracle(w.params, w.geom, w.init)
