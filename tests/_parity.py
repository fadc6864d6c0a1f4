"""Shared helpers of the parity tests (not a test module)."""
import numpy as np

import oracle
from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I

FIELDS = ("rho", "ux", "uy", "T")

# Per-field relative max-norm tolerances against the FP64 oracle.
TOL = {"f64": 1e-12, "f32": 1e-5}


def rel_inf(a, b, mask=None):
    """||a - b||_inf / ||b||_inf over the fluid nodes (deviation from rho0 for rho)."""
    if mask is not None:
        a, b = a[mask], b[mask]
    den = np.abs(b).max()
    if den == 0:
        return float(np.abs(a - b).max())
    return float(np.abs(a - b).max() / den)


def compare(w, gpu_fields, ora_fields, floor=False, vanishing=()):
    """Per-field max-norm errors ||a - b||_inf / ||b||_inf over the fluid nodes
    (the density as rho - rho0), each field against its own largest value.

    floor=True divides by max(||b||_inf, field scale) instead, the scale being
    rho0 for the density, the characteristic velocity U for u_x and u_y and the
    temperature difference for T; `vanishing` names the fields that get that
    floor alone.  A test passes either only where it states why: a field that
    is zero in exact arithmetic (u_y and rho - rho0 in a channel flow) or
    still tiny (a few steps from rest) is the difference of O(rho0) populations,
    so its rounding error is set by rho0 and U, not by its own size.
    """
    mask = None if w.geom.solid is None else (w.geom.solid == 0)
    scales = {"rho": w.params.rho0, "ux": w.u_scale, "uy": w.u_scale, "T": w.dT}
    out = {}
    for name, a, b in zip(FIELDS, gpu_fields, ora_fields):
        if name == "rho":
            a, b = a - w.params.rho0, b - w.params.rho0
        if mask is not None:
            a, b = a[mask], b[mask]
        den = float(np.abs(b).max())
        if floor or name in vanishing:
            den = max(den, abs(scales[name]))
        err = float(np.abs(a - b).max())
        out[name] = err / den if den > 0 else err
    return out


def run_pair(w, steps, precision="f64", floor=False, vanishing=()):
    s = clbm.from_workload(w, precision)
    o = oracle.from_workload(w)
    s.step(steps)
    o.step(steps)
    g = s.moments()
    r = o.moments()
    s_obj = (s, o)
    return compare(w, g, r, floor, vanishing), s_obj
