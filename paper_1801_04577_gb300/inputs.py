"""Seeded synthetic workloads for the cascaded thermal lattice Boltzmann solver.

This module only *describes* problems: lattice sizes, relaxation rates, wall
types, solid masks, wall-link lists and initial fields.  It contains none of
the scheme's arithmetic (no moments, no collision, no streaming), so that both
the CUDA library and the FP64 oracle can be driven by exactly the same inputs
without sharing any code that computes the method.

Conventions shared by every consumer of these descriptions:

* Nodes sit at cell centres (x + 1/2, y + 1/2), x = 0..nx-1, y = 0..ny-1,
  arrays are row major ``[ny][nx]``.  Walls of a non-periodic side lie half a
  lattice spacing outside the first/last node (half-way bounce-back, Sec. 3).
* D2Q9 velocities follow Eq. 3: ex = [0,1,0,-1,0,1,-1,-1,1],
  ey = [0,0,1,0,-1,1,1,-1,-1]; D2Q5 uses the first five of them (Sec. 2.2).
* A thermal boundary condition (Sec. 2.3) is a triple (b1, b2, b3) meaning
  b1 dT/dn + b2 T = b3 with n the unit normal pointing out of the fluid.
* ``side_tbc`` gives the condition index of the four box sides in the order
  x0 (left), x1 (right), y0 (bottom), y1 (top); it is ignored on periodic axes.
* A wall link (node, dir, n_dot_e, tbc) says that the D2Q5 link ``dir``
  (1..4) leaving fluid node ``node = y*nx + x`` enters a solid node; this is
  the e_i of Eq. 26-28, and n_dot_e is n.e_i of Eq. 27-28 (> 0).
"""
from __future__ import annotations

import dataclasses
import math
from fractions import Fraction
from typing import List, Optional, Sequence, Tuple

import numpy as np

EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)

SIDE_X0, SIDE_X1, SIDE_Y0, SIDE_Y1 = 0, 1, 2, 3

# Lattice sound speed of the D2Q5 temperature lattice used throughout Sec. 3.
CT2_PAPER = 0.4


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters of one lattice (all lattice units).

    s_3 <= 0 selects the non-slip rule s3 = (16 - 8 s_nu)/(8 - s_nu) (Sec. 3);
    lambda2 <= 0 selects lambda2 = 12(lambda1 - 2)/(lambda1 - 12) (Sec. 3.1).
    Both rules are applied by the solver that consumes the parameters.
    """

    nx: int
    ny: int
    periodic_x: int = 0
    periodic_y: int = 0
    s_nu: float = 1.0
    s_b: float = 1.0
    s_3: float = -1.0
    s_4: float = 1.0
    lambda0: float = 1.0
    lambda1: float = 1.0
    lambda2: float = -1.0
    rho0: float = 1.0
    T0: float = 0.0
    gbeta: float = 0.0
    Fvx: float = 0.0
    Fvy: float = 0.0
    Q: float = 0.0
    cT2: float = CT2_PAPER
    viscous_heating: int = 0  # 1: add the viscous dissipation source of Sec. 3.2


@dataclasses.dataclass
class Geometry:
    """Walls of one lattice: box sides, an optional solid mask and wall links."""

    tbc: List[Tuple[float, float, float]]
    side_tbc: Tuple[int, int, int, int] = (-1, -1, -1, -1)
    solid: Optional[np.ndarray] = None  # uint8 [ny][nx], 1 = solid
    link_node: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    link_dir: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    link_ne: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.float64))
    link_tbc: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    # fraction q in (0, 1] of each link from the fluid node to the wall; None = 1/2 for
    # every link (the paper's half-way walls).  Links of directions 5..8 carry only q.
    link_q: Optional[np.ndarray] = None
    # velocity (ux, uy) of each box side x0, x1, y0, y1 for the moving-wall
    # bounce-back (not in the paper); None = every side at rest
    side_u: Optional[Tuple[Tuple[float, float], ...]] = None

    @property
    def n_links(self) -> int:
        return int(self.link_node.shape[0])

    def link_q_or_half(self) -> np.ndarray:
        if self.link_q is None:
            return np.full(self.n_links, 0.5)
        return np.ascontiguousarray(self.link_q, np.float64)


@dataclasses.dataclass
class Fields:
    """Initial macroscopic fields (FP64, [ny][nx]); None means the rest value."""

    rho: Optional[np.ndarray] = None
    ux: Optional[np.ndarray] = None
    uy: Optional[np.ndarray] = None
    T: Optional[np.ndarray] = None


@dataclasses.dataclass
class Workload:
    name: str
    params: Params
    geom: Geometry
    init: Fields
    length: float = 1.0  # characteristic length H for Nusselt numbers
    dT: float = 1.0      # characteristic temperature difference
    u_scale: float = 0.1  # characteristic velocity (U of Sec. 3.3 for buoyant flows)


def dirichlet(T: float) -> Tuple[float, float, float]:
    return (0.0, 1.0, float(T))


def neumann(flux: float = 0.0) -> Tuple[float, float, float]:
    return (1.0, 0.0, float(flux))


def robin(b1: float, b2: float, b3: float) -> Tuple[float, float, float]:
    return (float(b1), float(b2), float(b3))


# ---------------------------------------------------------------------------
# Seeded random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014).
# ---------------------------------------------------------------------------
_MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the splitmix64 sequence started at ``seed``.

    Each output takes the top 53 bits of one 64-bit draw.  Vectorised with
    numpy uint64 wrap-around arithmetic, which matches the reference
    definition bit for bit.
    """
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def splitmix64_scalar(seed: int, n: int) -> List[int]:
    """Plain-integer splitmix64 (the published definition), for cross-checks."""
    out = []
    state = seed & _MASK64
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


# ---------------------------------------------------------------------------
# Parameter mapping for buoyancy-driven flows (Sec. 3.3).
# ---------------------------------------------------------------------------
def convection_rates(H: float, Ra: float, Pr: float, U: float = 0.1, dT: float = 1.0,
                     cT2: float = CT2_PAPER):
    """Lattice rates for Pr = nu/alpha, Ra = g beta dT H^3/(nu alpha), U = sqrt(g beta dT H).

    Returns (nu, alpha, s_nu, lambda1, gbeta) using nu = (1/s_nu - 1/2)/3
    (Sec. 2.1) and alpha = (1/lambda1 - 1/2) cT^2 (Sec. 2.2).
    """
    nu = U * H * math.sqrt(Pr / Ra)
    alpha = nu / Pr
    s_nu = 1.0 / (3.0 * nu + 0.5)
    lambda1 = 1.0 / (alpha / cT2 + 0.5)
    gbeta = U * U / (dT * H)
    return nu, alpha, s_nu, lambda1, gbeta


def rates_from_diffusivities(nu: float, alpha: float, cT2: float = CT2_PAPER):
    return 1.0 / (3.0 * nu + 0.5), 1.0 / (alpha / cT2 + 0.5)


# ---------------------------------------------------------------------------
# Workloads.
# ---------------------------------------------------------------------------
def natural_convection_cavity(H: int = 64, Ra: float = 1e4, Pr: float = 0.71, U: float = 0.1,
                              Th: float = 1.0, Tl: float = 0.0) -> Workload:
    """Differentially heated square cavity of Sec. 3.3: left wall Th, right wall Tl,
    adiabatic top and bottom, no-slip everywhere, rest start at T = (Th+Tl)/2."""
    dT = Th - Tl
    nu, alpha, s_nu, lambda1, gbeta = convection_rates(H, Ra, Pr, U, dT)
    T0 = 0.5 * (Th + Tl)
    p = Params(nx=H, ny=H, s_nu=s_nu, lambda1=lambda1, T0=T0, gbeta=gbeta)
    g = Geometry(tbc=[dirichlet(Th), dirichlet(Tl), neumann(0.0)],
                 side_tbc=(0, 1, 2, 2))
    return Workload(f"cavity_{H}x{H}_Ra{Ra:g}", p, g, Fields(), length=float(H), dT=dT)


RB_SEED = 1801045770


def rayleigh_benard(nx: int = 4096, ny: int = 2048, Ra: float = 1e6, Pr: float = 0.71,
                    U: float = 0.1, Q: float = 1e-5, noise: float = 1e-3,
                    seed: int = RB_SEED) -> Workload:
    """Rayleigh-Benard cell: periodic in x, bottom T=1, top T=0, uniform source Q.

    Initial T = 1 - (y + 1/2)/H + noise * (2u - 1) with u drawn by splitmix64
    (one draw per node, row-major order), at rest with rho = rho0.
    """
    H = ny
    nu, alpha, s_nu, lambda1, gbeta = convection_rates(H, Ra, Pr, U, 1.0)
    p = Params(nx=nx, ny=ny, periodic_x=1, s_nu=s_nu, lambda1=lambda1, T0=0.5,
               gbeta=gbeta, Q=Q)
    g = Geometry(tbc=[dirichlet(1.0), dirichlet(0.0)], side_tbc=(-1, -1, 0, 1))
    y = (np.arange(ny, dtype=np.float64) + 0.5) / H
    T = np.repeat((1.0 - y)[:, None], nx, axis=1)
    if noise:
        T = T + noise * (2.0 * splitmix64_uniform(seed, nx * ny).reshape(ny, nx) - 1.0)
    return Workload(f"rayleigh_benard_{nx}x{ny}_Ra{Ra:g}", p, g, Fields(T=T),
                    length=float(H), dT=1.0)


def _ratio_fraction(ratio: float) -> Fraction:
    return Fraction(ratio).limit_denominator(1000)


def annulus(n: int = 2048, ratio: float = 2.6, Ra: float = 1e5, Pr: float = 0.71, U: float = 0.1,
            T_in: float = 1.0, robin_b3: float = 0.0, gravity: bool = True,
            Q: float = 0.0, alpha: Optional[float] = None, interpolated: bool = False) -> Workload:
    """Annulus between concentric cylinders inside an n x n box.

    Centre c = ((n-1)/2, (n-1)/2), outer radius ro = n/2 - 1, inner radius
    ri = ro/ratio.  Inner wall Dirichlet T_in; outer wall Robin with b1 = 1,
    b2 = 1/(ro - ri), b3 = robin_b3.  Fluid/solid classification is done in
    exact integer arithmetic on doubled coordinates, so it is reproducible.
    Wall links carry n.e_i with n the outward (fluid -> wall) unit normal of
    the circle at the point where the link crosses it.  interpolated=True
    also lists the diagonal links and gives every link the fraction q at
    which it crosses the circle; otherwise the walls are half-way (the
    paper's staircase).
    """
    ro = n / 2.0 - 1.0
    fr = _ratio_fraction(ratio)
    ri = ro / float(fr)
    # doubled coordinates: X = 2x - (n-1); r^2 * 4 = X^2 + Y^2
    X = 2 * np.arange(n, dtype=np.int64) - (n - 1)
    R2 = X[None, :] ** 2 + X[:, None] ** 2          # (2r)^2, exact
    two_ro = int(round(2 * ro))
    outer_ok = R2 < two_ro * two_ro
    # (2r)^2 > (2 ro / ratio)^2  <=>  R2 * p^2 > (2 ro)^2 * q^2 with ratio = p/q
    inner_ok = R2 * (fr.numerator ** 2) > (two_ro ** 2) * (fr.denominator ** 2)
    fluid = outer_ok & inner_ok
    solid = (~fluid).astype(np.uint8)
    H = ro - ri
    nu, alpha_c, s_nu, lambda1, gbeta = convection_rates(H, Ra, Pr, U, 1.0)
    if not gravity:
        gbeta = 0.0
    if alpha is not None:  # conduction studies: choose the diffusivity directly
        s_nu, lambda1 = rates_from_diffusivities(alpha * Pr, alpha)
    p = Params(nx=n, ny=n, s_nu=s_nu, lambda1=lambda1, T0=0.5, gbeta=gbeta, Q=Q)
    tbc = [dirichlet(T_in), robin(1.0, 1.0 / H, robin_b3)]
    c = (n - 1) / 2.0
    nodes, dirs, nes, tbcs, qs = [], [], [], [], []
    ys, xs = np.nonzero(fluid)
    for d in ((1, 2, 3, 4, 5, 6, 7, 8) if interpolated else (1, 2, 3, 4)):
        ex, ey = EX[d], EY[d]
        xn, yn = xs + ex, ys + ey
        inb = (xn >= 0) & (xn < n) & (yn >= 0) & (yn < n)
        hit = np.zeros_like(inb)
        hit[inb] = solid[yn[inb], xn[inb]] == 1
        hit |= ~inb
        for x, y in zip(xs[hit], ys[hit]):
            # which circle: the solid neighbour is inside ri or outside ro
            rx, ry = x + ex - c, y + ey - c
            inner = (rx * rx + ry * ry) < ro * ro  # neighbour inside the outer circle -> inner wall
            R = ri if inner else ro
            # link crossing: |(x - c) + s e| = R for s in (0, 1)
            px, py = x - c, y - c
            # s^2 + 2 s (p.e) + |p|^2 - R^2 = 0
            pe = px * ex + py * ey
            disc = pe * pe - (px * px + py * py - R * R)
            disc = max(disc, 0.0)
            roots = (-pe - math.sqrt(disc), -pe + math.sqrt(disc))
            s = min((r for r in roots if r >= -1e-12), default=0.5)
            s = min(max(s, 0.0), 1.0)
            qx, qy = px + s * ex, py + s * ey
            rq = math.hypot(qx, qy)
            if inner:
                nx_, ny_ = -qx / rq, -qy / rq
            else:
                nx_, ny_ = qx / rq, qy / rq
            ne = nx_ * ex + ny_ * ey
            nodes.append(int(y) * n + int(x))
            dirs.append(d)
            # diagonal links carry only q (the thermal lattice has no diagonal links)
            nes.append(max(ne, 1e-3) if d <= 4 else 0.0)
            tbcs.append((0 if inner else 1) if d <= 4 else -1)
            qs.append(min(max(s, 1e-3), 1.0))
    order = np.lexsort((np.asarray(dirs), np.asarray(nodes)))
    g = Geometry(tbc=tbc, side_tbc=(1, 1, 1, 1), solid=solid,
                 link_node=np.asarray(nodes, np.int32)[order],
                 link_dir=np.asarray(dirs, np.int32)[order],
                 link_ne=np.asarray(nes, np.float64)[order],
                 link_tbc=np.asarray(tbcs, np.int32)[order],
                 link_q=np.asarray(qs, np.float64)[order] if interpolated else None)
    T = np.full((n, n), 0.5)
    name = f"annulus_{n}x{n}_ratio{ratio:g}" + ("_interpolated" if interpolated else "")
    return Workload(name, p, g, Fields(T=T), length=H, dT=1.0)


def axis_links(solid: np.ndarray, tbc_index: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Wall links with n.e = 1 for every D2Q5 link from a fluid node into a solid
    node of ``solid`` (suitable for axis-aligned rectangular obstacles)."""
    ny, nx = solid.shape
    nodes, dirs = [], []
    ys, xs = np.nonzero(solid == 0)
    for d in (1, 2, 3, 4):
        xn, yn = xs + EX[d], ys + EY[d]
        inb = (xn >= 0) & (xn < nx) & (yn >= 0) & (yn < ny)
        hit = np.zeros_like(inb)
        hit[inb] = solid[yn[inb], xn[inb]] == 1
        nodes.extend((ys[hit] * nx + xs[hit]).tolist())
        dirs.extend([d] * int(hit.sum()))
    nodes = np.asarray(nodes, np.int32)
    dirs = np.asarray(dirs, np.int32)
    order = np.lexsort((dirs, nodes))
    m = nodes.shape[0]
    return nodes[order], dirs[order], np.ones(m), np.full(m, tbc_index, np.int32)


def diffusion_channel(alpha: float, lambda2: float = -1.0, L: int = 6, nx: int = 4,
                      T_bottom: float = 0.0, T_top: float = 1.0, with_source: bool = True) -> Workload:
    """Steady 1-D diffusion with a uniform source (Sec. 3.1, Eq. 29).

    L fluid nodes across, periodic along x, Dirichlet walls at y = 0 and y = L,
    Q = 2 alpha dT / L^2 (so the exact profile is a parabola), fluid at rest.
    """
    dT = T_top - T_bottom
    Q = 2.0 * alpha * dT / (L * L) if with_source else 0.0
    s_nu, lambda1 = rates_from_diffusivities(0.1, alpha)
    p = Params(nx=nx, ny=L, periodic_x=1, s_nu=s_nu, lambda1=lambda1, lambda2=lambda2,
               T0=0.0, Q=Q)
    g = Geometry(tbc=[dirichlet(T_bottom), dirichlet(T_top)], side_tbc=(-1, -1, 0, 1))
    T = np.full((L, nx), 0.5 * (T_bottom + T_top))
    return Workload(f"diffusion_L{L}_alpha{alpha:g}", p, g, Fields(T=T), length=float(L), dT=dT)


def diffusion_exact(L: int, T_bottom: float = 0.0, T_top: float = 1.0) -> np.ndarray:
    """Exact profile of Sec. 3.1 at the node centres y = j + 1/2."""
    y = np.arange(L) + 0.5
    return T_bottom + (T_top - T_bottom) * (y / L) * (2.0 - y / L)


def poiseuille_channel(ny: int = 8, nu: float = 0.1, Fx: float = 1e-5, nx: int = 4,
                       s_b: Optional[float] = None, Tw: float = 0.0) -> Workload:
    """Body-force-driven channel flow between no-slip walls at y = 0 and y = ny
    (periodic in x), isothermal walls at Tw."""
    s_nu, lambda1 = rates_from_diffusivities(nu, 0.1)
    p = Params(nx=nx, ny=ny, periodic_x=1, s_nu=s_nu, s_b=s_nu if s_b is None else s_b,
               lambda1=lambda1, Fvx=Fx, T0=Tw)
    g = Geometry(tbc=[dirichlet(Tw)], side_tbc=(-1, -1, 0, 0))
    return Workload(f"poiseuille_{ny}", p, g, Fields(T=np.full((ny, nx), Tw)), length=float(ny),
                    u_scale=Fx * ny * ny / (8.0 * nu))


def offset_channel(N: int = 8, q_bottom: float = 0.3, q_top: float = 0.8, nu: float = 0.1,
                   alpha: float = 0.1, Fx: float = 1e-5, T_bottom: float = 1.0, T_top: float = 0.0,
                   nx: int = 4, top_tbc: Optional[Tuple[float, float, float]] = None,
                   Q: float = 0.0) -> Workload:
    """Channel whose walls are not half-way between nodes: solid rows y = 0 and
    y = N + 1, fluid rows 1..N, the bottom wall at y = 1 - q_bottom and the top
    wall at y = N + q_top (every link into a wall row, diagonal ones included,
    carries that fraction); periodic in x and y; body force Fx, uniform heat
    source Q, no gravity; Dirichlet T_bottom at the bottom, T_top or the
    condition top_tbc = (b1, b2, b3) at the top.  offset_channel_exact gives
    the steady solution."""
    ny = N + 2
    s_nu, lambda1 = rates_from_diffusivities(nu, alpha)
    p = Params(nx=nx, ny=ny, periodic_x=1, periodic_y=1, s_nu=s_nu, lambda1=lambda1, Fvx=Fx,
               T0=0.5 * (T_bottom + T_top), Q=Q)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    nodes, dirs, nes, tbcs, qs = [], [], [], [], []
    for x in range(nx):
        for d in (4, 7, 8):  # into the bottom wall row
            nodes.append(nx + x); dirs.append(d); qs.append(q_bottom)
            nes.append(1.0 if d == 4 else 0.0); tbcs.append(0 if d == 4 else -1)
        for d in (2, 5, 6):  # into the top wall row
            nodes.append(N * nx + x); dirs.append(d); qs.append(q_top)
            nes.append(1.0 if d == 2 else 0.0); tbcs.append(1 if d == 2 else -1)
    order = np.lexsort((np.asarray(dirs), np.asarray(nodes)))
    top = dirichlet(T_top) if top_tbc is None else robin(*top_tbc)
    g = Geometry(tbc=[dirichlet(T_bottom), top], side_tbc=(-1, -1, -1, -1), solid=solid,
                 link_node=np.asarray(nodes, np.int32)[order], link_dir=np.asarray(dirs, np.int32)[order],
                 link_ne=np.asarray(nes, np.float64)[order], link_tbc=np.asarray(tbcs, np.int32)[order],
                 link_q=np.asarray(qs, np.float64)[order])
    L = N + q_top - (1.0 - q_bottom)
    return Workload(f"offset_channel_{N}_q{q_bottom:g}_{q_top:g}", p, g,
                    Fields(T=np.full((ny, nx), p.T0)), length=L, u_scale=Fx * L * L / (8.0 * nu))


def offset_channel_exact(w: Workload, nu: float, alpha: float, T_bottom: float = 1.0):
    """(u_x, T) at rows 0..ny-1 of offset_channel (rows 0 and ny-1 are solid):
    u = Fx/(2 nu) (y - yb)(yt - y); with x = y - yb and L = yt - yb,
    T = T_bottom + s x + Q/(2 alpha) x (L - x), s fixed by the top condition
    b1 T'(L) + b2 T(L) = b3 (n = +y there)."""
    ny = w.params.ny
    N = ny - 2
    q, dirs = w.geom.link_q, w.geom.link_dir
    yb, yt = 1.0 - float(q[dirs == 4][0]), N + float(q[dirs == 2][0])
    L = yt - yb
    Fx, Q = w.params.Fvx, w.params.Q
    y = np.arange(ny, dtype=np.float64)
    u = Fx / (2.0 * nu) * (y - yb) * (yt - y)
    b1, b2, b3 = w.geom.tbc[1]
    c = Q / (2.0 * alpha)
    # b1 (s - c L) + b2 (T_bottom + s L) = b3
    s = (b3 - b2 * T_bottom + b1 * c * L) / (b1 + b2 * L)
    x = y - yb
    return u, T_bottom + s * x + c * x * (L - x)


def dissipation_channel(L: int = 16, nu: float = 0.1, alpha: float = 0.1, Fx: float = 1e-5,
                        nx: int = 4, Tw: float = 0.0) -> Workload:
    """Poiseuille flow with viscous heating (Sec. 3.2): body force Fx between
    no-slip walls at y = 0 and y = L held at Tw, heat source nu (du/dy)^2."""
    s_nu, lambda1 = rates_from_diffusivities(nu, alpha)
    p = Params(nx=nx, ny=L, periodic_x=1, s_nu=s_nu, s_b=s_nu, lambda1=lambda1, Fvx=Fx, T0=Tw,
               viscous_heating=1)
    g = Geometry(tbc=[dirichlet(Tw)], side_tbc=(-1, -1, 0, 0))
    return Workload(f"dissipation_{L}", p, g, Fields(T=np.full((L, nx), Tw)), length=float(L),
                    u_scale=Fx * L * L / (8.0 * nu))


def couette_channel(H: int = 16, Uw: float = 0.05, nu: float = 0.1, alpha: float = 0.1,
                    T_bottom: float = 1.0, T_top: float = 0.0, nx: int = 4,
                    viscous_heating: int = 0) -> Workload:
    """Thermal Couette flow (not in the paper): periodic in x, a wall at rest
    at y = 0 held at T_bottom and a wall at y = H moving along +x at Uw held at
    T_top (Dirichlet).  couette_exact gives the steady solution."""
    s_nu, lambda1 = rates_from_diffusivities(nu, alpha)
    p = Params(nx=nx, ny=H, periodic_x=1, s_nu=s_nu, s_b=s_nu, lambda1=lambda1,
               T0=0.5 * (T_bottom + T_top), viscous_heating=viscous_heating)
    g = Geometry(tbc=[dirichlet(T_bottom), dirichlet(T_top)], side_tbc=(-1, -1, 0, 1),
                 side_u=((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (Uw, 0.0)))
    return Workload(f"couette_{H}{'_vh' if viscous_heating else ''}", p, g,
                    Fields(T=np.full((H, nx), p.T0)), length=float(H), dT=abs(T_bottom - T_top) or 1.0,
                    u_scale=Uw)


def couette_exact(w: Workload, nu: float, alpha: float, T_bottom: float = 1.0,
                  T_top: float = 0.0):
    """(u_x, T) at the node centres s = y + 1/2 of couette_channel: u = Uw s / H;
    T = T_bottom + (T_top - T_bottom) s / H, plus Q_v s (H - s) / (2 alpha) with
    the uniform viscous source Q_v = nu (Uw / H)^2 when it is on (alpha T'' = -Q_v)."""
    H = w.params.ny
    Uw = w.geom.side_u[3][0]
    s = np.arange(H, dtype=np.float64) + 0.5
    u = Uw * s / H
    T = T_bottom + (T_top - T_bottom) * s / H
    if w.params.viscous_heating:
        Qv = nu * (Uw / H) ** 2
        T = T + Qv * s * (H - s) / (2.0 * alpha)
    return u, T


def dissipation_exact(L: int, nu: float, alpha: float, Fx: float, Tw: float = 0.0) -> np.ndarray:
    """Exact profile of Sec. 3.2 at the node centres: Tw + (h^2 Fx / 2)^2 [1 - (y/h)^4] / (3 nu alpha),
    y measured from the channel centre, h the half-width."""
    h = L / 2.0
    y = np.arange(L) + 0.5 - h
    return Tw + (h * h * Fx / 2.0) ** 2 * (1.0 - (y / h) ** 4) / (3.0 * nu * alpha)


def poiseuille_exact(ny: int, nu: float, Fx: float, rho0: float = 1.0) -> np.ndarray:
    """u(y) = Fx/(2 rho0 nu) * y (ny - y) at the node centres y = j + 1/2."""
    y = np.arange(ny) + 0.5
    return Fx / (2.0 * rho0 * nu) * y * (ny - y)


def periodic_box(nx: int = 16, ny: int = 12, seed: int = 7, amp: float = 0.02,
                 gbeta: float = 1e-3, Q: float = 1e-4, Fvx: float = 2e-5,
                 s_nu: float = 1.3, lambda1: float = 1.1) -> Workload:
    """Doubly periodic box with seeded random rho, u, T (conservation checks)."""
    r = splitmix64_uniform(seed, 4 * nx * ny).reshape(4, ny, nx)
    rho = 1.0 + amp * (2 * r[0] - 1)
    ux = amp * (2 * r[1] - 1)
    uy = amp * (2 * r[2] - 1)
    T = 0.5 + 0.25 * (2 * r[3] - 1)
    p = Params(nx=nx, ny=ny, periodic_x=1, periodic_y=1, s_nu=s_nu, lambda1=lambda1,
               T0=0.5, gbeta=gbeta, Q=Q, Fvx=Fvx)
    g = Geometry(tbc=[dirichlet(0.0)], side_tbc=(-1, -1, -1, -1))
    return Workload(f"periodic_{nx}x{ny}", p, g, Fields(rho=rho, ux=ux, uy=uy, T=T), dT=0.5,
                    u_scale=amp)


def random_fields(nx: int, ny: int, seed: int, amp: float = 0.02, T_mid: float = 0.5,
                  T_amp: float = 0.25) -> Fields:
    r = splitmix64_uniform(seed, 4 * nx * ny).reshape(4, ny, nx)
    return Fields(rho=1.0 + amp * (2 * r[0] - 1), ux=amp * (2 * r[1] - 1),
                  uy=amp * (2 * r[2] - 1), T=T_mid + T_amp * (2 * r[3] - 1))


def obstacle_channel(nx: int = 37, ny: int = 19, seed: int = 3) -> Workload:
    """Ragged-size box with walls on all sides, mixed thermal conditions and a
    rectangular adiabatic obstacle (exercises masks, corners and link lists)."""
    solid = np.zeros((ny, nx), np.uint8)
    solid[ny // 3: ny // 3 + 5, nx // 3: nx // 3 + 7] = 1
    tbc = [dirichlet(1.0), robin(1.0, 0.5, 0.1), neumann(0.0), neumann(0.02)]
    ln, ld, le, lt = axis_links(solid, 2)
    g = Geometry(tbc=tbc, side_tbc=(0, 1, 3, 2), solid=solid, link_node=ln, link_dir=ld,
                 link_ne=le, link_tbc=lt)
    p = Params(nx=nx, ny=ny, s_nu=1.2, lambda1=1.3, T0=0.5, gbeta=2e-4, Q=3e-5, Fvx=1e-5)
    return Workload(f"obstacle_{nx}x{ny}", p, g, random_fields(nx, ny, seed, amp=0.01), dT=1.0,
                    u_scale=0.01)


def link_arrays(geom: Geometry) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    return (np.ascontiguousarray(geom.link_node, np.int32), np.ascontiguousarray(geom.link_dir, np.int32),
            np.ascontiguousarray(geom.link_ne, np.float64), np.ascontiguousarray(geom.link_tbc, np.int32))


def fluid_count(w: Workload) -> int:
    if w.geom.solid is None:
        return w.params.nx * w.params.ny
    return int((w.geom.solid == 0).sum())


BATCH_SEED = 1801045771


def random_cavities(n: int = 512, seed: int = BATCH_SEED, hmin: int = 32, hmax: int = 512,
                    U: float = 0.1) -> List[Workload]:
    """Seeded batch of closed cavities of uneven size and physics.

    Per cavity: H ~ U{hmin..hmax}, aspect a ~ U[1, 4], W = min(hmax, round(a H)),
    orientation random (nx, ny) = (W, H) or (H, W); Ra log-uniform in
    [1e3, 1e6]; Pr ~ U[0.7, 7]; Q = 0 with probability 1/2, else log-uniform
    in [1e-6, 1e-4]; each side independently Dirichlet (T = 0 or 1), adiabatic
    or Robin (b1 = 1, b2 = 1/H, b3 = T_amb/H, T_amb ~ U[0, 1]).  Draws with a
    source and no wall that fixes the temperature level (b2 = 0 everywhere) are
    rejected: they have no steady state.  Gravity along -y, the rates follow
    Sec. 3.3 with the vertical size ny as H.
    """
    out = []
    draw = 0
    while len(out) < n:
        r = splitmix64_uniform(seed + 7919 * draw, 16)
        draw += 1
        H = hmin + int(r[0] * (hmax - hmin + 1))
        H = min(H, hmax)
        a = 1.0 + 3.0 * r[1]
        W = min(hmax, int(round(a * H)))
        nx, ny = (W, H) if r[2] < 0.5 else (H, W)
        Ra = 10.0 ** (3.0 + 3.0 * r[3])
        Pr = 0.7 + 6.3 * r[4]
        Q = 0.0 if r[5] < 0.5 else 10.0 ** (-6.0 + 2.0 * r[6])
        tbc, side = [], []
        fixes_level = False
        dirichlet_T = []
        for s in range(4):
            kind = min(2, int(3 * r[7 + s]))
            if kind == 0:
                Tw = 1.0 if r[11 + s] < 0.5 else 0.0
                tbc.append(dirichlet(Tw))
                dirichlet_T.append(Tw)
                fixes_level = True
            elif kind == 1:
                tbc.append(neumann(0.0))
            else:
                tbc.append(robin(1.0, 1.0 / ny, r[11 + s] / ny))
                fixes_level = True
            side.append(s)
        if Q > 0 and not fixes_level:
            continue
        nu, alpha, s_nu, lambda1, gbeta = convection_rates(ny, Ra, Pr, U, 1.0)
        T0 = float(np.mean(dirichlet_T)) if dirichlet_T else 0.5
        p = Params(nx=nx, ny=ny, s_nu=s_nu, lambda1=lambda1, T0=T0, gbeta=gbeta, Q=Q)
        g = Geometry(tbc=tbc, side_tbc=tuple(side))
        w = Workload(f"cavity{len(out)}_{nx}x{ny}_Ra{Ra:.3g}_Pr{Pr:.3g}", p, g,
                     Fields(T=np.full((ny, nx), T0)), length=float(ny), dT=1.0, u_scale=U)
        out.append(w)
    return out


SURROGATE_SEED = 1801045772


def obstacle_cavities(n: int, G: int = 64, seed: int = SURROGATE_SEED, ra_range=(1e3, 1e5),
                      max_obstacles: int = 2, U: float = 0.1) -> List[Workload]:
    """Seeded differentially heated cavities with rectangular obstacles.

    G x G fluid box, left wall T = 1, right wall T = 0, top and bottom
    adiabatic, no-slip everywhere; 0..max_obstacles adiabatic rectangles with
    sides in [G/16, G/4] kept at least two nodes away from the walls; Ra
    log-uniform in ra_range, Pr ~ U[0.7, 7], Q = 0 with probability 1/2, else
    log-uniform in [1e-6, 1e-4].  Rest start at T = 0.5.
    """
    out = []
    for k in range(n):
        r = splitmix64_uniform(seed + 104729 * k, 24)
        lo, hi = np.log10(ra_range[0]), np.log10(ra_range[1])
        Ra = 10.0 ** (lo + (hi - lo) * r[0])
        Pr = 0.7 + 6.3 * r[1]
        Q = 0.0 if r[2] < 0.5 else 10.0 ** (-6.0 + 2.0 * r[3])
        nob = min(max_obstacles, int(r[4] * (max_obstacles + 1)))
        solid = np.zeros((G, G), np.uint8)
        smin, smax = max(2, G // 16), max(3, G // 4)
        for o in range(nob):
            w = smin + int(r[5 + 4 * o] * (smax - smin + 1))
            h = smin + int(r[6 + 4 * o] * (smax - smin + 1))
            x0 = 2 + int(r[7 + 4 * o] * (G - 4 - w))
            y0 = 2 + int(r[8 + 4 * o] * (G - 4 - h))
            solid[y0:y0 + h, x0:x0 + w] = 1
        nu, alpha, s_nu, lambda1, gbeta = convection_rates(G, Ra, Pr, U, 1.0)
        p = Params(nx=G, ny=G, s_nu=s_nu, lambda1=lambda1, T0=0.5, gbeta=gbeta, Q=Q)
        tbc = [dirichlet(1.0), dirichlet(0.0), neumann(0.0)]
        if solid.any():
            ln, ld, le, lt = axis_links(solid, 2)
            g = Geometry(tbc=tbc, side_tbc=(0, 1, 2, 2), solid=solid, link_node=ln, link_dir=ld,
                         link_ne=le, link_tbc=lt)
        else:
            g = Geometry(tbc=tbc, side_tbc=(0, 1, 2, 2))
        out.append(Workload(f"obstacle_cavity{k}_G{G}_Ra{Ra:.3g}", p, g, Fields(T=np.full((G, G), 0.5)),
                            length=float(G), dT=1.0, u_scale=U))
        out[-1].Ra, out[-1].Pr = Ra, Pr
    return out
