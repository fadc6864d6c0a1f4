"""Learned warm start for steady solves (an extension beyond the paper).

A U-Net (paper_1801_04577_gb300.net, trained by the library's own kernels)
maps a problem description on a G x G grid -- fluid mask, wall-temperature
markers, log Ra, Pr and the heat source -- to the steady T, u_x, u_y.  Its
prediction initialises the lattice (clbm_init_fields, equilibrium at the
predicted fields) and the plain cascaded LBM refines it to the residual
tolerance: the solver stays the judge of the answer, and a lattice without a
prediction simply starts from rest.

Pipeline: generate steady states with the batched solver, train, then compare
warm- and rest-started batched solves on held-out problems.
"""
from __future__ import annotations

import time
from typing import List, Sequence

import numpy as np

from . import clbm
from . import inputs as I
from .net import Net

IN_CH, OUT_CH = 5, 3


def encode(ws: Sequence[I.Workload]) -> np.ndarray:
    """Network input [N, 5, G, G]: fluid mask, wall-temperature marker (+1 next
    to the hot wall, -1 next to the cold wall), log10 Ra - 4, (Pr - 3.85)/3.15,
    log10(1 + Q/1e-6)/2 -- the last three as constant planes."""
    G = ws[0].params.nx
    x = np.zeros((len(ws), IN_CH, G, G), np.float32)
    for i, w in enumerate(ws):
        fluid = 1.0 if w.geom.solid is None else (w.geom.solid == 0).astype(np.float32)
        x[i, 0] = fluid
        x[i, 1, :, 0] = 1.0
        x[i, 1, :, G - 1] = -1.0
        x[i, 1] *= x[i, 0]
        x[i, 2] = np.log10(w.Ra) - 4.0
        x[i, 3] = (w.Pr - 3.85) / 3.15
        x[i, 4] = np.log10(1.0 + w.params.Q / 1e-6) / 2.0
    return x


def targets_from_fields(ws, fields) -> np.ndarray:
    """[N, 3, G, G]: T - T0, u_x / U, u_y / U (zero at solid nodes)."""
    G = ws[0].params.nx
    y = np.zeros((len(ws), OUT_CH, G, G), np.float32)
    for i, (w, (rho, ux, uy, T)) in enumerate(zip(ws, fields)):
        y[i, 0] = T - w.params.T0
        y[i, 1] = ux / w.u_scale
        y[i, 2] = uy / w.u_scale
        if w.geom.solid is not None:
            y[i, :, w.geom.solid == 1] = 0.0
    return y


def fields_from_prediction(ws, y: np.ndarray):
    """Inverse of targets_from_fields: (T, u_x, u_y) per problem."""
    out = []
    for i, w in enumerate(ws):
        T = y[i, 0].astype(np.float64) + w.params.T0
        ux = y[i, 1].astype(np.float64) * w.u_scale
        uy = y[i, 2].astype(np.float64) * w.u_scale
        if w.geom.solid is not None:
            s = w.geom.solid == 1
            T[s], ux[s], uy[s] = w.params.T0, 0.0, 0.0
        out.append((T, ux, uy))
    return out


# Steps taken before the period-2 filter of a warm start (see clbm_damp_period2).
WARM_PRESTEPS = 2


def solve(ws, tol: float, max_steps: int, check_every: int = 100, precision: str = "f32",
          stream=None, warm: bool = False):
    """Batched solve; returns (batch, conv_steps, residuals, steps_run, seconds).

    warm=True: the lattices start from predicted fields; after WARM_PRESTEPS
    steps the state is replaced by the mean of its last two states, which
    removes the undamped period-2 component such a start excites.  Those steps
    are included in the returned counts and time."""
    b = clbm.Batch(ws, precision, autotune=True, stream=stream)
    t0 = time.perf_counter()
    pre = 0
    if warm:
        b.solve(0.0, WARM_PRESTEPS, WARM_PRESTEPS)
        b.damp_period2()
        pre = WARM_PRESTEPS
    conv, res, steps = b.solve(tol, max_steps, check_every)
    conv = np.where(conv > 0, conv + pre, conv)
    return b, conv, res, steps + pre, time.perf_counter() - t0


def generate(ws, tol: float = 1e-6, max_steps: int = 40000, check_every: int = 100, stream=None):
    """Steady states of the given problems from the batched solver."""
    b, conv, res, steps, el = solve(ws, tol, max_steps, check_every, stream=stream)
    fields = [b.moments(i) for i in range(len(ws))]
    b.close()
    return targets_from_fields(ws, fields), conv, el


def make_net(G: int, base: int, levels: int, max_batch: int, seed: int = 7, stream=None,
             math: str = "tensor") -> Net:
    return Net(G, IN_CH, OUT_CH, base, levels, max_batch, seed=seed, stream=stream, math=math)


def train(net: Net, X, Y, M, epochs: int, batch: int, lr: float, seed: int = 11, log=None,
          lr_final: float = None):
    """Adam on minibatches of the torch CUDA tensors X [N,5,G,G], Y [N,3,G,G], M [N,G,G];
    the learning rate decays geometrically from lr to lr_final over the epochs
    (constant when lr_final is None)."""
    import torch
    n = X.shape[0]
    losses = []
    lr0 = lr
    for ep in range(epochs):
        if lr_final is not None and epochs > 1:
            lr = lr0 * (lr_final / lr0) ** (ep / (epochs - 1))
        perm = np.argsort(I.splitmix64_uniform(seed + ep, n))
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(perm[s:s + batch], device=X.device)
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            mb = M.index_select(0, idx).contiguous()
            tot += net.train_step(xb, yb, mb, lr)
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return losses


def predict(net: Net, ws, stream_sync=True):
    import torch
    X = torch.from_numpy(encode(ws)).cuda()
    Y = torch.empty((len(ws), OUT_CH, X.shape[2], X.shape[3]), dtype=torch.float32, device=X.device)
    bs = net.cfg.max_batch
    for s in range(0, len(ws), bs):
        net.forward(X[s:s + bs], Y[s:s + bs])
    if stream_sync:
        torch.cuda.synchronize()
    return Y.cpu().numpy()


def warm_workloads(ws, y):
    out = []
    for w, (T, ux, uy) in zip(ws, fields_from_prediction(ws, y)):
        w2 = I.Workload(w.name + "_warm", w.params, w.geom, I.Fields(ux=ux, uy=uy, T=T), w.length,
                        w.dT, w.u_scale)
        w2.Ra, w2.Pr = w.Ra, w.Pr
        out.append(w2)
    return out


def compare_starts(net: Net, ws, tol: float, max_steps: int, check_every: int = 100, stream=None):
    """Rest start vs warm start on the same problems: steps, wall time (warm
    includes inference) and the converged Nusselt numbers of both."""
    import torch
    b0, conv0, res0, steps0, t0 = solve(ws, tol, max_steps, check_every, stream=stream)
    nu0 = [b0.nusselt(i, 0, w.length, 1.0) for i, w in enumerate(ws)]
    b0.close()
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    y = predict(net, ws)
    t_inf = time.perf_counter() - t_inf
    b1, conv1, res1, steps1, t1 = solve(warm_workloads(ws, y), tol, max_steps, check_every, stream=stream,
                                        warm=True)
    nu1 = [b1.nusselt(i, 0, w.length, 1.0) for i, w in enumerate(ws)]
    b1.close()
    return {"rest_steps": conv0, "warm_steps": conv1, "rest_time_s": t0, "warm_time_s": t1 + t_inf,
            "inference_s": t_inf, "nu_rest": np.array(nu0), "nu_warm": np.array(nu1),
            "rest_steps_run": steps0, "warm_steps_run": steps1}


def reference_nusselt(ws, tol: float = 1e-11, max_steps: int = 400000, stream=None):
    """Steady wall-0 Nusselt numbers from an FP64 batched solve to a tight tolerance."""
    b, conv, res, steps, el = solve(ws, tol, max_steps, 200, precision="f64", stream=stream)
    nu = np.array([b.nusselt(i, 0, w.length, 1.0) for i, w in enumerate(ws)])
    b.close()
    return nu, conv


def nusselt_settling(net: Net, ws, nu_ref, chunk: int = 1000, horizon: int = 120000,
                     thresholds=(1e-2, 1e-3), stream=None):
    """Time to steady state measured on the observable: for rest and warm
    starts, the number of steps after which the wall Nusselt number stays
    within each relative threshold of the reference.  Warm starts include the
    inference time and the period-2 filter."""
    import torch
    out = {}
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    y = predict(net, ws)
    t_inf = time.perf_counter() - t_inf
    for name, wl in (("rest", ws), ("warm", warm_workloads(ws, y))):
        b = clbm.Batch(wl, "f32", autotune=True, stream=stream)
        el, pre = 0.0, 0
        if name == "warm":
            t0 = time.perf_counter()
            b.solve(0.0, WARM_PRESTEPS, WARM_PRESTEPS)
            b.damp_period2()
            el += time.perf_counter() - t0
            pre = WARM_PRESTEPS
        traj = []
        for _ in range(horizon // chunk):
            t0 = time.perf_counter()
            b.solve(0.0, chunk, chunk)
            el += time.perf_counter() - t0
            traj.append([b.nusselt(i, 0, w.length, 1.0) for i, w in enumerate(wl)])
        b.close()
        err = np.abs(np.array(traj) - nu_ref[None]) / np.abs(nu_ref[None])
        step_s = el / (horizon + pre)
        res = {"seconds_per_batch_step": step_s}
        for thr in thresholds:
            bad = err >= thr
            settle = []
            for j in range(err.shape[1]):
                idx = np.where(bad[:, j])[0]
                first = 0 if len(idx) == 0 else idx[-1] + 1
                settle.append((first + 1) * chunk + pre if first < err.shape[0] else np.inf)
            res[thr] = np.array(settle, dtype=np.float64)
        out[name] = res
    out["inference_s"] = t_inf
    return out
