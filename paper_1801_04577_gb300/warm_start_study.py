"""Warm-start study: does a learned initial state shorten steady solves?

    python -m paper_1801_04577_gb300.warm_start_study --grid 128 --train 3000 --test 64

1. Seeded obstacle cavities (inputs.obstacle_cavities) are solved to steady
   state by the batched solver; the converged (T, u_x, u_y) are the targets.
2. The U-Net (tensor-core convolutions) is trained on them by the library's
   own kernels.
3. On held-out cavities, rest and warm starts are advanced side by side and
   the step after which the hot-wall Nusselt number stays within 1 %
   and 0.1 % of a tightly converged reference is recorded for each start, with
   the wall time per batched step and the inference time; the prediction's
   field error against the converged temperature is reported too.

Everything runs on the GPU through the C ABI; the printed JSON summary is the
result (and is written to --out when given).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import surrogate as SG


def _log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def run(G: int = 128, n_train: int = 3000, n_test: int = 64, ra_max: float = 1e6,
        levels: int = 5, base: int = 16, epochs: int = 300, batch: int = 32, lr: float = 2e-3,
        lr_final: float = 1e-4,
        gen_tol: float = 1e-7, gen_max_steps: int = 300000, ref_tol: float = 1e-9,
        horizon: int = 400000, chunk: int = 2000, seed_offset: int = 7919) -> dict:
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"grid": G, "n_train": n_train, "n_test": n_test, "ra_range": [1e3, ra_max],
           "levels": levels, "base": base, "epochs": epochs, "batch": batch, "lr": [lr, lr_final]}

    # 1. training data
    t0 = time.perf_counter()
    ws = I.obstacle_cavities(n_train, G, ra_range=(1e3, ra_max))
    Y, conv, t_solve = SG.generate(ws, gen_tol, gen_max_steps, check_every=1000,
                                   stream=stream.cuda_stream)
    ok = conv > 0
    out["train_converged"] = int(ok.sum())
    out["train_solve_s"] = t_solve
    out["train_median_steps"] = float(np.median(conv[ok])) if ok.any() else None
    _log(f"data: {ok.sum()}/{n_train} converged to {gen_tol:g} in {t_solve:.1f} s")
    ws_ok = [w for w, k in zip(ws, ok) if k]
    X = torch.from_numpy(SG.encode(ws_ok)).cuda()
    Yd = torch.from_numpy(Y[ok]).cuda()
    M = X[:, 0].contiguous()

    # 2. training
    net = SG.make_net(G, base=base, levels=levels, max_batch=batch, seed=9, stream=stream.cuda_stream)
    out["parameters"] = net.nparam
    t1 = time.perf_counter()
    losses = SG.train(net, X, Yd, M, epochs=epochs, batch=batch, lr=lr, lr_final=lr_final,
                      log=lambda m: _log(m) if m.split(":")[0].endswith("0") else None)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t1
    out["loss_first_last"] = [losses[0], losses[-1]]
    _log(f"trained {net.nparam} parameters for {epochs} epochs in {out['train_s']:.1f} s")
    del X, Yd, M

    # 3. held-out problems: reference, prediction error, settling of rest / warm starts
    wt = I.obstacle_cavities(n_test, G, seed=I.SURROGATE_SEED + seed_offset, ra_range=(1e3, ra_max))
    b, conv_ref, _, _, t_ref = SG.solve(wt, ref_tol, 2 * horizon, 1000, stream=stream.cuda_stream)
    good = np.where(conv_ref > 0)[0]  # judged only where the reference converged
    nu_ref = np.array([b.nusselt(int(i), 0, wt[i].length, 1.0) for i in good])
    T_ref = [b.moments(int(i))[3] for i in good]
    b.close()
    out["reference_converged"] = int(len(good))
    wt = [wt[i] for i in good]
    y = SG.predict(net, wt)
    errs = []
    for w, yi, Tr in zip(wt, y, T_ref):
        fl = np.ones_like(Tr, bool) if w.geom.solid is None else w.geom.solid == 0
        Tp = yi[0].astype(np.float64) + w.params.T0
        errs.append(np.sqrt(((Tp - Tr)[fl] ** 2).sum() / ((Tr[fl] - w.params.T0) ** 2).sum()))
    out["prediction_T_rel_L2_median"] = float(np.median(errs))
    _log(f"reference: {out['reference_converged']}/{n_test} converged ({t_ref:.1f} s); "
         f"prediction T error median {out['prediction_T_rel_L2_median']:.3e}")
    r = SG.nusselt_settling(net, wt, nu_ref, chunk=chunk, horizon=horizon, stream=stream.cuda_stream)
    out["inference_s"] = r["inference_s"]
    for thr in (1e-2, 1e-3):
        rest, warm = r["rest"][thr], r["warm"][thr]
        both = np.isfinite(rest) & np.isfinite(warm)
        key = f"nu_within_{thr:g}"
        out[key] = {
            "settled_both": int(both.sum()),
            "rest_median_steps": float(np.median(rest[both])) if both.any() else None,
            "warm_median_steps": float(np.median(warm[both])) if both.any() else None,
            "warm_faster_fraction": float((warm[both] < rest[both]).mean()) if both.any() else None,
            "rest_batch_wall_s": float(np.max(rest[both]) * r["rest"]["seconds_per_batch_step"]) if both.any() else None,
            "warm_batch_wall_s": float(np.max(warm[both]) * r["warm"]["seconds_per_batch_step"]
                                       + r["inference_s"]) if both.any() else None,
        }
        _log(f"{key}: {out[key]}")
    out["total_s"] = time.perf_counter() - t0
    net.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--train", type=int, default=3000)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--ra-max", type=float, default=1e6)
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--base", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--horizon", type=int, default=400000)
    ap.add_argument("--chunk", type=int, default=2000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = run(G=a.grid, n_train=a.train, n_test=a.test, ra_max=a.ra_max, levels=a.levels, base=a.base,
              epochs=a.epochs, batch=a.batch, horizon=a.horizon, chunk=a.chunk)
    print(json.dumps(res), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
