"""Time to steady state with and without the learned warm start, judged
against FP64 references (a measurement script, not a test module).

    python tests/measure_warm_start.py --grid 128 --train 20000 --test 32 --out gpurun_out/warm128.json

1. Seeded obstacle cavities on G x G grids (Ra log-uniform 1e3..1e6, Pr
   0.7..7, source 0 or 1e-6..1e-4, 0..2 adiabatic obstacles) are solved to an
   interval residual of --gen-tol by the batched GPU solver; their steady
   (T, u_x, u_y) train the U-Net on the GPU (the library's tensor-core
   kernels).  --save-net / --load-net keep the trained parameters.
2. References: each held-out cavity solved in FP64 by the batched GPU solver to
   an interval residual of --ref-tol (1e-11); the hot-wall Nusselt number is
   the mean over two consecutive steps (closed cavities carry a neutral
   period-2 mode).  The FP64 path is the oracle's scheme step for step (GPU
   parity tests: 1e-12); here it is also checked against the FP64 oracle
   directly: --oracle-cases cavities advanced --oracle-steps steps from rest by
   the oracle (host cores, spawned processes, while the GPU works) and by the
   GPU FP64 path, whose Nusselt numbers and temperature fields must agree.
3. Held-out cavities advanced from rest and from the network's prediction
   (inference time included, period-2 filter after two steps) by the FP32
   batched solver in chunks; a cavity is steady at the first chunk from which
   on its interval residual stays below --tol (1e-6) and its hot-wall Nusselt
   number within --nu-tol (1e-3) of the FP64 reference.  Wall time = steps x
   the measured seconds per batched step (+ inference for the warm start).

The oracle is test infrastructure: this script lives under tests/ for that
reason.  The result is one JSON object (stdout and --out).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1801_04577_gb300 import inputs as I  # noqa: E402


def _log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def two_step_nusselt(nusselt, step):
    """Mean hot-wall Nusselt number over two consecutive steps: closed cavities
    carry a neutral period-2 mode, and the mean removes its alternation."""
    a = nusselt()
    step()
    return 0.5 * (a + nusselt())


def oracle_run(args):
    """FP64 oracle: `steps` steps from rest; two-step mean Nu and T."""
    w, steps = args
    import oracle
    oracle.set_threads(1)
    o = oracle.from_workload(w)
    o.step(steps)
    nu = two_step_nusselt(lambda: o.nusselt(0, w.length, 1.0), lambda: o.step(1))
    return nu, o.moments()[3]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--ra-max", type=float, default=1e6)
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--base", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--gen-tol", type=float, default=1e-6)
    ap.add_argument("--gen-max-steps", type=int, default=400000)
    ap.add_argument("--gen-chunk", type=int, default=5000)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--nu-tol", type=float, default=1e-3)
    ap.add_argument("--ref-tol", type=float, default=1e-11)
    ap.add_argument("--horizon", type=int, default=400000)
    ap.add_argument("--chunk", type=int, default=1000)
    ap.add_argument("--oracle-cases", type=int, default=8)
    ap.add_argument("--oracle-steps", type=int, default=40000)
    ap.add_argument("--oracle-workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--save-net", default=None)
    ap.add_argument("--load-net", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)

    G = a.grid
    wt = I.obstacle_cavities(a.test, G, seed=I.SURROGATE_SEED + 7919, ra_range=(1e3, a.ra_max))
    n_or = min(a.test, a.oracle_cases)
    # the oracle runs (FP64, one host core each) start before any GPU work
    pool = mp.get_context("spawn").Pool(max(1, min(a.oracle_workers, n_or)))
    t_or = time.perf_counter()
    pending = pool.map_async(oracle_run, [(w, a.oracle_steps) for w in wt[:n_or]])

    import torch
    from paper_1801_04577_gb300 import clbm
    from paper_1801_04577_gb300 import surrogate as SG
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sid = stream.cuda_stream
    res = {"grid": G, "n_train": a.train, "n_test": a.test, "ra_range": [1e3, a.ra_max],
           "levels": a.levels, "base": a.base, "epochs": a.epochs, "batch": a.batch,
           "gen_tol": a.gen_tol, "tol": a.tol, "nu_tol": a.nu_tol, "ref_tol": a.ref_tol,
           "storage": "f32 deviations (batched solver)"}
    t_start = time.perf_counter()

    def finals(b, ws):
        """Two-step mean hot-wall Nusselt numbers and temperature fields of a batch."""
        nus, Ts = [], []
        for i, w in enumerate(ws):
            v = b.view(i)
            nus.append(two_step_nusselt(lambda: clbm.clbm_nusselt(v, 0, w.length, 1.0),
                                        lambda: clbm.clbm_step(v, 1)))
            Ts.append(b.moments(i)[3])
        return np.array(nus), Ts

    # 1. references: FP64 batched solve to ref_tol; FP64 from rest for oracle_steps steps
    b, conv_ref, _, _, t_ref = SG.solve(wt, a.ref_tol, 4 * a.horizon, 1000, precision="f64", stream=sid)
    nu_ref, T_ref = finals(b, wt)
    b.close()
    good = conv_ref > 0
    res["reference_converged"] = int(good.sum())
    res["reference_median_steps"] = float(np.median(conv_ref[good])) if good.any() else None
    res["reference_s"] = t_ref
    b = clbm.Batch(wt[:n_or], "f64", autotune=False, stream=sid)
    b.solve(0.0, a.oracle_steps, a.oracle_steps)
    nu_f64, T_f64 = finals(b, wt[:n_or])
    b.close()
    _log(f"references: {good.sum()}/{len(wt)} converged to {a.ref_tol:g} in {t_ref:.1f} s")

    # 2. the network: trained here, or loaded
    net = SG.make_net(G, base=a.base, levels=a.levels, max_batch=a.batch, seed=9, stream=sid)
    res["parameters"] = net.nparam
    if a.load_net:
        net.set_params(np.load(a.load_net))
        res["net"] = f"loaded from {os.path.basename(a.load_net)}"
    else:
        Ys, Xs, n_ok, t_gen = [], [], 0, 0.0
        ws_all = I.obstacle_cavities(a.train, G, ra_range=(1e3, a.ra_max))
        for s0 in range(0, a.train, a.gen_chunk):
            ws = ws_all[s0:s0 + a.gen_chunk]
            Y, conv, el = SG.generate(ws, a.gen_tol, a.gen_max_steps, check_every=1000, stream=sid)
            ok = conv > 0
            n_ok += int(ok.sum())
            t_gen += el
            Ys.append(Y[ok])
            Xs.append(SG.encode([w for w, k in zip(ws, ok) if k]))
            _log(f"data {s0 + len(ws)}/{a.train}: {n_ok} converged, {t_gen:.0f} s")
        res["train_converged"] = n_ok
        res["train_solve_s"] = t_gen
        X = torch.from_numpy(np.concatenate(Xs)).cuda()
        Yd = torch.from_numpy(np.concatenate(Ys)).cuda()
        M = X[:, 0].contiguous()
        del Xs, Ys
        t1 = time.perf_counter()
        losses = SG.train(net, X, Yd, M, epochs=a.epochs, batch=a.batch, lr=a.lr, lr_final=a.lr_final,
                          log=lambda m: _log(m) if m.split(":")[0].endswith("0") else None)
        torch.cuda.synchronize()
        res["train_s"] = time.perf_counter() - t1
        res["loss_first_last"] = [losses[0], losses[-1]]
        del X, Yd, M
        if a.save_net:
            np.save(a.save_net, net.get_params())

    # 3. rest and warm starts in chunks: steps until residual < tol and Nu within nu_tol, for good
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    y = SG.predict(net, wt)
    t_inf = time.perf_counter() - t_inf
    chunks = a.horizon // a.chunk
    for name, wl in (("rest", wt), ("warm", SG.warm_workloads(wt, y))):
        b = clbm.Batch(wl, "f32", autotune=True, stream=sid)
        pre = 0
        if name == "warm":
            b.solve(0.0, SG.WARM_PRESTEPS, SG.WARM_PRESTEPS)
            b.damp_period2()
            pre = SG.WARM_PRESTEPS
        ok_hist = np.zeros((chunks, len(wl)), bool)
        nu_hist = np.zeros((chunks, len(wl)))
        steps = pre
        for c in range(chunks):
            _, r, st = b.solve(0.0, a.chunk, a.chunk // 2)  # residual over the chunk's last half
            steps += st
            nu = np.array([two_step_nusselt(lambda v=b.view(i), w=w: clbm.clbm_nusselt(v, 0, w.length, 1.0),
                                            lambda v=b.view(i): clbm.clbm_step(v, 1))
                           for i, w in enumerate(wl)])
            steps += 1
            nu_hist[c] = nu
            ok_hist[c] = (r < a.tol) & (np.abs(nu - nu_ref) <= a.nu_tol * np.abs(nu_ref))
        # seconds per batched FP32 step of this batch, timed on a plain solve
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.solve(0.0, 10 * a.chunk, 10 * a.chunk)
        torch.cuda.synchronize()
        sps = (time.perf_counter() - t0) / (10 * a.chunk)
        b.close()
        settle = np.full(len(wl), np.inf)
        for j in range(len(wl)):
            bad = np.where(~ok_hist[:, j])[0]
            first = 0 if len(bad) == 0 else bad[-1] + 1
            if first < chunks:
                settle[j] = pre + (first + 1) * (a.chunk + 1)
        sel = good & np.isfinite(settle)
        res[name] = {
            "steady": int(np.isfinite(settle[good]).sum()), "of": int(good.sum()),
            "median_steps": float(np.median(settle[sel])) if sel.any() else None,
            "max_steps": float(np.max(settle[sel])) if sel.any() else None,
            "seconds_per_batch_step": sps,
            "batch_wall_s": float(np.max(settle[sel]) * sps + (t_inf if name == "warm" else 0.0))
            if sel.any() else None,
            "final_nu_rel_err_median": float(np.median(np.abs(nu_hist[-1][good] - nu_ref[good])
                                                       / np.abs(nu_ref[good]))),
        }
        res[name + "_settle_steps"] = [None if not np.isfinite(v) else int(v) for v in settle]
        _log(f"{name}: {res[name]}")
    both = good & np.isfinite(np.array([np.inf if v is None else v for v in res["rest_settle_steps"]])) & \
        np.isfinite(np.array([np.inf if v is None else v for v in res["warm_settle_steps"]]))
    rs = np.array([v or 0 for v in res["rest_settle_steps"]], float)
    ws_ = np.array([v or 0 for v in res["warm_settle_steps"]], float)
    res["judged_both"] = int(both.sum())
    res["warm_fewer_steps_fraction"] = float((ws_[both] < rs[both]).mean()) if both.any() else None
    res["inference_s"] = t_inf
    if res["rest"]["batch_wall_s"] and res["warm"]["batch_wall_s"]:
        res["speedup_wall"] = res["rest"]["batch_wall_s"] / res["warm"]["batch_wall_s"]

    # 4. the FP64 path against the oracle itself
    _log("waiting for the oracle")
    refs = pending.get()
    pool.close()
    res["oracle_s"] = time.perf_counter() - t_or
    nu_o = np.array([x[0] for x in refs])
    dT = [float(np.abs(T - x[1]).max() / np.abs(x[1]).max()) for T, x in zip(T_f64, refs)]
    res["oracle_check"] = {"cases": n_or, "steps": a.oracle_steps,
                           "nu_rel_diff_max": float(np.max(np.abs(nu_f64 - nu_o) / np.abs(nu_o))),
                           "T_rel_diff_max": float(np.max(dT))}
    res["total_s"] = time.perf_counter() - t_start
    net.close()
    line = {"metric": "time_to_steady_s", "value": res["warm"]["batch_wall_s"], "unit": "s",
            "higher_is_better": False, "baseline_rest_start_s": res["rest"]["batch_wall_s"],
            "data": "synthetic", "config": {"workload": f"warm_start_obstacle_cavities_g{G}"}, "study": res}
    print(json.dumps(line), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(line, fh, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
