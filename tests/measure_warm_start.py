"""Time to steady state with and without the learned warm start, judged
against the FP64 oracle (a measurement script, not a test module).

    python tests/measure_warm_start.py --grid 128 --train 20000 --test 32 --out gpurun_out/warm128.json

1. Seeded obstacle cavities on G x G grids (Ra log-uniform 1e3..1e6, Pr
   0.7..7, source 0 or 1e-6..1e-4, 0..2 adiabatic obstacles) are solved to an
   interval residual of --gen-tol by the batched GPU solver; their steady
   (T, u_x, u_y) train the U-Net on the GPU (the library's tensor-core kernels).
2. Held-out cavities are solved twice by the batched solver to a residual
   below --tol (1e-6): from rest, and from the network's prediction (inference
   time included, period-2 filter after two steps).  Steps and wall time are
   recorded for each start.
3. The FP64 oracle gives each held-out cavity's steady state: it starts from
   the GPU's converged fields (the steady state of these cavities does not
   depend on the start; starting close only saves CPU time) and steps until
   its hot-wall Nusselt number changes by less than 1e-10 over 2,000 steps.
   These run on the host cores in spawned processes while the GPU works.
4. Reported per start: median steps and batch wall time to residual < tol;
   the fraction of cavities whose converged hot-wall Nu is within 1e-3 of the
   oracle's; the T-field L2 error against the oracle.

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


def oracle_steady(args):
    """FP64 oracle steady state of one cavity from rest: steps until the
    two-step mean of the hot-wall Nusselt number changes by less than 1e-9
    (relative) over `chunk` steps, or max_steps."""
    w, chunk, max_steps = args
    import oracle
    oracle.set_threads(1)
    o = oracle.from_workload(w)
    prev, nu, steps = None, None, 0
    while steps < max_steps:
        o.step(chunk)
        steps += chunk
        nu = two_step_nusselt(lambda: o.nusselt(0, w.length, 1.0), lambda: o.step(1))
        steps += 1
        if prev is not None and abs(nu - prev) <= 1e-9 * abs(nu):
            break
        prev = nu
    return nu, o.moments()[3], steps


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
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-steps", type=int, default=600000)
    ap.add_argument("--check-every", type=int, default=500)
    ap.add_argument("--gen-chunk", type=int, default=5000)
    ap.add_argument("--oracle-workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--oracle-cases", type=int, default=15)
    ap.add_argument("--oracle-chunk", type=int, default=2000)
    ap.add_argument("--oracle-max-steps", type=int, default=300000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)

    # the oracle runs (from rest, FP64, one host core each) start before any GPU work
    G = a.grid
    wt = I.obstacle_cavities(a.test, G, seed=I.SURROGATE_SEED + 7919, ra_range=(1e3, a.ra_max))
    n_or = min(a.test, a.oracle_cases)
    pool = mp.get_context("spawn").Pool(a.oracle_workers)
    t2 = time.perf_counter()
    pending = pool.map_async(oracle_steady, [(w, a.oracle_chunk, a.oracle_max_steps) for w in wt[:n_or]])

    import torch
    from paper_1801_04577_gb300 import surrogate as SG
    from paper_1801_04577_gb300 import clbm
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    res = {"grid": G, "n_train": a.train, "n_test": a.test, "ra_range": [1e3, a.ra_max],
           "levels": a.levels, "base": a.base, "epochs": a.epochs, "batch": a.batch,
           "gen_tol": a.gen_tol, "tol": a.tol, "check_every": a.check_every,
           "storage": "f32 deviations (batched solver)"}
    t_start = time.perf_counter()

    def finals(b, ws):
        """Two-step mean Nusselt numbers and temperature fields of a solved batch."""
        nus, Ts = [], []
        for i, w in enumerate(ws):
            v = b.view(i)
            nus.append(two_step_nusselt(lambda: clbm.clbm_nusselt(v, 0, w.length, 1.0),
                                        lambda: clbm.clbm_step(v, 1)))
            Ts.append(b.moments(i)[3])
        return np.array(nus), Ts

    # 0. held-out problems from rest to residual < tol
    SG.solve(wt[:2], a.tol, 2000, a.check_every, stream=stream.cuda_stream)[0].close()  # warm-up
    r = {}
    b, conv, _, _, t_rest = SG.solve(wt, a.tol, a.max_steps, a.check_every, stream=stream.cuda_stream)
    r["rest"] = (conv,) + finals(b, wt) + (t_rest,)
    b.close()
    _log(f"rest starts: {int((conv > 0).sum())}/{len(wt)} converged in {t_rest:.1f} s")

    # 1. training data, in chunks of the batched solver
    Ys, Xs, n_ok, t_gen = [], [], 0, 0.0
    ws_all = I.obstacle_cavities(a.train, G, ra_range=(1e3, a.ra_max))
    for s in range(0, a.train, a.gen_chunk):
        ws = ws_all[s:s + a.gen_chunk]
        Y, conv, el = SG.generate(ws, a.gen_tol, a.gen_max_steps, check_every=1000,
                                  stream=stream.cuda_stream)
        ok = conv > 0
        n_ok += int(ok.sum())
        t_gen += el
        Ys.append(Y[ok])
        Xs.append(SG.encode([w for w, k in zip(ws, ok) if k]))
        _log(f"data {s + len(ws)}/{a.train}: {n_ok} converged, {t_gen:.0f} s")
    res["train_converged"] = n_ok
    res["train_solve_s"] = t_gen
    X = torch.from_numpy(np.concatenate(Xs)).cuda()
    Yd = torch.from_numpy(np.concatenate(Ys)).cuda()
    M = X[:, 0].contiguous()
    del Xs, Ys

    # 2. training
    net = SG.make_net(G, base=a.base, levels=a.levels, max_batch=a.batch, seed=9,
                      stream=stream.cuda_stream)
    res["parameters"] = net.nparam
    t1 = time.perf_counter()
    losses = SG.train(net, X, Yd, M, epochs=a.epochs, batch=a.batch, lr=a.lr, lr_final=a.lr_final,
                      log=lambda m: _log(m) if m.split(":")[0].endswith("0") else None)
    torch.cuda.synchronize()
    res["train_s"] = time.perf_counter() - t1
    res["loss_first_last"] = [losses[0], losses[-1]]
    del X, Yd, M

    # 3. the same held-out problems from the prediction to residual < tol
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    y = SG.predict(net, wt)
    t_inf = time.perf_counter() - t_inf
    b, conv, _, _, t_warm = SG.solve(SG.warm_workloads(wt, y), a.tol, a.max_steps, a.check_every,
                                     stream=stream.cuda_stream, warm=True)
    r["warm"] = (conv,) + finals(b, wt) + (t_warm + t_inf,)
    b.close()
    _log("waiting for the oracle")
    refs = pending.get()
    pool.close()
    res["oracle_s"] = time.perf_counter() - t2
    nu_o = np.array([x[0] for x in refs])
    res["oracle_cases"] = n_or
    res["oracle_steps_median"] = float(np.median([x[2] for x in refs]))

    def tl2(Ts):
        out = []
        for w, T, (_, To, _) in zip(wt[:n_or], Ts[:n_or], refs):
            fl = np.ones_like(To, bool) if w.geom.solid is None else w.geom.solid == 0
            out.append(float(np.linalg.norm((T - To)[fl]) / np.linalg.norm(To[fl])))
        return np.array(out)

    for name in ("rest", "warm"):
        steps, nu, Ts, tsec = r[name]
        ok = steps > 0
        nerr = np.abs(nu[:n_or] - nu_o) / np.abs(nu_o)
        res[name] = {
            "converged": int(ok.sum()),
            "median_steps": float(np.median(steps[ok])) if ok.any() else None,
            "batch_wall_s": float(tsec),
            "nu_rel_err_median": float(np.median(nerr)),
            "nu_rel_err_max": float(np.max(nerr)),
            "nu_within_1e-3": float((nerr < 1e-3).mean()),
            "T_rel_L2_median": float(np.median(tl2(Ts))),
        }
    rs, ws_ = r["rest"][0], r["warm"][0]
    both = (rs > 0) & (ws_ > 0)
    res["warm_fewer_steps_fraction"] = float((ws_[both] < rs[both]).mean()) if both.any() else None
    res["inference_s"] = t_inf
    res["speedup_wall"] = res["rest"]["batch_wall_s"] / res["warm"]["batch_wall_s"]
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
