#!/usr/bin/env python
"""Throughput benchmark of the fused cascaded thermal LBM step on GB300.

Workload (default): Rayleigh-Benard cell 4096 x 2048, periodic in x, bottom
T = 1, top T = 0, Ra = 1e6, Pr = 0.71, U = 0.1, uniform heat source Q = 1e-5,
initial T linear plus seeded noise of amplitude 1e-3, FP32 storage and
collision.  One benchmark step is one lattice time step (one launch of the
fused collide-and-stream kernel over all nodes).  Metric: MLUPS (million
fluid-node updates per second), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun with N > 1 the Rayleigh-Benard cell has N times the rows and
is split into y-slabs, one 4096 x 2048 slab per rank, whose edge rows are
exchanged with the neighbouring ranks after every step (NCCL point-to-point;
weak scaling); the timing is combined (max over ranks).  --slabs k splits the
one-GPU lattice into k slabs on that GPU (decomposition overhead).
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample lattice of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1801_04577_gb300 import inputs as I  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# FP64 storage and collision are bound by the FP64 pipe, not by HBM.  FP64 operations per
# lattice update of step_fused_kernel<double>, counted with ncu on the 2048 x 1024
# Rayleigh-Benard lattice (sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on: 165.9 M
# DFMA, 140.7 M DADD, 51.5 M DMUL per launch of 2,097,152 nodes; an FMA counts two): 249.8.
FP64_FLOP_PER_LU = 249.8
# FP64 peak of the GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
ELEM_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
DTYPE = {"f64": "f64", "f32": "f32", "f16": "f16-storage/f32-compute", "bf16": "bf16-storage/f32-compute"}

# DRAM traffic per launch of the step kernel measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by storage type and
# workload, valid only for the kernel source whose SHA-256 prefix is stored.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (1 pass) on the full 4096 x 2048
    # lattice, three launches of step_fused_kernel each: FP32 479.30-479.34 MB read + 415.3-418.8 MB
    # written; FP16 243.0-243.1 MB read + 189.3-191.8 MB written (the rest of the written lines
    # is still dirty in L2 when the launch ends).
    "f32:rb4096": {"bytes_per_launch": 896.1e6, "kernel_hash": "fc7666131524faae"},
    "f16:rb4096": {"bytes_per_launch": 433.4e6, "kernel_hash": "fc7666131524faae"},
}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("clbm_kernels.cuh", "clbm_internal.h"):
        with open(os.path.join(ROOT, "paper_1801_04577_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def workload(name: str, ranks: int = 1):
    """The named workload; with ranks > 1 the Rayleigh-Benard cell has ranks
    times the rows (one 4096 x 2048 slab per rank)."""
    if name == "rb4096":
        return I.rayleigh_benard(4096, 2048 * ranks)
    if ranks > 1:
        raise SystemExit(f"bench.py: workload {name} runs on one GPU only")
    if name == "rb256":
        return I.rayleigh_benard(256, 128)
    if name == "rb2048":
        return I.rayleigh_benard(2048, 1024)
    if name == "cavity64":
        return I.natural_convection_cavity(64, 1e4)
    if name == "annulus2048":
        return I.annulus(2048, 2.6, Ra=1e5)
    if name == "annulus2048i":  # walls at each link's crossing fraction (interpolated)
        return I.annulus(2048, 2.6, Ra=1e5, interpolated=True)
    raise SystemExit(f"unknown workload {name}")


def workload_config(w, name, precision):
    cfg = {"workload": w.name + f"_{precision}", "nx": w.params.nx, "ny": w.params.ny,
           "fluid_nodes": I.fluid_count(w), "storage": f"{precision} deviations from rest state",
           "bytes_per_lattice_update": 28 * ELEM_BYTES[precision],
           "l2": "no flush: inputs larger than L2 (two ping-pong buffers of "
                 f"{14 * w.params.nx * w.params.ny * ELEM_BYTES[precision] / 1e6:.0f} MB each)"}
    return cfg


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def device_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            pass
    return local_rank


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_rb_sample(nx: int, ny: int):
    w = I.rayleigh_benard(nx, ny)
    import oracle
    return w, oracle.from_workload(w), oracle.threads()


def time_oracle(budget_s: float = 12.0, nx: int = 2048, ny: int = 1024):
    """MLUPS of the FP64 oracle on an RB sample lattice: steps until the budget."""
    w, o, cores = oracle_rb_sample(nx, ny)
    o.step(1)  # warm-up
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 200:
            break
    out = {"value": nx * ny * n / el / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle, Rayleigh-Benard {nx}x{ny} (same parameters as the workload), "
                     f"{n} steps after 1 warm-up step, {el:.1f} s"}
    # the same program on one core, on a smaller sample of the workload (about 3 s)
    import oracle
    del o
    w1, o1, _ = oracle_rb_sample(512, 256)
    oracle.set_threads(1)
    try:
        o1.step(1)
        t0, n1 = time.perf_counter(), 0
        while n1 < 100 and time.perf_counter() - t0 < 3.0:
            o1.step(1)
            n1 += 1
        el1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    out["single_thread"] = {"value": 512 * 256 * n1 / el1 / 1e6, "unit": "MLUPS",
                            "sample": f"512x256, {n1} steps, {el1:.1f} s, 1 thread"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    # size the sample so that warmup + steps finish within about two minutes
    budget = 120.0
    w_probe, o_probe, cores = oracle_rb_sample(256, 128)
    o_probe.step(1)
    t0 = time.perf_counter()
    o_probe.step(3)
    rate = 256 * 128 * 3 / (time.perf_counter() - t0)  # node updates per second
    total = max(1, args.steps + args.warmup)
    nodes = max(64 * 32, min(4096 * 2048, int(rate * budget / total)))
    ny = max(32, int((nodes / 2) ** 0.5))
    nx = 2 * ny
    w = I.rayleigh_benard(nx, ny)
    o = oracle.from_workload(w)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    value = nx * ny * args.steps / el / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rayleigh_benard_4096x2048_Ra{1e6:g}_{args.precision}",
                       "sample": f"{nx}x{ny} lattice of the same workload"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"FP64 oracle, Rayleigh-Benard {nx}x{ny}, {args.steps} steps "
                                       f"after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def combine_ranks(elapsed_ms: float, nodes: int, steps: int, device=None):
    """Whole-job throughput over the ranks (one y-slab each): the slowest
    rank's time (max over ranks) bounds the job; every rank advanced `nodes`
    nodes for `steps` steps.  Returns (max elapsed ms, MLUPS over all ranks)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el = float(t.item())
    return el, world * nodes * steps / (el * 1e-3) / 1e6


def box_lattice(w) -> bool:
    """No solid mask and no listed links (a plain box lattice)."""
    return w.geom.solid is None and len(w.geom.link_node) == 0


def step_kernel_name(w) -> str:
    """Box and masked lattices alike take one fused launch per step: the
    listed boundary nodes in the first blocks, the interior warp tiles in the
    rest (masked lattices skip tiles without fluid and leave flagged nodes to
    the boundary blocks)."""
    if box_lattice(w):
        return "step_fused_kernel (interior tiles + boundary nodes, one launch per step)"
    return "step_fused_kernel<masked> (tile classes + listed boundary nodes, one launch per step)"


def step_launches(w, steps: int, graph_levels: int = 5) -> int:
    """Kernels that clbm_step(steps) launches: one fused launch per step.  A
    run of two or more steps replays captured graphs of 32, 16, ..., 2 steps
    (the binary digits of `steps`; a last odd step is launched on its own),
    each ending with one step-counter kernel, after one kernel that sets the
    counter."""
    n = steps
    if steps >= 2:
        top = 1 << graph_levels
        graphs = steps // top + bin((steps % top) >> 1).count("1")
        n += 1 + graphs
    return n


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_1801_04577_gb300 import clbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1801_04577_gb300 import slabs

    # With N > 1 ranks the lattice is split into y-slabs, one per rank (weak
    # scaling: the whole lattice has N times the rows of the one-GPU workload);
    # --slabs k > 1 splits the one-GPU lattice into k slabs on this GPU.
    mode = "dist" if world > 1 else ("group" if args.slabs > 1 else "single")
    w = workload(args.workload, world if mode == "dist" else 1)
    p = w.params
    nodes = I.fluid_count(w) // (world if mode == "dist" else 1)  # per rank
    # a dedicated stream: the library launches on it and the events below are
    # recorded on it (torch's default stream has handle 0, which the library
    # would replace by a private stream)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    if mode == "dist":
        d = slabs.DistSlab(w, args.precision, args.rounding, stream=stream.cuda_stream)
        run_steps, residual = d.step, d.residual
    elif mode == "group":
        g = slabs.SlabGroup(w, args.slabs, args.precision, args.rounding, stream=stream.cuda_stream)
        run_steps, residual = g.step, g.residual
    else:
        s = clbm.from_workload(w, args.precision, stream=stream.cuda_stream, rounding=args.rounding)
        run_steps, residual = (lambda n: clbm.clbm_step(s.ctx, n)), s.residual
    # clocks are sampled from before the warm-up to the end of the timed region
    sampler = ClockSampler(device_index(local))
    sampler.start()
    run_steps(args.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    el_ms = e0.elapsed_time(e1)
    # the state must still be finite after the timed steps
    res = residual()

    el_ms, value = combine_ranks(el_ms, nodes, args.steps, dev)

    # end to end through the public API: host fields in, solve, host fields out
    e2e = None
    if not args.no_e2e and mode != "single":
        rows = d.rows if mode == "dist" else p.ny
        n = p.nx * rows
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if mode == "dist":
            d.slab.init(I.Fields(T=w.init.T))
            d.exchange()
            d.step(args.steps)
            out = d.slab.moments()
        else:
            for sl in g.slabs:
                sl.init(I.Fields(T=w.init.T))
            g.exchange()
            g.step(args.steps)
            out = g.moments()
        el2 = time.perf_counter() - t0
        el2_t = torch.tensor([el2], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(el2_t, op=dist.ReduceOp.MAX)
        el2 = float(el2_t.item())
        e2e = {"value": world * nodes * args.steps / el2 / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * n / args.steps, "d2h_bytes_per_step": 4 * 8 * n / args.steps,
               "note": f"per rank: slab initialisation from host T ({8 * n} B), halo exchange, "
                       f"{args.steps} steps with halo exchanges, moments (rho, ux, uy, T) to host "
                       f"({32 * n} B); bytes reported per lattice step"}
    if not args.no_e2e and mode == "single":
        n = p.nx * p.ny
        T_host = torch.from_numpy(w.init.T.astype("float64").ravel()).pin_memory()
        outs = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]

        def solve_from_host(steps):
            clbm.clbm_init_fields(s.ctx, None, None, None, T_host.data_ptr(), on_device=False)
            clbm.clbm_step(s.ctx, steps)
            clbm.clbm_moments(s.ctx, None, outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                              on_device=False)

        # warm-up of the same sequence with the warm-up step count (the library's
        # field scratch is allocated on first use of host fields)
        solve_from_host(args.warmup)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solve_from_host(args.steps)
        el2 = time.perf_counter() - t0
        # the fields that came back: finite, and the temperature within the walls' range
        Tb = outs[2].numpy()
        if not all(bool(torch.isfinite(o).all()) for o in outs) or not (
                -0.5 < float(Tb.min()) and float(Tb.max()) < 1.5):
            raise SystemExit("bench.py: the end-to-end run returned invalid fields")
        el2_t = torch.tensor([el2], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(el2_t, op=dist.ReduceOp.MAX)
        el2 = float(el2_t.item())
        e2e = {"value": world * nodes * args.steps / el2 / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * n / args.steps, "d2h_bytes_per_step": 3 * 8 * n / args.steps,
               "note": f"per run: one clbm_init_fields from pinned host T ({8 * n} B, read over "
                       f"the host link by the initialisation kernel), {args.steps} steps, one "
                       f"clbm_moments of ux, uy, T written by the kernel to pinned host "
                       f"({24 * n} B); bytes reported per lattice step; after one untimed run "
                       f"of the same sequence with the warm-up step count"}

    peak, peak_kind = measured_peak()
    bytes_lu = 28 * ELEM_BYTES[args.precision]
    per_launch_s = el_ms * 1e-3 / args.steps
    achieved = bytes_lu * nodes / per_launch_s / 1e9
    key = f"{args.precision}:{args.workload}"
    traffic = None
    rec = NCU_TRAFFIC.get(key)
    if rec and rec["kernel_hash"] == kernel_source_hash():
        traffic = rec["bytes_per_launch"]
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": dict(workload_config(w, args.workload, args.precision),
                           parallelism={"dist": f"yslab{world} (one slab per GPU, NCCL halo exchange)",
                                        "group": f"yslab{args.slabs} on one GPU (device halo copies)",
                                        "single": "single"}[mode]),
            "roofline": ({"bound": "alu", "achieved": FP64_FLOP_PER_LU * nodes / per_launch_s / 1e9,
                          "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                          "frac": FP64_FLOP_PER_LU * nodes / per_launch_s / 1e9 / FP64_PEAK_GFLOPS,
                          "traffic": traffic, "kernel": step_kernel_name(w),
                          "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clock x 2 x 2.07 GHz",
                          "flop_per_lattice_update": FP64_FLOP_PER_LU,
                          "hbm_frac": achieved / peak}
                         if args.precision == "f64" else
                         {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "traffic": traffic,
                          "kernel": step_kernel_name(w),
                          "peak_kind": peak_kind,
                          "algorithmic_bytes_per_launch": bytes_lu * nodes}),
            # slabs: one step launch per slab per step, plus (one process) one halo-copy launch
            "gpu_launches": step_launches(w, args.steps) if mode == "single" else args.steps * (
                args.slabs + 1 if mode == "group" else 1),
            "residual_after": res}
    if e2e is not None:
        line["e2e"] = e2e
    if clocks is not None:
        line["clocks"] = clocks
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle()
    if rank == 0:
        print(json.dumps(line), flush=True)
    {"dist": lambda: d.close(), "group": lambda: g.close(), "single": lambda: s.close()}[mode]()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched solve of the seeded 512-cavity set: --steps is the step cap."""
    import torch

    from paper_1801_04577_gb300 import clbm
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the library has no CPU path)")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ws = I.random_cavities(args.batch_size, hmax=args.batch_hmax)
    nodes = np.array([w.params.nx * w.params.ny for w in ws], dtype=np.int64)
    t0 = time.perf_counter()
    b = clbm.Batch(ws, args.precision, rounding=args.rounding, autotune=True, stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    # warm-up: one replay of the check interval (this also captures the solve graph,
    # which the timed solve reuses: same interval and tolerance)
    _, _, warm_steps = b.solve(args.tol, max(args.warmup, 1), check_every=args.check_every)
    torch.cuda.synchronize()
    sampler = ClockSampler(device_index(0))
    sampler.start()
    t0 = time.perf_counter()
    conv, res, steps = b.solve(args.tol, args.steps, check_every=args.check_every)
    el = time.perf_counter() - t0
    clocks = sampler.stop()
    per = np.where(conv > 0, conv, steps)
    per = np.where(conv == -2, 0, per)
    updates = float((nodes * per).sum())
    value = updates / el / 1e6
    peak, peak_kind = measured_peak()
    bytes_lu = 28 * ELEM_BYTES[args.precision]
    widths = [b.tile_width(i) for i in range(len(ws))]
    K = (args.check_every + 1) // 2 * 2
    replays = -(-int(steps) // K)
    # per step: one interior launch per tile-width group + the boundary launch;
    # per replay: residual (2), update, scan, tile rebuild
    launches = int(steps) * (len(set(widths)) + 1) + replays * 5
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1,
            "steps": int(steps), "warmup": int(warm_steps), "ms_per_step": el / max(steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": f"batch_{len(ws)}_random_cavities_h32-{args.batch_hmax}_{args.precision}"
                                   + ("_sr" if args.rounding else ""),
                       "total_nodes": int(nodes.sum()), "tol": args.tol, "step_cap": args.steps,
                       "check_every": args.check_every, "rounding": args.rounding},
            "roofline": {"bound": "hbm", "achieved": bytes_lu * updates / el / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bytes_lu * updates / el / 1e9 / peak,
                         "traffic": None, "kernel": "clbm::batch_step_kernel (whole solve)",
                         "peak_kind": peak_kind},
            "batch": {"converged": int((conv > 0).sum()), "converged_fraction": float((conv > 0).mean()),
                      "diverged": int((conv == -2).sum()),
                      "time_to_solution_s": el if (conv > 0).all() else None,
                      "not_converged": int((conv == -1).sum()),
                      "median_steps_converged": float(np.median(conv[conv > 0])) if (conv > 0).any() else None,
                      "residual_quantiles_10_50_90": [float(v) for v in np.quantile(
                          res[np.isfinite(res)], [0.1, 0.5, 0.9])] if np.isfinite(res).any() else None,
                      "create_s": t_create, "solve_s": el,
                      "tile_widths": {str(k): widths.count(k) for k in (32, 64, 128)}},
            "gpu_launches": launches}
    if clocks is not None:
        line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def conv_flops_per_train_step(G, cin, cout, base, levels, batch):
    """Multiply-adds x 2 of every convolution GEMM in one training step: the
    forward pass, the weight gradients and the input gradients (none for the
    first layer, whose input is data)."""
    from paper_1801_04577_gb300.net import layer_shapes
    shapes = layer_shapes(G, cin, cout, base, levels)
    # resolution of each layer, in layer order (encoder, bottleneck, decoder, head)
    res = []
    for l in range(levels - 1):
        res += [G >> l, G >> l]
    res += [G >> (levels - 1)] * 2
    for l in range(levels - 2, -1, -1):
        res += [G >> l, G >> l]
    res.append(G)
    total = 0.0
    for li, ((ci, co, k), h) in enumerate(zip(shapes, res)):
        f = 2.0 * batch * h * h * co * ci * k * k
        total += f * (2 if li == 0 else 3)
    return total


def conv_bytes_per_train_step(G, cin, cout, base, levels, batch, elem_bytes=4):
    """Algorithmic DRAM bytes of the convolution passes of one training step:
    each pass reads its input activations and writes its output once (FP32
    activations); the weight gradients read the layer input and the output
    gradient.  The weights themselves are small beside the activations."""
    from paper_1801_04577_gb300.net import layer_shapes
    shapes = layer_shapes(G, cin, cout, base, levels)
    res = []
    for l in range(levels - 1):
        res += [G >> l, G >> l]
    res += [G >> (levels - 1)] * 2
    for l in range(levels - 2, -1, -1):
        res += [G >> l, G >> l]
    res.append(G)
    total = 0.0
    for li, ((ci, co, k), h) in enumerate(zip(shapes, res)):
        total += (ci + co) * batch * h * h * elem_bytes * (2 if li == 0 else 3)
    return total


def conv_roofline_ms(G, cin, cout, base, levels, batch, tflops, gbs):
    """Lower bound on a training step's convolution time: every pass at the
    larger of its tensor-core time (flops at the BF16 peak) and its DRAM time
    (its activation bytes at the copy bandwidth).  At these widths (24-192
    channels) most passes are memory-bound: 2 x 9 ci x co flops per (ci + co)
    x 4 bytes is below the machine balance of the tensor cores."""
    from paper_1801_04577_gb300.net import layer_shapes
    shapes = layer_shapes(G, cin, cout, base, levels)
    res = []
    for l in range(levels - 1):
        res += [G >> l, G >> l]
    res += [G >> (levels - 1)] * 2
    for l in range(levels - 2, -1, -1):
        res += [G >> l, G >> l]
    res.append(G)
    t = 0.0
    for li, ((ci, co, k), h) in enumerate(zip(shapes, res)):
        f = 2.0 * batch * h * h * co * ci * k * k
        b = (ci + co) * batch * h * h * 4
        t += max(f / (tflops * 1e12), b / (gbs * 1e9)) * (2 if li == 0 else 3)
    return t * 1e3


def run_unet(args):
    """Training steps of the warm-start U-Net on the tensor cores (default: 64^2
    grid, widths 24..192, 1.1 M parameters, batch 32; --net-grid 128 gives the
    same network on 128^2 grids)."""
    import torch

    from paper_1801_04577_gb300.net import Net
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the library has no CPU path)")
    G, cin, cout, base, levels, B = args.net_grid, 5, 3, args.net_base, args.net_levels, args.net_batch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    net = Net(G, cin, cout, base, levels, B, seed=3, stream=stream.cuda_stream, math=args.net_math)
    r = I.splitmix64_uniform(1801045773, B * (cin + cout + 1) * G * G)
    o1, o2 = B * cin * G * G, B * (cin + cout) * G * G
    x = torch.from_numpy((2 * r[:o1] - 1).reshape(B, cin, G, G).astype(np.float32)).cuda()
    t = torch.from_numpy((2 * r[o1:o2] - 1).reshape(B, cout, G, G).astype(np.float32)).cuda()
    m = torch.from_numpy((r[o2:] > 0.25).reshape(B, G, G).astype(np.float32)).cuda()
    for _ in range(args.warmup):
        net.train_step(x, t, m, 1e-3)
    torch.cuda.synchronize()
    sampler = ClockSampler(device_index(0))
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        loss = net.train_step(x, t, m, 1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    y = torch.empty((B, cout, G, G), dtype=torch.float32, device="cuda")
    net.forward(x, y)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(20):
        net.forward(x, y)
    f1.record(stream)
    torch.cuda.synchronize()
    flops = conv_flops_per_train_step(G, cin, cout, base, levels, B)
    nbytes = conv_bytes_per_train_step(G, cin, cout, base, levels, B)
    achieved = flops / (ms * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured bf16 burst"
    except Exception:
        peak, kind = 1900.0, "fallback bf16 burst"
    hbm, hbm_kind = measured_peak()
    roof_ms = conv_roofline_ms(G, cin, cout, base, levels, B, peak, hbm)
    line = {"metric": "train_samples_per_s", "value": B * 1000.0 / ms, "unit": "samples/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands, fp32 accumulate" if args.net_math == "tensor" else "fp32",
            "data": "synthetic",
            "config": {"workload": f"unet_g{G}_b{base}_l{levels}_batch{B}_{args.net_math}",
                       "parameters": net.nparam, "forward_ms": f0.elapsed_time(f1) / 20,
                       "conv_gflop_per_step": flops / 1e9, "loss_last": loss,
                       "l2": f"activations of one batch (~{0.3 * (G / 64) ** 2:.1f} GB) larger than L2 in the first level"},
            # most convolution passes are memory-bound at these widths: the bound is
            # the activations' DRAM bytes; the tensor-core rate is reported beside it
            "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "traffic": None,
                         "kernel": "tc::gemm_kernel (all convolution passes of a training step)",
                         "peak_kind": hbm_kind, "algorithmic_bytes_per_step": nbytes,
                         "roofline_ms": roof_ms, "roofline_time_frac": roof_ms / ms,
                         "tensor_tflops": achieved, "tensor_peak": peak, "tensor_frac": achieved / peak,
                         "tensor_peak_kind": kind},
            "gpu_launches": None}
    if clocks is not None:
        line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=list(ELEM_BYTES), default="f32")
    ap.add_argument("--workload", default="rb4096")
    ap.add_argument("--rounding", type=int, choices=[0, 1], default=0,
                    help="16-bit storage: 0 = nearest even, 1 = stochastic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--slabs", type=int, default=1,
                    help="one GPU: split the lattice into this many y-slabs (halo copies each step)")
    ap.add_argument("--batch-size", type=int, default=512)
    ap.add_argument("--batch-hmax", type=int, default=512,
                    help="batch512: largest cavity side (sides drawn from 32..hmax)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--net-batch", type=int, default=32)
    ap.add_argument("--net-grid", type=int, default=64)
    ap.add_argument("--net-base", type=int, default=24)
    ap.add_argument("--net-levels", type=int, default=4)
    ap.add_argument("--net-math", choices=["tensor", "fp32"], default="tensor")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("bench.py: at least 3 warm-up steps are required")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "unet64":
        return run_unet(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
