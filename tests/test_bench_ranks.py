"""Host logic of the multi-process benchmark path on CPU: two gloo ranks (one
y-slab each); the job time is the slowest rank's and the throughput counts
every rank's nodes (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el, mlups = bench.combine_ranks(10.0 * (rank + 1), nodes=1000, steps=50)
    q.put((rank, el, mlups))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, el, mlups in out:
        assert el == pytest.approx(20.0)                      # slowest rank
        assert mlups == pytest.approx(2 * 1000 * 50 / 20e-3 / 1e6)


def test_single_process_has_no_collective():
    import bench
    el, mlups = bench.combine_ranks(5.0, nodes=100, steps=10)
    assert el == 5.0 and mlups == pytest.approx(100 * 10 / 5e-3 / 1e6)


def test_launch_count_claim_follows_the_launch_scheme():
    """gpu_launches: one fused launch per step on box and masked lattices
    alike; a run of two or more steps adds one counter-setting kernel and one
    step-counter kernel per replayed graph (graphs of 32, 16, ..., 2 steps)."""
    import bench
    rb = bench.workload("rb256")
    an = bench.workload("annulus2048")
    assert bench.box_lattice(rb) and not bench.box_lattice(an)
    assert "step_fused_kernel" in bench.step_kernel_name(an)
    assert bench.step_launches(rb, 1) == 1
    assert bench.step_launches(rb, 3) == 3 + 1 + 1          # graph of 2 + one single step
    assert bench.step_launches(rb, 20) == 20 + 1 + 2        # graphs of 16 and 4
    assert bench.step_launches(rb, 64) == 64 + 1 + 2        # two graphs of 32
    assert bench.step_launches(an, 100) == 100 + 1 + 4     # 3 x 32 + 4


def test_reference_arm_names_the_same_workload():
    """Both bench arms spell the benchmark workload the same way."""
    import bench
    from paper_1801_04577_gb300 import inputs as I
    name = I.rayleigh_benard(64, 32).name.replace("64x32", "4096x2048")
    assert name == f"rayleigh_benard_4096x2048_Ra{1e6:g}"


def test_unet_flop_count_by_hand():
    """Two-level U-Net on 4^2, one sample: forward GEMM flops counted layer by
    layer (2 x pixels x co x ci x k^2) = 8128; a training step is three times
    that minus the first layer's input gradient (576)."""
    import bench
    assert bench.conv_flops_per_train_step(4, 1, 1, 2, 2, 1) == 3 * 8128 - 576
