"""The y-slab decomposition on one GPU: k slabs of a lattice (each with a
ghost row on each side, halos copied after every step) against the single
lattice.  The per-node arithmetic is the same and every pulled value is the
same stored number, so the fields must agree bit for bit, in every storage
format (stochastic rounding included: its bits are keyed by the global node);
the reductions, summed per slab and then across slabs, agree to rounding."""
import numpy as np
import pytest

from paper_1801_04577_gb300 import clbm
from paper_1801_04577_gb300 import inputs as I
from paper_1801_04577_gb300 import slabs

pytestmark = pytest.mark.gpu


def case(name):
    if name == "rb":
        w = I.rayleigh_benard(300, 70, Ra=1e5, Q=1e-4, noise=1e-2)
        w.init = I.random_fields(300, 70, seed=31, amp=0.02)
        return w, 120, [2, 3]
    if name == "periodic_box":
        return I.periodic_box(133, 37), 100, [1, 2, 4]
    if name == "obstacle":  # obstacle rows 6..10 of 19 straddle the seams
        return I.obstacle_channel(), 150, [2, 3]
    if name == "annulus":  # curved links crossing the seams
        return I.annulus(96, 2.6, Ra=1e4), 150, [2, 3]
    if name == "viscous":
        w = I.natural_convection_cavity(48, 1e5)
        w.params.viscous_heating = 1
        return w, 150, [2]
    if name == "one_row_slabs":
        return I.poiseuille_channel(4, 0.1, 1e-4, nx=40), 60, [4]
    raise ValueError(name)


CASES = [("rb", "f64", 0), ("rb", "f32", 0), ("rb", "bf16", 1), ("rb", "f16", 0),
         ("periodic_box", "f32", 0), ("periodic_box", "f64", 0), ("obstacle", "f64", 0),
         ("obstacle", "f32", 0), ("annulus", "f32", 0), ("viscous", "f64", 0),
         ("one_row_slabs", "f32", 0)]


@pytest.mark.parametrize("name,precision,rounding", CASES)
def test_slabs_reproduce_the_single_lattice_bit_for_bit(name, precision, rounding):
    w, steps, parts_list = case(name)
    ref = clbm.from_workload(w, precision, rounding=rounding)
    ref.step(steps)
    want = ref.moments()
    r_ref = ref.residual()
    tot_ref = ref.totals()
    for parts in parts_list:
        g = slabs.SlabGroup(w, parts, precision, rounding)
        g.step(steps)
        got = g.moments()
        for k, (a, b) in enumerate(zip(got, want)):
            np.testing.assert_array_equal(a, b, err_msg=f"{name} {precision} {parts} slabs field {k}")
        assert g.residual() == pytest.approx(r_ref, rel=1e-12)
        np.testing.assert_allclose(g.totals(), tot_ref, rtol=1e-12, atol=1e-9)
        for which in range(4):
            side_periodic = w.params.periodic_x if which < 2 else w.params.periodic_y
            if side_periodic:
                continue
            try:
                nu_ref = ref.nusselt(which, w.length, w.dT)
            except clbm.ClbmError as e:  # a side without fluid nodes (the annulus box)
                assert e.status == clbm.CLBM_EINVAL
                with pytest.raises(clbm.ClbmError):
                    g.nusselt(which, w.length, w.dT)
                continue
            assert g.nusselt(which, w.length, w.dT) == pytest.approx(nu_ref, rel=1e-12, abs=1e-14)
        g.close()
    ref.close()


def test_slab_listed_link_nusselt_matches():
    """Nusselt numbers of listed (curved) links summed over slabs."""
    w = I.annulus(64, 2.6, Ra=1e4)
    ref = clbm.from_workload(w, "f64")
    ref.step(200)
    g = slabs.SlabGroup(w, 3, "f64")
    g.step(200)
    for which in (4, 5):
        assert g.nusselt(which, w.length, w.dT) == pytest.approx(ref.nusselt(which, w.length, w.dT),
                                                                 rel=1e-12)


def test_uneven_slab_bounds():
    """Slabs of 1, 30 and 39 rows (any partition is valid)."""
    w = I.rayleigh_benard(130, 70, Ra=1e5, Q=1e-4, noise=1e-2)
    ref = clbm.from_workload(w, "f32")
    ref.step(80)
    g = slabs.SlabGroup(w, 3, "f32", bounds=[(0, 1), (1, 30), (31, 39)])
    g.step(80)
    for a, b in zip(g.moments(), ref.moments()):
        np.testing.assert_array_equal(a, b)


def test_one_slab_per_process_path_on_one_rank():
    """DistSlab with one rank on a periodic lattice: the packed rows go
    through slabs.exchange (world = 1: the slab is its own neighbour) and
    clbm_halo_pack / clbm_halo_unpack; equal to the single lattice."""
    w = I.periodic_box(133, 37)
    ref = clbm.from_workload(w, "f32")
    ref.step(50)
    d = slabs.DistSlab(w, "f32")
    d.step(50)
    for a, b in zip(d.slab.moments(), ref.moments()):
        np.testing.assert_array_equal(a, b)
    assert d.residual() == pytest.approx(ref.residual(), rel=1e-12)
    d.close()


def test_slab_rejects_bad_bounds_and_thin_offset_links():
    w = I.rayleigh_benard(64, 16)
    p = clbm.make_params(w.params, "f32")
    for y0, rows in ((-1, 4), (0, 0), (10, 7)):
        with pytest.raises(clbm.ClbmError) as ei:
            clbm.clbm_create_slab(p, y0, rows)
        assert ei.value.status == clbm.CLBM_EINVAL
    # a Dirichlet wall at q < 1/2 reads T two nodes into the fluid: a one-row
    # slab next to it cannot hold that node
    w = I.offset_channel(10, 0.05, 0.1, 0.1, 0.1, 1e-4, Q=1e-3)
    with pytest.raises(clbm.ClbmError) as ei:
        clbm.Slab(w.params, 1, 1, w.geom, "f32")
    assert ei.value.status == clbm.CLBM_EINVAL


def _dist_worker(rank, world, port, name, precision, steps, q):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w, _, _ = case(name)
        d = slabs.DistSlab(w, precision)
        d.step(steps)
        m = [np.array(a) for a in d.slab.moments()]
        r = d.residual()
        tot = d.totals()
        q.put((rank, d.y0, m, r, tot))
        dist.barrier()
        d.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,precision,world", [("rb", "f32", 2), ("periodic_box", "f64", 2),
                                                  ("obstacle", "f32", 3)])
def test_one_slab_per_process_on_one_gpu(name, precision, world):
    """The multi-process path end to end on one GPU: `world` gloo ranks, each
    holding one slab on cuda:0, pack their edge rows on the device, exchange
    them through host memory (gloo), unpack them into the ghost rows, and add
    their reduction sums with an all-reduce.  No kernel of one rank waits on
    another's: each host completes the exchange before its next launch.  The
    fields equal the single lattice bit for bit; residual and conservation
    sums to 1e-12."""
    import socket
    import torch.multiprocessing as mp
    w, _, _ = case(name)
    steps = 60
    ref = clbm.from_workload(w, precision)
    ref.step(steps)
    want = ref.moments()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dist_worker, args=(r, world, port, name, precision, steps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[1])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = [np.concatenate([o[2][k] for o in out], axis=0) for k in range(4)]
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    for o in out:
        assert o[3] == pytest.approx(ref.residual(), rel=1e-12)
        np.testing.assert_allclose(o[4], ref.totals(), rtol=1e-12, atol=1e-9)
