"""The y-slab decomposition's host logic on CPU, with the FP64 oracle as the
per-slab solver.

Each gloo rank holds rows [y0, y0 + rows) of a lattice as an oracle lattice
of its own rows plus a ghost row on each side that is not a box wall (the
rows of the neighbouring slabs, cut from the same description).  After every
step the ranks exchange their first and last own rows -- the oracle's
pre-collision distributions, all 14 -- through ``slabs.exchange``, the same
function the GPU slabs use with NCCL.  Because the step at a node reads only
its neighbours' populations and the temperature one node further along a wall
link (Eq. 11, 21, 27-28), the slabs must reproduce the single-domain oracle
bit for bit.  A wrong neighbour, a swapped send, a missing periodic wrap or a
stale ghost row breaks that equality.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1801_04577_gb300 import inputs as I  # noqa: E402
from paper_1801_04577_gb300 import slabs  # noqa: E402


def test_partition_covers_the_rows_once():
    for ny, parts in ((10, 3), (2048, 8), (7, 7), (19, 2)):
        b = slabs.partition(ny, parts)
        assert len(b) == parts
        assert b[0][0] == 0 and sum(r for _, r in b) == ny
        assert all(b[k][0] + b[k][1] == b[k + 1][0] for k in range(parts - 1))
        assert max(r for _, r in b) - min(r for _, r in b) <= 1
    with pytest.raises(ValueError):
        slabs.partition(3, 4)


def test_neighbours_walled_and_periodic():
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 3, True) == (2, 1)
    assert slabs.neighbours(2, 3, True) == (1, 0)
    assert slabs.neighbours(0, 1, True) == (0, 0)
    assert slabs.neighbours(0, 1, False) == (None, None)


class OracleSlab:
    """Rows [y0, y0 + rows) of workload w in the FP64 oracle, stored with one
    ghost row on each side that is not a box wall."""

    def __init__(self, w, y0, rows):
        import oracle
        p, g = w.params, w.geom
        NY, nx = p.ny, p.nx
        periodic = bool(p.periodic_y)
        self.lo = 1 if (periodic or y0 > 0) else 0
        self.hi = 1 if (periodic or y0 + rows < NY) else 0
        self.rows, self.nx = rows, nx
        ext = rows + self.lo + self.hi
        gmap = [(y0 - self.lo + r) % NY for r in range(ext)]
        ep = I.Params(**{**p.__dict__, "ny": ext, "periodic_y": 0})
        tbc = list(g.tbc) + [I.dirichlet(p.T0)]  # stand-in condition beyond a ghost row
        dummy = len(tbc) - 1
        side = list(g.side_tbc)
        side[2] = dummy if self.lo else g.side_tbc[2]
        side[3] = dummy if self.hi else g.side_tbc[3]
        solid = None if g.solid is None else np.ascontiguousarray(g.solid[gmap])
        nodes, dirs, nes, tbcs, qs = [], [], [], [], []
        lq = g.link_q_or_half()
        for k in range(g.n_links):
            gy, x = divmod(int(g.link_node[k]), nx)
            for r, gr in enumerate(gmap):
                if gr == gy:
                    nodes.append(r * nx + x); dirs.append(int(g.link_dir[k]))
                    nes.append(float(g.link_ne[k])); tbcs.append(int(g.link_tbc[k])); qs.append(float(lq[k]))
        eg = I.Geometry(tbc=tbc, side_tbc=tuple(side), solid=solid,
                        link_node=np.asarray(nodes, np.int32), link_dir=np.asarray(dirs, np.int32),
                        link_ne=np.asarray(nes, np.float64), link_tbc=np.asarray(tbcs, np.int32),
                        link_q=np.asarray(qs, np.float64) if g.link_q is not None else None)
        shape = (NY, nx)
        init = I.Fields(*[None if a is None else np.ascontiguousarray(np.broadcast_to(a, shape)[gmap])
                          for a in (w.init.rho, w.init.ux, w.init.uy, w.init.T)])
        self.o = oracle.Oracle(ep, eg, init)

    def edge(self, side):
        f, g = self.o.dfs()
        r = self.lo if side == 0 else self.lo + self.rows - 1
        return torch.from_numpy(np.concatenate([f[r].ravel(), g[r].ravel()]))

    def set_ghost(self, side, t):
        f, g = self.o.dfs()
        r = 0 if side == 0 else self.lo + self.rows
        v = t.numpy()
        f[r] = v[:9 * self.nx].reshape(self.nx, 9)
        g[r] = v[9 * self.nx:].reshape(self.nx, 5)
        self.o.set_dfs(f, g)

    def own_moments(self):
        return tuple(m[self.lo:self.lo + self.rows] for m in self.o.moments())


def _exchange(sl, rank, world, periodic):
    n = 14 * sl.nx
    send_lo, send_hi = sl.edge(0), sl.edge(1)
    recv_lo, recv_hi = torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)
    slabs.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic)
    below, above = slabs.neighbours(rank, world, periodic)
    if below is not None:
        sl.set_ghost(0, recv_lo)
    if above is not None:
        sl.set_ghost(1, recv_hi)


def make_case(name):
    if name == "rb_walled":
        return I.rayleigh_benard(40, 26, Ra=1e5, Q=1e-4, noise=1e-2), 60
    if name == "periodic_box":
        return I.periodic_box(24, 21), 60
    if name == "obstacle":  # the obstacle's rows straddle the slab seams
        return I.obstacle_channel(), 60
    if name == "viscous_cavity":
        w = I.natural_convection_cavity(20, 1e5)
        w.params.viscous_heating = 1
        return w, 40
    raise ValueError(name)


def _worker(rank, world, port, name, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, steps = make_case(name)
        y0, rows = slabs.partition(w.params.ny, world)[rank]
        sl = OracleSlab(w, y0, rows)
        periodic = bool(w.params.periodic_y)
        _exchange(sl, rank, world, periodic)
        for _ in range(steps):
            sl.o.step(1)
            _exchange(sl, rank, world, periodic)
        q.put((rank, y0, [np.array(m) for m in sl.own_moments()]))
        # the reduction sums are added across ranks
        tot = slabs.allreduce_sums(np.array([rank + 1.0, 2.0 * rank]))
        q.put(("sum", rank, tot))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name,world", [("rb_walled", 2), ("rb_walled", 3), ("periodic_box", 2),
                                        ("periodic_box", 3), ("obstacle", 2), ("viscous_cavity", 2)])
def test_oracle_slabs_reproduce_the_single_domain_bit_for_bit(name, world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts, sums = {}, []
    for _ in range(2 * world):
        item = q.get(timeout=300)
        if item[0] == "sum":
            sums.append(item[2])
        else:
            parts[item[1]] = item
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w, steps = make_case(name)
    o = oracle.from_workload(w)
    o.step(steps)
    ref = o.moments()
    got = [np.concatenate([parts[y0][2][k] for y0 in sorted(parts)], axis=0) for k in range(4)]
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    want = np.array([sum(r + 1.0 for r in range(world)), sum(2.0 * r for r in range(world))])
    for s in sums:
        np.testing.assert_array_equal(s, want)


def test_single_rank_periodic_exchange_wraps_onto_itself():
    """world = 1 on a periodic axis: the slab's own first row is its ghost row
    above and its last row its ghost row below (no process group needed)."""
    a, b = torch.arange(5.0), torch.arange(5.0) + 10
    lo, hi = torch.zeros(5), torch.zeros(5)
    slabs.exchange(a, b, lo, hi, 0, 1, True)
    assert torch.equal(hi, a) and torch.equal(lo, b)
