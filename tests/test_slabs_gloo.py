"""Slab decomposition on CPU: the library's host orchestration of a domain split along x
(paper_1901_02955_gb300.slabs.SlabRun: exchange order, neighbours across a periodic seam,
the time step as the minimum over the slabs) run by two gloo ranks, each slab advanced by the
oracle on its cells plus three ghost columns per slab boundary. A stage's result in a cell
depends only on the cells within three along each axis, so the slabs must reproduce the
undecomposed oracle run exactly, walls and periodic, dry and moist. The same orchestration
drives the CUDA library's slabs (test_gpu_slabs.py)."""
import dataclasses
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from paper_1901_02955_gb300.slabs import Decomposition, SlabRun, gather, slab_bounds


class OracleSlab:
    """Slab s of w advanced by the oracle (test stand-in for the library's GpuSlab): the
    state of every slot is held with three extra columns beyond each slab boundary, which the
    exchange fills; the oracle's own ghost cells beyond those columns only affect the extra
    columns' results, which are discarded."""

    def __init__(self, w, dec, s):
        import torch
        self.torch = torch
        x0, x1 = dec.bounds[s]
        self.n = x1 - x0
        self.nl = 3 if dec.neighbour(s, 0) is not None else 0
        self.nr = 3 if dec.neighbour(s, 1) is not None else 0
        shape = w.Y.shape[:-1]
        ext = np.zeros(shape + (self.nl + self.n + self.nr,))
        ext[..., self.nl:self.nl + self.n] = w.Y[..., x0:x1]
        bc = list(w.bc)
        for side in (0, 1):
            if dec.neighbour(s, side) is not None:
                bc[side] = W.REFLECT  # placeholder beyond the exchanged columns
        if bc[0] != bc[1] and W.PERIODIC in bc[:2]:
            bc[0] = bc[1] = W.REFLECT
        self.o = Oracle(dataclasses.replace(w, nx=ext.shape[-1], Y=ext, bc=tuple(bc)))
        own = dataclasses.replace(w, nx=self.n, Y=np.ascontiguousarray(w.Y[..., x0:x1]),
                                  bc=(W.REFLECT,) * 6)
        self.o_own = Oracle(own)
        self.Y = [ext, np.zeros_like(ext), np.zeros_like(ext)]
        self.shape = shape

    def own(self, slot):
        return self.Y[slot][..., self.nl:self.nl + self.n]

    def pack(self, slot, side):
        o = self.own(slot)
        cols = o[..., :3] if side == 0 else o[..., self.n - 3:]
        return self.torch.from_numpy(np.ascontiguousarray(cols))

    def recv_buffer(self, side):
        return self.torch.empty(self.shape + (3,), dtype=self.torch.float64)

    def put_halo(self, slot, side, data):
        a = data.numpy()
        if side == 0:
            self.Y[slot][..., :3] = a
        else:
            self.Y[slot][..., self.nl + self.n:] = a

    def local_dt(self):
        return self.o_own.dt_cfl(np.ascontiguousarray(self.own(0)))

    def stage(self, st, dt):
        out, rc = self.o.stage(st, self.Y[0], self.Y[st], dt)
        assert rc >= 0
        self.Y[(1, 2, 0)[st]] = out

    def state(self):
        return np.ascontiguousarray(self.own(0))


def cases():
    return {
        "walls_dry_xz": W.add_random_motion(W.warm_bubble(n=30)),
        "periodic_moist_3d": W.add_random_motion(W.jovian(nx=13, ny=7, nz=12)),
    }


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, nslab, nsteps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = cases()[name]
        dec = Decomposition(w.nx, nslab, periodic=w.bc[0] == W.PERIODIC)
        engines = {s: OracleSlab(w, dec, s) for s in dec.slabs_of(rank, world)}
        run = SlabRun(dec, engines, rank, world, dist)
        dt = run.step(nsteps)
        mine = {s: e.state() for s, e in engines.items()}
        allst = [None] * world
        dist.all_gather_object(allst, mine)
        if rank == 0:
            merged = {}
            for d in allst:
                merged.update(d)
            q.put((gather(dec, merged), dt))
    finally:
        dist.destroy_process_group()


def run_ranks(name, nslab, nsteps, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, nslab, nsteps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("nslab", [2, 3])
@pytest.mark.parametrize("name", list(cases()))
def test_slabs_on_two_gloo_ranks_reproduce_the_domain(name, nslab):
    w = cases()[name]
    nsteps = 3
    Y, dt = run_ranks(name, nslab, nsteps)
    Yo, dto, rc = Oracle(w).step(w.Y, nsteps, dt=0.0)
    assert rc >= 0
    assert dt == dto
    assert np.array_equal(Y, Yo), float(np.abs(Y - Yo).max())


def test_decomposition_geometry():
    assert slab_bounds(40, 3) == [(0, 14), (14, 27), (27, 40)]
    with pytest.raises(ValueError):
        slab_bounds(8, 3)
    with pytest.raises(ValueError):
        slab_bounds(40, 1)
    ring = Decomposition(12, 3, periodic=True)
    chain = Decomposition(12, 3, periodic=False)
    assert [ring.neighbour(s, 0) for s in range(3)] == [2, 0, 1]
    assert [ring.neighbour(s, 1) for s in range(3)] == [1, 2, 0]
    assert [chain.neighbour(s, 0) for s in range(3)] == [None, 0, 1]
    assert [chain.neighbour(s, 1) for s in range(3)] == [1, 2, None]
    # each boundary is exchanged once in each direction
    assert len(ring.messages()) == 6 and len(chain.messages()) == 4
    assert [ring.owner(s, 2) for s in range(3)] == [0, 0, 1]
    assert sorted(s for r in range(4) for s in Decomposition(20, 5, True).slabs_of(r, 4)) == \
        list(range(5))
