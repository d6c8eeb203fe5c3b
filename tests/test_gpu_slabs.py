"""Slab decomposition of one domain along x in the CUDA library, through the C ABI: the
slabs reproduce the undecomposed run bit for bit (a stage's result in a cell depends only on
the cells within three along each axis, and linked slabs share the domain's CFL time step).
Two ways: every slab a domain of one context with its boundaries linked (snap_link_halo: the
kernels read the neighbour's cells in place), and one context per slab with the host
exchanging packed columns through the ghost buffers (snap_halo_pack, snap_halo_buffer;
SlabRun, the orchestration the multi-process path uses, here with every slab in one
process). FP64 dry walls and periodic over 10 CFL steps, FP32 moist 3-D periodic; then the
argument checks of the entry points."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()
    return t


def cases():
    return {
        "walls_dry_xz_f64": (W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f64")),
                             "f64"),
        "periodic_dry_3d_f64": (W.add_random_motion(W.dry_bubble_3d(nx=31, ny=10, nz=9)), "f64"),
        "periodic_moist_3d_f32": (W.add_random_motion(W.jovian(nx=26, ny=11, nz=18)), "f32"),
    }


def whole(w, dtype, nsteps, variant):
    from paper_1901_02955_gb300 import Context
    ctx = Context(w, dtype=dtype)
    ctx.set_tile_variant(variant)
    ctx.set_state(w.Y)
    dt = ctx.step(nsteps)
    Y = ctx.get_state()
    ctx.close()
    return Y, dt


@pytest.mark.parametrize("nslab", [2, 3])
@pytest.mark.parametrize("name", list(cases()))
def test_linked_slabs_in_one_context_reproduce_the_domain(torch, name, nslab):
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.slabs import Decomposition, gather, link_slabs, slab_workload
    w, dtype = cases()[name]
    nsteps = 10
    dec = Decomposition(w.nx, nslab, periodic=w.bc[0] == W.PERIODIC)
    slabs = [slab_workload(w, dec, s) for s in range(nslab)]
    ctx = Context(slabs, dtype=dtype)
    v = ctx.info()["tile_variant"]  # the same kernel instance for both runs
    link_slabs(ctx, dec)
    for s, ws in enumerate(slabs):
        ctx.set_state(ws.Y, domain=s)
    dt = ctx.step(nsteps)
    Y = gather(dec, {s: ctx.get_state(domain=s) for s in range(nslab)})
    ctx.close()
    Yw, dtw = whole(w, dtype, nsteps, v)
    assert dt == dtw
    assert np.array_equal(Y, Yw), float(np.abs(Y - Yw).max())


@pytest.mark.parametrize("nslab", [2, 3])
@pytest.mark.parametrize("name", ["walls_dry_xz_f64", "periodic_dry_3d_f64"])
def test_slab_contexts_with_host_exchange_reproduce_the_domain(torch, name, nslab):
    """One context per slab; before every stage the host packs each boundary's columns and
    copies them into the neighbour's ghost buffer (dry layouts: every tile shape rounds
    alike, so the contexts' own tile choices do not matter)."""
    from paper_1901_02955_gb300.slabs import (Decomposition, GpuSlab, SlabRun, gather,
                                              slab_workload)
    w, dtype = cases()[name]
    nsteps = 10
    dec = Decomposition(w.nx, nslab, periodic=w.bc[0] == W.PERIODIC)
    engines = {s: GpuSlab(slab_workload(w, dec, s), dtype) for s in range(nslab)}
    run = SlabRun(dec, engines)
    dt = run.step(nsteps)
    Y = gather(dec, {s: e.state() for s, e in engines.items()})
    for e in engines.values():
        e.close()
    Yw, dtw = whole(w, dtype, nsteps, 0)
    assert dt == dtw
    assert np.array_equal(Y, Yw), float(np.abs(Y - Yw).max())


def test_halo_entry_points_check_their_arguments(torch):
    from paper_1901_02955_gb300 import Context, SnapError, capi
    from paper_1901_02955_gb300.slabs import Decomposition, slab_workload
    w, _ = cases()["walls_dry_xz_f64"]
    dec = Decomposition(w.nx, 2, periodic=False)
    slabs = [slab_workload(w, dec, s) for s in range(2)]
    ctx = Context(slabs, dtype="f64")
    for s, ws in enumerate(slabs):
        ctx.set_state(ws.Y, domain=s)
    # an unlinked halo side stops the step
    with pytest.raises(SnapError) as e:
        ctx.step(1)
    assert e.value.code == capi.EINVAL
    with pytest.raises(SnapError):
        ctx.link_halo(0, 0, 1)  # slab 0's x- is a wall
    with pytest.raises(SnapError):
        ctx.link_halo(0, 1, 0)  # the facing side of slab 0 is not SNAP_HALO
    out = torch.empty(1, device="cuda")
    with pytest.raises(SnapError):
        ctx.halo_pack(0, 1, 3, out)  # no slot 3
    ctx.link_halo(0, 1, 1)
    ctx.link_halo(1, 0, 0)
    with pytest.raises(SnapError):
        ctx.halo_view(0, 1)  # linked sides have no ghost buffer
    ctx.step(1)
    ctx.close()
    # a different reference profile is not a slab of the same domain
    other = W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f64"))
    other.p_bar_face = other.p_bar_face * 1.001
    other.rho_bar = other.rho_bar * 1.001
    s1 = slab_workload(other, dec, 1)
    ctx = Context([slabs[0], s1], dtype="f64")
    with pytest.raises(SnapError):
        ctx.link_halo(0, 1, 1)
    ctx.close()
    # the adjoint is not built for slabs
    ctx = Context(slabs[0], dtype="f64")
    with pytest.raises(SnapError) as e:
        ctx.record(2, 1)
    assert e.value.code == capi.ENOTSUP
    ctx.close()


def _slab_rank(rank, world, port, name, nslab, nsteps, q):
    import os
    import torch
    import torch.distributed as dist
    from paper_1901_02955_gb300.slabs import Decomposition, GpuSlab, SlabRun, slab_workload
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w, dtype = cases()[name]
        dec = Decomposition(w.nx, nslab, periodic=w.bc[0] == W.PERIODIC)
        engines = {s: GpuSlab(slab_workload(w, dec, s), dtype) for s in dec.slabs_of(rank, world)}
        dt = SlabRun(dec, engines, rank, world, dist).step(nsteps)
        mine = {s: e.state() for s, e in engines.items()}
        allst = [None] * world
        dist.all_gather_object(allst, mine)
        if rank == 0:
            merged = {}
            for d in allst:
                merged.update(d)
            q.put((np.concatenate([merged[s] for s in range(nslab)], axis=-1), dt))
        for e in engines.values():
            e.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["walls_dry_xz_f64", "periodic_dry_3d_f64"])
def test_slabs_in_two_processes_reproduce_the_domain(torch, name):
    """The multi-process path with the CUDA library: two processes on the GPU, each holding
    its slabs (of three) in contexts of its own, exchange the ghost columns before every
    stage through torch.distributed (gloo, staged through host memory; NCCL carries device
    tensors directly) and take the CFL step as an all-reduced minimum: bitwise the
    undecomposed run over 10 steps."""
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_rank, args=(r, 2, port, name, 3, 10, q)) for r in range(2)]
    for p in procs:
        p.start()
    Y, dt = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w, dtype = cases()[name]
    Yw, dtw = whole(w, dtype, 10, 0)
    assert dt == dtw
    assert np.array_equal(Y, Yw), float(np.abs(Y - Yw).max())
