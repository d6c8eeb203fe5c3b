"""Slab decomposition of one domain along x: the way Athena++, the framework the paper's
solver runs in, spreads one grid over processes. Each slab advances its own cells; before
every Runge-Kutta stage (Sec. 4.3) it receives from each neighbouring slab the three columns
next to their common boundary, the reach of the WENO5 stencil (Sec. 4.2), which the stage
kernels use as that side's ghost cells (the library's SNAP_HALO sides). All slabs of a domain
advance with one time step: the CFL rule's minimum over every slab, i.e. over the whole
domain. A slab decomposition therefore reproduces the undecomposed run exactly.

Two ways to run it:
  - all slabs as domains of one context on one GPU, linked (link_slabs): the kernels read a
    neighbour's cells straight from its state buffer, no copy and no extra launch, and the
    linked slabs share one CFL time step inside the library;
  - one slab per context, the contexts on any mix of processes and GPUs (SlabRun): the host
    exchanges the packed columns before every stage (a device copy between slabs of one
    process, torch.distributed send/receive between processes -- NCCL for GPUs, gloo on CPU)
    and takes the minimum of the slabs' time steps with an all-reduce.
The engines SlabRun drives only need pack / recv_buffer / put_halo / local_dt / stage; GpuSlab
is the library's."""
import dataclasses

import numpy as np

from .capi import HALO, Context


def slab_bounds(nx, nslab):
    """x ranges [x0, x1) of nslab slabs of an nx-cell domain, sizes as equal as possible
    (the larger first), each at least 3 cells (the ghost columns a neighbour takes)."""
    if nslab < 2:
        raise ValueError("a decomposition has at least two slabs")
    if nx < 3 * nslab:
        raise ValueError("each slab needs at least 3 cells in x")
    base, extra = divmod(nx, nslab)
    out, x = [], 0
    for s in range(nslab):
        n = base + (1 if s < extra else 0)
        out.append((x, x + n))
        x += n
    return out


class Decomposition:
    """nslab slabs along x of an nx-cell domain; periodic: the last slab's x+ neighbour is the
    first slab (an x-periodic domain), else the two outer sides keep the domain's walls."""

    def __init__(self, nx, nslab, periodic):
        self.nx = nx
        self.nslab = nslab
        self.periodic = bool(periodic)
        self.bounds = slab_bounds(nx, nslab)

    def neighbour(self, s, side):
        """Slab across side (0: x-, 1: x+) of slab s, or None at a wall."""
        n = s - 1 if side == 0 else s + 1
        if 0 <= n < self.nslab:
            return n
        return n % self.nslab if self.periodic else None

    def owner(self, s, world):
        """Rank holding slab s: consecutive slabs on each rank, ranks in order."""
        return s * world // self.nslab

    def slabs_of(self, rank, world):
        return [s for s in range(self.nslab) if self.owner(s, world) == rank]

    def messages(self):
        """Every exchange of one stage in a fixed global order: (sender slab, sender side,
        receiving slab, receiving side). The sender's columns next to its side become the
        receiver's ghost columns on the opposite side."""
        out = []
        for s in range(self.nslab):
            for side in (0, 1):
                n = self.neighbour(s, side)
                if n is not None:
                    out.append((s, side, n, 1 - side))
        return out


def slab_workload(w, dec, s):
    """Workload of slab s of w (same parameters and reference profile, the slab's cells;
    SNAP_HALO on every side facing another slab)."""
    if dec.nx != w.nx:
        raise ValueError("decomposition and workload differ in nx")
    periodic_x = w.bc[0] == 1 and w.bc[1] == 1
    if periodic_x != dec.periodic:
        raise ValueError("the decomposition's periodicity must match the workload's x sides")
    x0, x1 = dec.bounds[s]
    bc = list(w.bc)
    for side in (0, 1):
        if dec.neighbour(s, side) is not None:
            bc[side] = HALO
    return dataclasses.replace(w, nx=x1 - x0, Y=np.ascontiguousarray(w.Y[..., x0:x1]),
                               bc=tuple(bc), name=f"{w.name}_slab{s}")


def link_slabs(ctx, dec, first=0):
    """Link every slab boundary of a context whose domains first .. first + nslab - 1 are the
    slabs of dec in order (snap_link_halo from both sides)."""
    for s, side, n, _ in dec.messages():
        ctx.link_halo(first + s, side, first + n)


class GpuSlab:
    """One slab in a context of its own (CUDA library), on the current torch stream."""

    def __init__(self, w_slab, dtype, Y=None):
        import torch
        self.torch = torch
        self.w = w_slab
        self.ctx = Context(w_slab, dtype=dtype)
        self.ctx.set_stream(torch.cuda.current_stream())
        self.tdtype = torch.float32 if self.ctx.f32 else torch.float64
        self.ghost = {side: self.ctx.halo_view(0, side) for side in (0, 1)
                      if w_slab.bc[side] == HALO}
        self.ctx.set_state(w_slab.Y if Y is None else Y)

    def pack(self, slot, side):
        out = self.torch.empty((self.w.nv, self.w.nz, self.w.ny, 3), dtype=self.tdtype,
                               device="cuda")
        self.ctx.halo_pack(0, side, slot, out)
        return out

    def recv_buffer(self, side):
        return self.ghost[side]

    def put_halo(self, slot, side, data):
        if data is not self.ghost[side]:
            self.ghost[side].copy_(data)  # device copy, or host to device after a gloo receive

    def local_dt(self):
        return self.ctx.compute_dt()

    def stage(self, st, dt):
        self.ctx.stage(st, dt)

    def state(self):
        return self.ctx.get_state()

    def close(self):
        self.ctx.close()


class SlabRun:
    """Steps the slabs of a Decomposition held by this rank (engines: slab -> engine) in
    lockstep with the other ranks' slabs. dist: torch.distributed (initialised) or None for a
    single process holding every slab."""

    def __init__(self, dec, engines, rank=0, world=1, dist=None, device=None):
        self.dec = dec
        self.engines = dict(engines)
        self.rank, self.world, self.dist = rank, world, dist
        self.device = device
        if sorted(self.engines) != dec.slabs_of(rank, world):
            raise ValueError("engines must be exactly this rank's slabs")
        # a backend without device tensors (gloo) moves the columns through host memory
        self.host_staged = dist is not None and world > 1 and dist.get_backend() == "gloo"

    def exchange(self, slot):
        """Ghost columns of every slab boundary for the stage whose input is state slot `slot`
        (0, 1, 2): local pairs by direct copy, remote ones by send/receive, posted by every
        rank in the same global order so that each pair of ranks matches them in sequence."""
        ops, post = [], []
        for s, side, n, nside in self.dec.messages():
            mine, theirs = s in self.engines, n in self.engines
            if mine and theirs:
                self.engines[n].put_halo(slot, nside, self.engines[s].pack(slot, side))
            elif mine:
                data = self.engines[s].pack(slot, side)
                if self.host_staged and data.is_cuda:
                    data = data.cpu()
                ops.append(self.dist.P2POp(self.dist.isend, data, self.dec.owner(n, self.world)))
            elif theirs:
                buf = self.engines[n].recv_buffer(nside)
                if self.host_staged and buf.is_cuda:
                    buf = buf.new_empty(buf.shape, device="cpu")
                ops.append(self.dist.P2POp(self.dist.irecv, buf, self.dec.owner(s, self.world)))
                post.append((n, nside, buf))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        for n, nside, buf in post:
            self.engines[n].put_halo(slot, nside, buf)

    def global_dt(self):
        """CFL time step of the whole domain: the smallest of the slabs' own."""
        dt = min(e.local_dt() for e in self.engines.values())
        if self.dist is not None and self.world > 1:
            import torch
            t = torch.tensor([dt], dtype=torch.float64, device=self.device)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
            dt = float(t.item())
        return dt

    def step(self, nsteps=1, dt_fixed=0.0):
        """nsteps SSP-RK3 steps of every slab; returns the last time step."""
        dt = dt_fixed
        for _ in range(nsteps):
            dt = dt_fixed if dt_fixed > 0 else self.global_dt()
            for st in range(3):
                self.exchange(st)
                for s in sorted(self.engines):
                    self.engines[s].stage(st, dt)
        return dt


def gather(dec, states):
    """The whole domain's state from the slabs' states (slab -> array), along x."""
    return np.concatenate([states[s] for s in range(dec.nslab)], axis=-1)
