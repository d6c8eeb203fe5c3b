"""Locality of one Runge-Kutta stage in the oracle (Sec. 4: WENO5 reads three cells on either
side of a face, LMARS and the flux divergence one face on either side of a cell, the
saturation adjustment and the sources the cell itself): a cell's stage result depends only
on the cells within three along each axis. So the stage run on the 7-cell window around a
cell (x and y wrapped as the periodic domain is) gives that cell's value bit for bit, which
is what the full-size Jovian parity check relies on; a stencil that reached a fourth cell
(an index one off in a halo) makes the two differ."""
import dataclasses

import numpy as np

import workloads as W
from oracle import Oracle


def window_of(w, i, j, k):
    """The workload cut to the 7 x 7 x 7 (x-z: 7 x 1 x 7) window centred on cell (i, j, k)."""
    xi = [(i + s) % w.nx for s in range(-3, 4)]
    yj = [(j + s) % w.ny for s in range(-3, 4)] if w.ny > 1 else [0]
    Y = np.ascontiguousarray(w.Y[:, k - 3:k + 4][:, :, yj][:, :, :, xi])
    return dataclasses.replace(w, nx=7, ny=len(yj), nz=7, Y=Y, rho_bar=w.rho_bar[k - 3:k + 4],
                               p_bar_face=w.p_bar_face[k - 3:k + 5])


def check_windows(w, nsamp, seed, dt):
    full, _ = Oracle(w).stage(0, w.Y, w.Y, dt)
    rs = np.random.default_rng(seed)
    for _ in range(nsamp):
        i, j = int(rs.integers(w.nx)), int(rs.integers(w.ny))
        k = int(rs.integers(3, w.nz - 3))
        ww = window_of(w, i, j, k)
        out, _ = Oracle(ww).stage(0, ww.Y, ww.Y, dt)
        jj = 3 if w.ny > 1 else 0
        assert np.array_equal(out[:, 3, jj, 3], full[:, k, j, i]), (i, j, k)


def test_moist_3d_stage_depends_on_three_cells_each_way():
    w = W.add_random_motion(W.jovian(nx=16, ny=16, nz=16, dtype="f64"))
    check_windows(w, 10, 5, dt=0.5)


def test_moist_xz_stage_depends_on_three_cells_each_way():
    # periodic in x like the Jovian column (the window wraps x); walls only above and below
    w = W.add_random_motion(W.moist_bubble(nx=24, nz=20))
    w = dataclasses.replace(w, bc=(W.PERIODIC, W.PERIODIC) + tuple(w.bc[2:]))
    check_windows(w, 10, 6, dt=0.02)


def test_a_stencil_reaching_four_cells_would_be_seen():
    """The window check is sensitive: at the cell next to the window's centre, whose stencil
    reaches one cell past the window's edge, the window's result differs from the full
    domain's once the flow there is not uniform."""
    w = W.add_random_motion(W.jovian(nx=16, ny=16, nz=16, dtype="f64"))
    full, _ = Oracle(w).stage(0, w.Y, w.Y, 0.5)
    ww = window_of(w, 8, 8, 8)
    out, _ = Oracle(ww).stage(0, ww.Y, ww.Y, 0.5)
    # the cell next to the window's centre sees the window's (mirrored) edge within 3 cells
    assert not np.array_equal(out[:, 3, 3, 4], full[:, 8, 8, 9])
