"""Lower boundary of the Jovian simulation (Sec. 6) in the oracle: a no-slip wall and a fixed
bottom temperature, both set in the ghost cells below the bottom wall. Pinned by closed forms
of the first tendency on uniform states (the wall stress of a uniform shear-free flow, the
heat flux into a gas at rest), and by invariants (nothing crosses a wall; the no-slip ghost
changes nothing where there is no tangential velocity; a bottom temperature equal to the
bottom cells' own changes nothing)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from helpers import uniform_column
from oracle.oracle import Oracle

RHO, P0, R, GAMMA = 1.1, 1e5, 287.0, 1.4


def strip(U=0.0, nu=0.0, nz=6, nx=8):
    return uniform_column(nx, 800.0, lambda x: RHO + 0 * x, lambda x: U + 0 * x,
                          lambda x: 0 * x, p0=P0, nz=nz, nu=nu)


def with_bottom(w, bc4=W.NOSLIP, T_bottom=0.0):
    bc = list(w.bc)
    bc[4] = bc4
    return dataclasses.replace(w, bc=tuple(bc), T_bottom=T_bottom)


def test_noslip_wall_stress_of_a_uniform_flow():
    """u = U everywhere over a no-slip bottom: the ghosts carry -U, so the only nonzero
    tendency is the viscous stress at the wall face, rho nu (U - (-U))/dz, drawn from the
    bottom row: d(rho u)/dt = -2 rho nu U / dz^2 there. The work term vanishes at the wall
    (the face velocity is the mean of U and -U), so rho e does not change; a free-slip wall
    gives no tendency at all."""
    U, nu = 5.0, 10.0
    w = with_bottom(strip(U=U, nu=nu))
    d = Oracle(w).rhs(w.Y)
    want = np.zeros_like(d)
    want[1, 0] = -2.0 * RHO * nu * U / w.dz ** 2
    scale = float(np.abs(want[1, 0]).max())
    np.testing.assert_allclose(d[:3], want[:3], rtol=0, atol=1e-12 * scale)
    assert np.abs(d[3]).max() <= 1e-9 * scale * P0
    d_free = Oracle(with_bottom(strip(U=U, nu=nu), W.REFLECT)).rhs(w.Y)
    assert np.abs(d_free[:3]).max() <= 1e-12 * scale


def test_fixed_bottom_temperature_heat_flux():
    """Gas at rest at T0 above ghosts held at T_b: the ghosts keep the pressure, so their
    density is rho T0 / T_b, and the wall face carries the heat flux
    -rho_f c_p nu (T0 - T_b) / dz with rho_f the mean of the two densities. The bottom row
    gains d(rho e)/dt = rho_f c_p nu (T_b - T0) / dz^2; mass and momenta do not change (the
    pressure is mirrored, so u* = 0 and p* = p at the wall)."""
    nu = 10.0
    T0 = P0 / (RHO * R)
    Tb = T0 + 30.0
    w = with_bottom(strip(nu=nu), W.REFLECT, T_bottom=Tb)
    d = Oracle(w).rhs(w.Y)
    rho_f = 0.5 * (RHO + RHO * T0 / Tb)
    cp = GAMMA * R / (GAMMA - 1.0)
    want = rho_f * cp * nu * (Tb - T0) / w.dz ** 2
    np.testing.assert_allclose(d[3, 0], want, rtol=1e-10)
    assert np.abs(d[3, 1:]).max() <= 1e-10 * want
    assert np.abs(d[:3]).max() <= 1e-12 * RHO * 1e3
    # no heat without viscosity: the wall advects nothing
    d0 = Oracle(with_bottom(strip(nu=0.0), W.REFLECT, T_bottom=Tb)).rhs(w.Y)
    assert np.abs(d0).max() <= 1e-9


def test_noslip_equals_free_slip_without_tangential_velocity():
    """With no velocity along the bottom wall the two walls' ghosts agree, and so do the
    tendencies (bitwise)."""
    w = uniform_column(8, 800.0, lambda x: RHO + 0.1 * np.sin(2 * np.pi * x / 800.0),
                       lambda x: 0 * x, lambda x: 2.0 * np.cos(2 * np.pi * x / 800.0),
                       p0=P0, nz=6, nu=5.0)
    a = Oracle(with_bottom(w, W.NOSLIP)).rhs(w.Y)
    b = Oracle(with_bottom(w, W.REFLECT)).rhs(w.Y)
    assert np.array_equal(a, b)


def jovian_closed(T_bottom=0.0, noise=0.1):
    w = W.add_random_motion(W.jovian(nx=6, ny=5, nz=16, noise_K=noise))
    Y = w.Y.copy()
    nvap, nc = len(w.vapors), w.ncond
    rs = np.random.default_rng(5)
    for i in range(nvap):  # some cloud and rain to fall
        for j in range(nc):
            Y[1 + nvap + i * nc + j] = Y[1 + i] * rs.uniform(0.0, 0.05, size=Y[1].shape)
    w = w.with_state(Y)
    return dataclasses.replace(w, bc=(W.NOSLIP,) * 6, T_bottom=T_bottom, w_term=(0.0, -20.0))


def test_nothing_crosses_noslip_walls_with_a_fixed_bottom_temperature():
    """Closed box of no-slip walls, a fixed bottom temperature and falling precipitation:
    every mass total and the total of rho e + rho g z keep zero tendency (no advective or
    sedimentation flux through a wall, inviscid)."""
    T_bot = 600.0
    w = jovian_closed(T_bot)
    o = Oracle(w, satadj=False)
    d = o.rhs(w.Y)
    nmass = 1 + len(w.vapors) * (1 + w.ncond)
    for s in range(nmass):
        tot = np.abs(w.Y[s]).sum()
        assert abs(d[s].sum()) * w.dz <= 1e-12 * tot, s
    z = (np.arange(w.nz) + 0.5) * w.dz
    rho_t = d[:nmass].sum(axis=0)
    e_t = d[-1] + rho_t * w.grav * z[:, None, None]
    assert abs(e_t.sum()) <= 1e-11 * np.abs(w.Y[-1]).sum() / 1e3
    # and the fixed temperature does change the tendency next to the wall
    d_off = Oracle(dataclasses.replace(w, T_bottom=0.0), satadj=False).rhs(w.Y)
    assert np.abs(d - d_off)[:, :3].max() > 0.0
    assert np.array_equal(d[:, 6:], d_off[:, 6:])


def test_bottom_temperature_equal_to_the_bottom_cells_changes_nothing():
    """Ghosts held at the temperature of the cells they mirror are the mirrored cells
    themselves."""
    w = W.jovian(nx=4, ny=4, nz=12, noise_K=0.0)
    o = Oracle(w, satadj=False)
    nv = o.nv
    _, T, _ = o.cons_to_prim(w.Y[:, 0, 0, 0])
    a = Oracle(dataclasses.replace(w, T_bottom=float(T)), satadj=False).rhs(w.Y)
    b = o.rhs(w.Y)
    # the state is at rest and balanced, so both tendencies are rounding noise: compare each
    # field on the scale of its own advective rate (|Y| * 1000 m/s / dz)
    for f in range(nv):
        tol = 1e-12 * np.abs(w.Y[f]).max() * 1000.0 / w.dz
        assert np.abs(a[f] - b[f]).max() <= tol, f


def test_adjoint_refuses_the_new_walls():
    w = jovian_closed()
    w = dataclasses.replace(w, w_term=(0.0, 0.0), cooling=(), sponge=())
    o = Oracle(w, satadj=False)
    with pytest.raises(Exception):
        o.rhs_adjoint(w.Y, np.ones_like(w.Y))
