"""Whole-scheme pins of the oracle (Sec. 4: Eqs. forward, riemann, q+, rp, ru, weno5 and the
SSP-RK3 of Sec. 4.3) against what the equations fix: hydrostatic rest, conservation in a
closed box, mirror symmetry, Galilean translation of a uniform state, the order of the
Runge-Kutta stages and of the whole scheme, and the viscous decay rate."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from oracle.oracle import rk3_combine

from helpers import no_gravity, uniform_column


def test_isentropic_rest_stays_at_rest():
    w = W.rest_state(nx=24, nz=24)
    o = Oracle(w)
    Y, _, _ = o.step(w.Y, 100)
    rho = Y[0]
    assert np.abs(Y[1] / rho).max() < 1e-10
    assert np.abs(Y[2] / rho).max() < 1e-10
    np.testing.assert_allclose(Y[3], w.Y[3], rtol=1e-13)


def test_isothermal_rest_stays_at_rest():
    w = W.isothermal_rest(nx=16, nz=32, T0=250.0)
    o = Oracle(w)
    Y, _, _ = o.step(w.Y, 100)
    assert np.abs(Y[2] / Y[0]).max() < 1e-10
    assert np.abs(Y[1] / Y[0]).max() < 1e-10


def test_viscous_rest_stays_at_rest():
    """The isentropic background has uniform theta, so it carries no heat flux."""
    w = dataclasses.replace(W.rest_state(nx=16, nz=24), nu=75.0)
    o = Oracle(w)
    Y, _, _ = o.step(w.Y, 50)
    assert np.abs(Y[2] / Y[0]).max() < 1e-10
    np.testing.assert_allclose(Y[3], w.Y[3], rtol=1e-12)


def test_moist_rest_stays_at_rest():
    w = W.jovian(nx=4, ny=4, nz=24, noise_K=0.0)
    o = Oracle(w)
    Y, _, rc = o.step(w.Y, 5)
    assert rc >= 0
    rho = Y[:7].sum(axis=0)
    assert np.abs(Y[7:10] / rho).max() < 1e-9
    np.testing.assert_allclose(Y[:7], w.Y[:7], rtol=1e-11, atol=1e-15)


def closed_box_cases():
    b = W.add_random_motion(W.warm_bubble(n=16))
    m = W.add_random_motion(W.moist_bubble(n=16))
    j = W.add_random_motion(W.jovian(nx=6, ny=5, nz=12, Lx=3e3, Ly=2.5e3, Lz=6e3))
    return [b, dataclasses.replace(b, nu=75.0), m, j]


@pytest.mark.parametrize("idx", range(4))
def test_conservation_without_gravity(idx):
    w = no_gravity(closed_box_cases()[idx])
    o = Oracle(w)
    Y, _, rc = o.step(w.Y, 10)
    assert rc >= 0
    b0, b1 = o.budget(w.Y), o.budget(Y)
    nvap, nc = len(w.vapors), w.ncond
    im0 = 1 + nvap + nvap * nc
    assert b1[0] == pytest.approx(b0[0], rel=1e-13)
    for i in range(nvap):  # each species summed over its phases
        s0 = b0[1 + i] + sum(b0[1 + nvap + i * nc + j] for j in range(nc))
        s1 = b1[1 + i] + sum(b1[1 + nvap + i * nc + j] for j in range(nc))
        assert s1 == pytest.approx(s0, rel=1e-12)
    assert b1[o.nv - 1] == pytest.approx(b0[o.nv - 1], rel=1e-13)
    if w.bc[0] == W.PERIODIC:  # periodic horizontal momentum is conserved
        scale = np.abs(w.Y[im0]).sum() * w.dx * w.dy * w.dz
        assert abs(b1[im0] - b0[im0]) < 1e-12 * scale


@pytest.mark.parametrize("idx", range(4))
def test_total_energy_with_potential_is_conserved(idx):
    w = closed_box_cases()[idx]
    o = Oracle(w)
    Y, _, rc = o.step(w.Y, 10)
    assert rc >= 0
    b0, b1 = o.budget(w.Y), o.budget(Y)
    assert b1[o.nv] == pytest.approx(b0[o.nv], rel=1e-13)
    assert b1[0] == pytest.approx(b0[0], rel=1e-13)


def test_pointwise_energy_source_is_not_exactly_conservative():
    """The option -g (rho w)_k only conserves rho e + rho g z to truncation error; the flux
    form is exact (reading of the energy source)."""
    w = W.add_random_motion(W.warm_bubble(n=16))
    o = Oracle(w, energy_pointwise=True)
    Y, _, _ = o.step(w.Y, 10)
    b0, b1 = o.budget(w.Y), o.budget(Y)
    assert abs(b1[o.nv] / b0[o.nv] - 1.0) > 1e-12


def test_mirror_symmetry_of_centred_bubble():
    w = W.warm_bubble(n=32, xc=500.0, zc=300.0)
    o = Oracle(w)
    Y, _, _ = o.step(w.Y, 20)
    for v in (0, 2, 3):
        np.testing.assert_allclose(Y[v], Y[v][..., ::-1], rtol=1e-14, atol=0)
    np.testing.assert_allclose(Y[1], -Y[1][..., ::-1], rtol=0,
                               atol=1e-14 * np.abs(Y[1]).max())
    assert np.abs(Y[2]).max() > 1e-3  # the bubble has started to rise


def test_uniform_flow_stays_uniform():
    w = uniform_column(24, 1000.0, lambda x: 1.2 + 0 * x, lambda x: 17.0 + 0 * x,
                       lambda x: 0 * x)
    o = Oracle(w)
    Y, _, _ = o.step(w.Y, 20)
    np.testing.assert_allclose(Y, w.Y, rtol=1e-13)


def test_rk3_stage_algebra_is_third_order():
    lam = -1.3 + 0.0j
    errs = []
    for n in (20, 40, 80):
        dt = 1.0 / n
        y = np.array([1.0])
        for _ in range(n):
            y1 = rk3_combine(0, y, y, lam.real * y, dt)
            y2 = rk3_combine(1, y, y1, lam.real * y1, dt)
            y = rk3_combine(2, y, y2, lam.real * y2, dt)
        errs.append(abs(y[0] - np.exp(lam.real)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.9 and max(orders) < 3.1, orders


def test_advected_density_converges():
    """A smooth density profile carried by a uniform flow at uniform pressure is translated
    exactly by the Euler equations; after one period the scheme's error must fall at least
    at third order (SSP-RK3 at fixed CFL; WENO5 in space)."""
    L, U = 1000.0, 50.0
    errs = []
    for n in (16, 32, 64):
        w = uniform_column(n, L, lambda x: 1.0 + 0.2 * np.sin(2 * np.pi * x / L),
                           lambda x: U + 0 * x, lambda x: 0 * x)
        o = Oracle(w)
        t_end = L / U
        dt0 = o.dt_cfl(w.Y, 0.8)
        nst = int(np.ceil(t_end / dt0))
        Y, _, _ = o.step(w.Y, nst, dt=t_end / nst)
        errs.append(np.sqrt(np.mean((Y[0] - w.Y[0]) ** 2)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.7, (errs, orders)


def test_viscous_shear_decays_at_the_diffusive_rate():
    """u = U cos(pi z / H) between free-slip (mirror) walls, periodic in x, no gravity:
    constant viscosity makes it decay as exp(-nu (pi/H)^2 t)."""
    H, nu, nz, nx = 1000.0, 75.0, 64, 4
    dz = H / nz
    z = (np.arange(nz) + 0.5) * dz
    u = 2.0 * np.cos(np.pi * z / H)[:, None, None] * np.ones((nz, 1, nx))
    Y = np.zeros((4, nz, 1, nx))
    Y[0] = 1.0
    Y[1] = u
    Y[3] = 1e5 / 0.4 + 0.5 * u * u
    w = W.Workload(name="shear", nx=nx, ny=1, nz=nz, dx=dz, dy=dz, dz=dz,
                   bc=(W.PERIODIC, W.PERIODIC, W.REFLECT, W.REFLECT, W.REFLECT, W.REFLECT),
                   grav=0.0, gamma_d=1.4, R_d=287.0, vapors=[], ncond=0, rho_bar=np.ones(nz),
                   p_bar_face=np.full(nz + 1, 1e5), Y=Y, nu=nu)
    o = Oracle(w)
    t_end = 40.0
    nst = int(np.ceil(t_end / o.dt_cfl(w.Y, 0.8)))
    Yt, _, _ = o.step(w.Y, nst, dt=t_end / nst)
    mode = np.cos(np.pi * z / H)
    amp0 = np.sum(w.Y[1][:, 0, 0] * mode)
    amp1 = np.sum(Yt[1][:, 0, 0] * mode)
    assert amp1 / amp0 == pytest.approx(np.exp(-nu * (np.pi / H) ** 2 * t_end), rel=2e-3)
    # without viscosity the mode is kept (the scheme's own dissipation is far smaller)
    o0 = Oracle(dataclasses.replace(w, nu=0.0))
    Y0, _, _ = o0.step(w.Y, nst, dt=t_end / nst)
    assert np.sum(Y0[1][:, 0, 0] * mode) / amp0 == pytest.approx(1.0, abs=1e-4)
    b0, b1 = o.budget(w.Y), o.budget(Yt)
    assert b1[3] == pytest.approx(b0[3], rel=1e-13)  # kinetic energy went into heat


def test_cfl_time_step_uses_the_sound_speed():
    w = uniform_column(8, 800.0, lambda x: 1.1 + 0 * x, lambda x: -12.0 + 0 * x,
                       lambda x: 0 * x)
    o = Oracle(w)
    c = np.sqrt(1.4 * 1e5 / 1.1)  # ideal-gas sound speed
    # unsplit rule: cfl / sum over directions of (|u_d| + c) / dx_d
    assert o.dt_cfl(w.Y, 0.8) == pytest.approx(0.8 / ((12.0 + c) / 100.0 + c / 100.0),
                                               rel=1e-13)


def test_budget_of_uniform_state():
    w = uniform_column(8, 800.0, lambda x: 1.1 + 0 * x, lambda x: 0 * x, lambda x: 0 * x)
    o = Oracle(w)
    b = o.budget(w.Y)
    assert b[0] == pytest.approx(1.1 * 800.0 * 3 * 100.0, rel=1e-14)
