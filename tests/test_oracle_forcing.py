"""Pins of the forcing of the Jovian simulation (Sec. 6): the body cooling (-C_v Q of the
energy in the cooled levels, C_v the heat capacity of the cell's mixture at constant volume)
and the sponge (Newtonian relaxation of the horizontal momenta at 1/(tau0 (p/p0)^2), the
total energy unchanged). Tendencies against the closed forms, the exact SSP-RK3 decay of a
uniform flow in the sponge, and the energy budget under uniform cooling."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

Q = 1.0 / 86400.0  # 1 K/day


def column(noise_K=0.1, **kw):
    w = W.jovian(nx=4, ny=4, nz=24, seed=W.BASE_SEED + 81, noise_K=noise_K)
    return dataclasses.replace(w, **kw)


def heat_capacity(w, Y):
    """C_v of each cell from the species table: c_vd rho_d + sum c_v,i rho_i + sum c_ij rho_ij."""
    c_vd = w.R_d / (w.gamma_d - 1.0)
    nvap, nc = len(w.vapors), w.ncond
    cv = c_vd * Y[0]
    for i, v in enumerate(w.vapors):
        cv = cv + v.sigma_v * c_vd * Y[1 + i]
        for j in range(nc):
            cv = cv + v.cond[j].sigma_v * c_vd * Y[1 + nvap + i * nc + j]
    return cv


def pbar(w):
    return 0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:])


def with_condensate(w, seed=82):
    """Cloud and precipitation in every cell, fractions of the vapour."""
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    nvap, nc = len(w.vapors), w.ncond
    for i in range(nvap):
        for j in range(nc):
            Y[1 + nvap + i * nc + j] = Y[1 + i] * rs.uniform(0.05, 0.3, size=Y[1].shape)
    return w.with_state(Y)


def test_cooling_tendency_in_the_band_only():
    w0 = W.add_random_motion(with_condensate(column()))
    pk = pbar(w0)
    lo, hi = np.sort(pk)[6], np.sort(pk)[16]
    w1 = dataclasses.replace(w0, cooling=(Q, lo, hi))
    d = Oracle(w1).rhs(w0.Y) - Oracle(w0).rhs(w0.Y)
    band = ((pk >= lo) & (pk <= hi))[:, None, None]
    want = np.where(band, -heat_capacity(w0, w0.Y) * Q, 0.0)
    assert d[-1] == pytest.approx(want, rel=1e-9, abs=1e-12 * np.abs(want).max())
    assert np.all(d[:-1] == 0.0)


def test_sponge_tendency_and_energy():
    w0 = W.add_random_motion(column())
    pk = pbar(w0)
    p0, tau0 = np.sort(pk)[8], 1e4
    w1 = dataclasses.replace(w0, sponge=(tau0, p0))
    d = Oracle(w1).rhs(w0.Y) - Oracle(w0).rhs(w0.Y)
    lay = (pk < p0)[:, None, None]
    tau = tau0 * (pk / p0)[:, None, None] ** 2
    im0 = 1 + len(w0.vapors) * (1 + w0.ncond)
    for m in (0, 1):  # x and y momenta
        f = im0 + m
        want = np.where(lay, -w0.Y[f] / tau, 0.0)
        assert d[f] == pytest.approx(want, rel=1e-12, abs=1e-14 * np.abs(want).max())
    others = [f for f in range(w0.nv) if f not in (im0, im0 + 1)]
    assert np.all(d[others] == 0.0)  # vertical momentum and the energy are untouched


def test_sponge_decays_a_uniform_flow_like_rk3_on_the_linear_ode():
    """A uniform horizontal flow in a horizontally uniform, discretely hydrostatic column with
    periodic sides: the sponge is the only
    tendency, and SSP-RK3 advances du/dt = -u/tau by the factor 1 - z + z^2/2 - z^3/6,
    z = dt/tau, per step."""
    w = column(noise_K=0.0)  # horizontally uniform and discretely hydrostatic
    Y = w.Y.copy()
    im0 = 1 + len(w.vapors) * (1 + w.ncond)
    rho = Y[:im0].sum(axis=0)
    # slow enough that the heat of the damped kinetic energy (its buoyancy ~ U^2) stays below
    # rounding relative to the decay itself
    U = 0.04
    Y[im0] = rho * U
    Y[-1] += 0.5 * rho * U * U
    pk = pbar(w)
    dt, n = 0.5 * Oracle(w).dt_cfl(Y, 0.8), 5
    p0 = np.sort(pk)[10]
    tau0 = 4.0 * dt * (p0 / pk.min()) ** 2  # dt/tau <= 1/4 at every level (RK3 stable)
    w = dataclasses.replace(w.with_state(Y), sponge=(tau0, p0))
    o = Oracle(w, satadj=False)
    Yn = o.step(Y, n, dt=dt)[0]
    z = dt / (tau0 * (pk / p0) ** 2)
    fac = np.where(pk < p0, (1 - z + z * z / 2 - z ** 3 / 6) ** n, 1.0)[:, None, None]
    assert Yn[im0] == pytest.approx(Y[im0] * fac, rel=1e-9)
    # the sponge leaves the total energy unchanged
    assert o.budget(Yn)[-1] == pytest.approx(o.budget(Y)[-1], rel=1e-13)


def test_uniform_cooling_drains_energy_at_the_total_heat_capacity():
    """Cooling every level: d/dt sum(rho e + rho g z) dV = -Q sum_k c_k M_k, a constant (the
    masses M_k of the components are conserved), which SSP-RK3 integrates exactly."""
    w = W.add_random_motion(column())
    w = dataclasses.replace(w, cooling=(Q * 100, 0.0, 1e12))
    o = Oracle(w, satadj=False)
    b0 = o.budget(w.Y)
    dt, n = 0.5 * o.dt_cfl(w.Y, 0.8), 4
    Y1 = o.step(w.Y, n, dt=dt)[0]
    b1 = o.budget(Y1)
    vol = w.dx * w.dy * w.dz
    drain = Q * 100 * heat_capacity(w, w.Y).sum() * vol * dt * n
    assert b0[-1] - b1[-1] == pytest.approx(drain, rel=1e-9)
