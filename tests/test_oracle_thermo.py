"""Pins of the oracle's thermodynamics: the App. B maps against the equation of state and
energy of Sec. 2 written in density form, the effective adiabatic index special case,
virtual temperature, the Clausius-Clapeyron relation of App. D, and the isochoric
phase-change heating of Sec. 2 (Eq. phase)."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

from test_oracle_lmars import indep_cons, random_prim


def moist():
    return Oracle(W.jovian(nx=4, ny=4, nz=8))


def earth():
    return Oracle(W.moist_bubble(n=8))


@pytest.mark.parametrize("make", [moist, earth])
def test_prim_cons_round_trip(make):
    o = make()
    rs = np.random.default_rng(11)
    for _ in range(200):
        X = random_prim(o, rs, 0.0)
        X[-1] = rs.uniform(1e3, 3e6)
        Y = o.prim_to_cons(X)
        X2, T, gam = o.cons_to_prim(Y)
        np.testing.assert_allclose(X2, X, rtol=1e-13, atol=1e-13 * np.abs(X).max())


@pytest.mark.parametrize("make", [moist, earth])
def test_cons_to_prim_matches_density_form(make):
    """App. B's q-form (Eq. p2) against Sec. 2's p = (rho_d R_d + sum rho_i R_i) T and
    rho e = C_v T + K + A evaluated directly on densities."""
    o = make()
    rs = np.random.default_rng(12)
    for _ in range(200):
        X = random_prim(o, rs, 0.0)
        X[-1] = rs.uniform(1e3, 3e6)
        Y, T = indep_cons(o, X, 0.0)
        X2, T2, _ = o.cons_to_prim(Y)
        np.testing.assert_allclose(X2, X, rtol=1e-12, atol=1e-12 * np.abs(X).max())
        assert T2 == pytest.approx(T, rel=1e-12)


def test_gamma_special_case():
    """sigma_v,i = 1/eps_i and no condensate: gamma = gamma_d and p = (gamma - 1) U (App. B)."""
    w = W.jovian(nx=4, ny=4, nz=8)
    for v in w.vapors:
        v.sigma_v = 1.0 / v.eps
    o = Oracle(w)
    rs = np.random.default_rng(13)
    for _ in range(100):
        X = random_prim(o, rs, 0.0)
        X[3:7] = 0.0  # no condensates
        X[-1] = rs.uniform(1e3, 3e6)
        Y = o.prim_to_cons(X)
        _, T, gam = o.cons_to_prim(Y)
        assert gam == pytest.approx(w.gamma_d, rel=1e-14)
        rho = X[0]
        K = 0.5 * rho * np.sum(X[7:10] ** 2)
        assert X[-1] == pytest.approx((gam - 1.0) * (Y[-1] - K), rel=1e-12)


@pytest.mark.parametrize("make", [moist, earth])
def test_virtual_temperature(make):
    """p = rho R_d T_v with T_v = T [1 + sum q_i (1/eps_i - 1) - sum q_ij] (Eqs. eos, tv)."""
    o = make()
    w = o.w
    nvap = len(w.vapors)
    rs = np.random.default_rng(14)
    for _ in range(100):
        X = random_prim(o, rs, 0.0)
        X[-1] = rs.uniform(1e3, 3e6)
        Y = o.prim_to_cons(X)
        X2, T, _ = o.cons_to_prim(Y)
        Tv = T * (1.0 + sum(X2[1 + i] * (1.0 / v.eps - 1.0) for i, v in enumerate(w.vapors))
                  - X2[1 + nvap:1 + nvap + nvap * w.ncond].sum())
        assert X2[-1] == pytest.approx(X2[0] * w.R_d * Tv, rel=1e-13)


@pytest.mark.parametrize("make", [moist, earth])
def test_clausius_clapeyron(make):
    """d ln p*/dT = L(T)/(R_i T^2) with L(T) = L^r - dc (T - T^r) (App. D and Eq. latent),
    and p*(T^r) = p^r."""
    o = make()
    w = o.w
    c_vd = w.R_d / (w.gamma_d - 1.0)
    for i, v in enumerate(w.vapors):
        assert o.sat_pressure(i, v.T_ref) == pytest.approx(v.p_ref, rel=1e-15)
        Ri = w.R_d / v.eps
        dc = v.cond[0].sigma_v * c_vd - (v.sigma_v * c_vd + Ri)
        for T in np.linspace(0.6 * v.T_ref, 1.6 * v.T_ref, 11):
            h = 1e-4 * T
            num = (np.log(o.sat_pressure(i, T + h)) - np.log(o.sat_pressure(i, T - h))) / (2 * h)
            L = v.cond[0].L_ref - dc * (T - v.T_ref)
            assert num == pytest.approx(L / (Ri * T * T), rel=1e-7)


@pytest.mark.parametrize("make", [moist, earth])
def test_isochoric_phase_change_heating(make):
    """Moving d rho of vapour k into condensate (k,l) at fixed rho e changes T by
    d rho (L_kl(T) - R_k T) / C_v(after)  (Sec. 2, Eq. phase and the dT that follows)."""
    o = make()
    w = o.w
    nvap, nc = len(w.vapors), w.ncond
    c_vd = w.R_d / (w.gamma_d - 1.0)
    rs = np.random.default_rng(15)
    for _ in range(100):
        X = random_prim(o, rs, 0.0)
        X[-1] = rs.uniform(1e4, 3e6)
        Y = o.prim_to_cons(X)
        _, T0, _ = o.cons_to_prim(Y)
        for k, v in enumerate(w.vapors):
            for l in range(nc):
                Y2 = Y.copy()
                drho = 0.3 * Y[1 + k] * rs.uniform(-1, 1)
                Y2[1 + k] -= drho
                Y2[1 + nvap + k * nc + l] += drho
                _, T1, _ = o.cons_to_prim(Y2)
                Rk = w.R_d / v.eps
                dc = v.cond[l].sigma_v * c_vd - (v.sigma_v * c_vd + Rk)
                L = v.cond[l].L_ref - dc * (T0 - v.T_ref)
                Cv_after = c_vd * (Y2[0] + sum(vv.sigma_v * Y2[1 + i] for i, vv in enumerate(w.vapors))
                                   + sum(vv.cond[j].sigma_v * Y2[1 + nvap + i * nc + j]
                                         for i, vv in enumerate(w.vapors) for j in range(nc)))
                assert T1 - T0 == pytest.approx(drho * (L - Rk * T0) / Cv_after,
                                                rel=1e-9, abs=1e-12 * T0)
