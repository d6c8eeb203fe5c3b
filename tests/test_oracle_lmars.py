"""Pins of the oracle's LMARS flux (Sec. 4.1, Eqs. rp, ru) and of its primitive/conserved
maps (App. B) against independent routes: the Euler flux of a uniform state built from the
equation of state and total energy as stated in Sec. 2, the symmetries of the Riemann
problem, and the exact Riemann solver of an ideal gas in the acoustic limit."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def dry():
    return Oracle(W.warm_bubble(n=8))


def moist():
    return Oracle(W.jovian(nx=4, ny=4, nz=8))


def indep_cons(o, X, pref):
    """Conserved vector from primitives via Sec. 2: p = (rho_d R_d + sum rho_i R_i) T and
    rho e = (rho_d c_vd + sum rho_i c_vi + sum rho_ij c_ij) T + K + sum mu_ij rho_ij."""
    w = o.w
    nvap, nc = len(w.vapors), w.ncond
    im0 = 1 + nvap + nvap * nc
    rho = X[0]
    Y = np.zeros_like(X)
    Y[1:im0] = rho * X[1:im0]
    Y[0] = rho - Y[1:im0].sum()
    nm = o.nv - 1 - im0
    Y[im0:im0 + nm] = rho * X[im0:im0 + nm]
    c_vd = w.R_d / (w.gamma_d - 1.0)
    Rsum = Y[0] * w.R_d
    Cv = Y[0] * c_vd
    A = 0.0
    for i, v in enumerate(w.vapors):
        Ri = w.R_d / v.eps
        Rsum += Y[1 + i] * Ri
        Cv += Y[1 + i] * v.sigma_v * c_vd
        cpi = v.sigma_v * c_vd + Ri
        for j, c in enumerate(v.cond):
            rij = Y[1 + nvap + i * nc + j]
            cij = c.sigma_v * c_vd
            Cv += rij * cij
            A += -(c.L_ref + (cij - cpi) * v.T_ref) * rij
    p = pref + X[-1]
    T = p / Rsum
    K = 0.5 * rho * np.sum(X[im0:im0 + nm] ** 2)
    Y[-1] = Cv * T + K + A
    return Y, T


def random_prim(o, rs, pref):
    w = o.w
    nvap, nc = len(w.vapors), w.ncond
    im0 = 1 + nvap + nvap * nc
    X = np.zeros(o.nv)
    X[0] = rs.uniform(0.2, 3.0)
    if nvap:
        X[1:1 + nvap] = rs.uniform(0, 0.03, nvap)
        X[1 + nvap:im0] = rs.uniform(0, 0.01, nvap * nc)
    X[im0:o.nv - 1] = rs.normal(0, 20.0, o.nv - 1 - im0)
    X[-1] = rs.normal(0, 300.0)  # p' about pref
    return X


def dirs(o):
    return [0, 1, 2] if o.w.ny > 1 else [0, 2]


def mom_slot(o, d):
    nvap = len(o.w.vapors)
    im0 = 1 + nvap + nvap * o.w.ncond
    if o.w.ny > 1:
        return im0 + d
    return im0 + (1 if d == 2 else 0)


@pytest.mark.parametrize("make", [dry, moist])
def test_uniform_state_gives_exact_euler_flux(make):
    o = make()
    rs = np.random.default_rng(5)
    for _ in range(50):
        pref = rs.uniform(2e4, 2e6)
        X = random_prim(o, rs, pref)
        Y, _ = indep_cons(o, X, pref)
        for d in dirs(o):
            F, us, ps = o.lmars(X, X, d, pref)
            un = X[mom_slot(o, d)]
            want = un * Y
            want[mom_slot(o, d)] += X[-1]
            want[-1] += un * (pref + X[-1])
            assert us == pytest.approx(un, rel=1e-13, abs=1e-12)
            assert ps == pytest.approx(X[-1], rel=1e-13, abs=1e-9)
            np.testing.assert_allclose(F, want, rtol=1e-11, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("make", [dry, moist])
def test_contact_at_rest_has_no_mass_or_energy_flux(make):
    o = make()
    rs = np.random.default_rng(6)
    for _ in range(50):
        pref = rs.uniform(2e4, 2e6)
        XL = random_prim(o, rs, pref)
        XR = random_prim(o, rs, pref)
        nvap = len(o.w.vapors)
        im0 = 1 + nvap + nvap * o.w.ncond
        XL[im0:-1] = 0.0
        XR[im0:-1] = 0.0
        XR[-1] = XL[-1]
        for d in dirs(o):
            F, us, ps = o.lmars(XL, XR, d, pref)
            assert us == 0.0
            expect = np.zeros(o.nv)
            expect[mom_slot(o, d)] = XL[-1]
            np.testing.assert_allclose(F, expect, atol=1e-12 * abs(XL[-1]) + 1e-300)


@pytest.mark.parametrize("make", [dry, moist])
def test_reflection_antisymmetry(make):
    """Swapping the sides and negating normal velocities negates every flux except the
    normal-momentum flux."""
    o = make()
    rs = np.random.default_rng(7)
    for _ in range(50):
        pref = rs.uniform(2e4, 2e6)
        XL, XR = random_prim(o, rs, pref), random_prim(o, rs, pref)
        for d in dirs(o):
            m = mom_slot(o, d)
            F, us, ps = o.lmars(XL, XR, d, pref)
            ML, MR = XR.copy(), XL.copy()
            ML[m] *= -1.0
            MR[m] *= -1.0
            G, vs, qs = o.lmars(ML, MR, d, pref)
            sign = -np.ones(o.nv)
            sign[m] = 1.0
            np.testing.assert_allclose(G, sign * F, rtol=1e-12, atol=1e-9 * np.abs(F).max())
            assert vs == pytest.approx(-us, rel=1e-13, abs=1e-13)
            assert qs == pytest.approx(ps, rel=1e-13, abs=1e-9)


@pytest.mark.parametrize("make", [dry, moist])
def test_mirror_wall_has_zero_normal_velocity(make):
    o = make()
    rs = np.random.default_rng(8)
    for _ in range(50):
        pref = rs.uniform(2e4, 2e6)
        XL = random_prim(o, rs, pref)
        for d in dirs(o):
            XR = XL.copy()
            XR[mom_slot(o, d)] *= -1.0
            F, us, ps = o.lmars(XL, XR, d, pref)
            assert us == 0.0
            assert F[0] == 0.0 and F[-1] == 0.0


def exact_riemann_star(rl, ul, pl, rr, ur, pr, g):
    """Star-region pressure and velocity of the exact Riemann problem of an ideal gas
    (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, ch. 4), by Newton."""
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:
            A, B = 2.0 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            f = (p - pk) * np.sqrt(A / (p + B))
            df = np.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:
            f = 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)
            df = (p / pk) ** (-(g + 1) / (2 * g)) / (rk * ck)
        return f, df

    p = 0.5 * (pl + pr)
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p -= dp
        if abs(dp) < 1e-15 * p:
            break
    f1, _ = fk(p, rl, pl, cl)
    f2, _ = fk(p, rr, pr, cr)
    return p, 0.5 * (ul + ur) + 0.5 * (f2 - f1)


def test_acoustic_limit_matches_exact_riemann_solver():
    """For jumps of relative size delta, LMARS p* and u* agree with the exact Riemann solver
    to O(delta^2): the error shrinks 4x when delta halves."""
    o = dry()
    g = o.w.gamma_d
    rs = np.random.default_rng(9)
    for _ in range(20):
        r0, p0, u0 = rs.uniform(0.5, 1.5), rs.uniform(5e4, 1.5e5), rs.normal(0, 10)
        c0 = np.sqrt(g * p0 / r0)
        jr, ju, jp = rs.normal(size=3)
        errs = []
        for delta in (1e-3, 5e-4, 2.5e-4):
            rl, rr = r0 * (1 - delta * jr), r0 * (1 + delta * jr)
            ul, ur = u0 - c0 * delta * ju, u0 + c0 * delta * ju
            pl, pr = p0 * (1 - delta * jp), p0 * (1 + delta * jp)
            XL = np.array([rl, ul, 0.0, pl - p0])
            XR = np.array([rr, ur, 0.0, pr - p0])
            F, us, ps = o.lmars(XL, XR, 0, p0)
            pe, ue = exact_riemann_star(rl, ul, pl, rr, ur, pr, g)
            errs.append((abs(p0 + ps - pe) / p0, abs(us - ue) / c0))
            assert abs(p0 + ps - pe) / p0 < 5 * delta ** 2
            assert abs(us - ue) / c0 < 5 * delta ** 2
        ratio_p = errs[0][0] / max(errs[2][0], 1e-300)
        assert ratio_p > 8 or errs[0][0] < 1e-12
