"""Pins of the oracle's Kessler microphysics (Sec. 3, backward Euler of Eq. x_n+1) and of the
sedimentation fluxes (Sec. 2, Eq. d3 and the momentum and energy equations with terminal
velocities): closed-form backward Euler solutions of the linear and quadratic cases, the
implicit equation itself evaluated independently, conservation, positivity, and the
sedimentation tendency of a resting rain layer."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

K_JOVIAN = (1e9, 1e-4, 0.0, 1e-2)  # k1..k4 of the paper's Jovian run (Sec. 5)


def earth(**kw):
    w = W.moist_bubble(n=8)
    return dataclasses.replace(w, **kw)


def cell(w, rs, fv=1.0, fc=0.0, fr=0.0, motion=True):
    """One cell of the workload with vapour scaled by fv and cloud / rain set as fractions of
    the vapour, energy rebuilt for the same temperature, optional random motion."""
    o = Oracle(w)
    y = w.Y.reshape(w.nv, -1)[:, rs.integers(w.Y[0].size)].copy()
    X, T, _ = o.cons_to_prim(y)
    v = y[1] * fv
    y[1], y[2], y[3] = v, v * fc, v * fr
    X2, _, _ = o.cons_to_prim(y)
    X2[-1] = X[-1] * (y[:4].sum() / X[0])  # keep roughly the same temperature
    if motion:
        X2[4:-1] = rs.normal(0, 3.0, 2)
    return o.prim_to_cons(X2)


def mixing(y):
    rho = y[:4].sum()
    return np.array([y[1], y[2], y[3]]) / rho, rho


def test_autoconversion_alone_is_the_closed_form_backward_euler_step():
    w = earth(kessler_k=(0.0, 3e-3, 0.0, 0.0), kessler_tol=1e-15)
    o = Oracle(w)
    rs = np.random.default_rng(61)
    for _ in range(20):
        y = cell(w, rs, fv=0.8, fc=rs.uniform(0.01, 0.3), fr=rs.uniform(0, 0.2))
        (qv, qc, qr), rho = mixing(y)
        dt = rs.uniform(1.0, 500.0)
        out, it = o.kessler_cell(y, dt)
        assert it > 0
        (pv, pc, pr), _ = mixing(out)
        qc_new = qc / (1.0 + 3e-3 * dt)
        assert pv == pytest.approx(qv, rel=1e-14)
        assert pc == pytest.approx(qc_new, rel=1e-12)
        assert pr == pytest.approx(qr + qc - qc_new, rel=1e-12)


def test_accretion_and_autoconversion_match_the_quadratic_root():
    k2, k3 = 1e-3, 2.0
    w = earth(kessler_k=(0.0, k2, k3, 0.0), kessler_tol=1e-15)
    o = Oracle(w)
    rs = np.random.default_rng(62)
    for _ in range(20):
        y = cell(w, rs, fv=0.8, fc=rs.uniform(0.05, 0.3), fr=rs.uniform(0.01, 0.3))
        (qv, qc, qr), _ = mixing(y)
        dt = rs.uniform(1.0, 200.0)
        out, it = o.kessler_cell(y, dt)
        (pv, pc, pr), _ = mixing(out)
        # c' = c - dt (k3 c' r' + k2 c'), r' = r + c - c':
        #   dt k3 c'^2 - (1 + dt k2 + dt k3 (r + c)) c' + c = 0, the smaller root (-> c/(1 + dt k2)
        #   as k3 -> 0), written without cancellation
        a, B = k3 * dt, 1.0 + dt * k2 + k3 * dt * (qr + qc)
        root = 2 * qc / (B + np.sqrt(B * B - 4 * a * qc))
        assert pc == pytest.approx(root, rel=1e-10)
        assert pr == pytest.approx(qr + qc - root, rel=1e-10)
        assert pv == pytest.approx(qv, rel=1e-14)


@pytest.mark.parametrize("sat", [False, True])
def test_result_solves_the_implicit_equation(sat):
    """(X' - X)/dt = Phi(X') with q* evaluated independently at the temperature of the new
    state (the backward Euler equation itself, checked to the iteration tolerance)."""
    k = (5.0, 1e-3, 1.0, 1e-2)
    w = earth(kessler_k=k, kessler_tol=1e-13)  # the stiff k1 term leaves ~1e-15 of noise
    o = Oracle(w)
    rs = np.random.default_rng(63 + sat)
    vap = w.vapors[0]
    for _ in range(20):
        y = cell(w, rs, fv=rs.uniform(1.05, 1.3) if sat else rs.uniform(0.5, 0.9),
                 fc=rs.uniform(0.0, 0.2), fr=rs.uniform(0.01, 0.3))
        (qv, qc, qr), rho = mixing(y)
        dt = rs.uniform(0.5, 5.0)
        out, it = o.kessler_cell(y, dt)
        assert it > 0
        (pv, pc, pr), _ = mixing(out)
        _, T, _ = o.cons_to_prim(out)
        qs = o.sat_pressure(0, T) / ((w.R_d / vap.eps) * T * rho)
        sup = pv - qs
        k1, k2, k3, k4 = k
        phi = np.array([-k1 * max(sup, 0) + k4 * pr * max(-sup, 0),
                        k1 * max(sup, 0) - k3 * pc * pr - k2 * pc,
                        -k4 * pr * max(-sup, 0) + k3 * pc * pr + k2 * pc])
        res = (np.array([pv, pc, pr]) - np.array([qv, qc, qr])) / dt - phi
        assert np.abs(res).max() <= 1e-9 * (qv + qc + qr) / dt


def test_conservation_and_positivity():
    w = earth(kessler_k=K_JOVIAN)
    o = Oracle(w)
    rs = np.random.default_rng(65)
    for _ in range(50):
        y = cell(w, rs, fv=rs.uniform(0.3, 1.5), fc=rs.uniform(0, 0.5), fr=rs.uniform(0, 0.5))
        out, it = o.kessler_cell(y, rs.uniform(0.1, 30.0))
        assert it > 0
        assert out[0] == y[0] and np.all(out[4:] == y[4:])  # rho_d, momenta, rho e untouched
        assert out[1:4].sum() == pytest.approx(y[1:4].sum(), rel=1e-14)
        assert np.all(out[1:4] >= -1e-18 * y[1:4].sum())


def test_fast_condensation_reaches_saturation():
    """k1 = 1e9 (the paper's Jovian value): a supersaturated cell ends at q_v = q*(T')."""
    w = earth(kessler_k=(1e9, 0.0, 0.0, 0.0), kessler_tol=1e-13)
    o = Oracle(w)
    rs = np.random.default_rng(66)
    vap = w.vapors[0]
    n = 0
    while n < 10:
        y = cell(w, rs, fv=rs.uniform(1.1, 1.6))
        _, T0, _ = o.cons_to_prim(y)
        if y[1] <= o.sat_pressure(0, T0) / ((w.R_d / vap.eps) * T0):
            continue  # not supersaturated
        n += 1
        out, it = o.kessler_cell(y, 1.0)
        assert it > 0
        # the same equilibrium as the saturation adjustment of App. D
        ya, _ = o.satadj_cell(y)
        assert out[1] == pytest.approx(ya[1], rel=1e-8)
        _, T, _ = o.cons_to_prim(out)
        rho = out[:4].sum()
        qs = o.sat_pressure(0, T) / ((w.R_d / vap.eps) * T * rho)
        assert out[1] / rho == pytest.approx(qs, rel=1e-8)
        assert out[2] > 0


def rain_column(nz=12, wt=-5.0, qr=None):
    """A column at rest whose total density and rain mixing ratio are linear in height (WENO5
    reproduces linear data exactly, so every face value is the mean of its two cells) and
    whose pressure equals the reference (p' = 0, so u* = 0 at every face); qr may give
    another rain profile."""
    w0 = W.moist_bubble(n=8, nz=nz, A=0.0)
    o = Oracle(w0)
    pk = 0.5 * (w0.p_bar_face[:-1] + w0.p_bar_face[1:])
    k = np.arange(nz)
    rho = 1.15 - 0.004 * k
    qr = 0.002 + 0.0003 * k if qr is None else qr
    Y = np.zeros_like(w0.Y)
    for kk in range(nz):
        X = np.array([rho[kk], 0.01, 0.0, qr[kk], 0.0, 0.0, pk[kk]])
        Y[:, kk, 0, :] = o.prim_to_cons(X)[:, None]
    return dataclasses.replace(w0.with_state(Y), w_term=(0.0, wt)), rho, qr


def test_resting_rain_layer_sediments_through_the_column():
    """Rain at rest: the rain tendency is the sedimentation flux difference alone, w^t times
    the face values of rho and q_r (means of the two cells for linear data, away from the
    walls' mirror ghosts); nothing crosses the walls, so the column total does not change."""
    wt = -5.0
    w, rho, qr = rain_column(wt=wt)
    o = Oracle(w)
    L = o.rhs(w.Y)
    flux = np.zeros(w.nz + 1)
    flux[1:-1] = wt * 0.5 * (rho[1:] + rho[:-1]) * 0.5 * (qr[1:] + qr[:-1])
    want = -(flux[1:] - flux[:-1]) / w.dz
    # cells whose faces reconstruct from interior cells only (mirror ghosts are not linear)
    inner = slice(3, w.nz - 3)
    for i in range(w.nx):
        got = L[3][:, 0, i]
        assert got[inner] == pytest.approx(want[inner], rel=1e-9)
    assert abs(L[3].sum()) <= 1e-12 * np.abs(L[3]).sum()


def test_rain_falls_out_of_a_slab_from_above():
    """Rain only in the upper half of a resting column: the cell below the slab's lower edge
    receives w^t rho_r from the slab (the flux takes the state above, where the rain is)."""
    wt, nz = -5.0, 12
    top = nz // 2
    # a heavy slab (q_r = 0.05, far above the WENO epsilon, so its edge stays sharp) in
    # pressure equilibrium with the reference
    w, rho, qr = rain_column(nz=nz, wt=wt, qr=np.where(np.arange(nz) >= top, 0.05, 0.0))
    L = Oracle(w).rhs(w.Y)
    gain = L[3][top - 1, 0, :]
    want = -wt * w.Y[3][top, 0, :] / w.dz
    assert np.all(gain > 0.9 * want) and np.all(gain < 1.1 * want)


def test_sedimentation_is_galilean_invariant():
    """A uniform horizontal velocity U added to the resting rain column (periodic in x) changes
    the tendencies
    only by what the moving frame requires: d(rho u)/dt = U d(rho)/dt and d(rho e)/dt gains
    U^2/2 d(rho)/dt, rho the total density (the rain carries its kinetic energy)."""
    w, _, _ = rain_column()
    w = dataclasses.replace(w, bc=(W.PERIODIC, W.PERIODIC) + tuple(w.bc[2:]))
    o = Oracle(w)
    U = 7.0
    Y = w.Y.copy()
    rho = Y[:4].sum(axis=0)
    Y[4] = rho * U
    Y[-1] += 0.5 * rho * U * U
    L0, L1 = o.rhs(w.Y), o.rhs(Y)
    drho = L0[:4].sum(axis=0)
    scale = np.abs(L0[-1]).max()
    assert L1[4] == pytest.approx(U * drho, rel=1e-9, abs=1e-12 * np.abs(U * drho).max())
    assert L1[-1] - L0[-1] == pytest.approx(0.5 * U * U * drho, rel=1e-6, abs=1e-9 * scale)


def test_sedimentation_conserves_species_mass_and_total_energy():
    w = dataclasses.replace(W.add_random_motion(W.moist_bubble(n=10)), w_term=(0.0, -8.0))
    Y = w.Y.copy()
    Y[3] = 0.2 * Y[1]
    Y[2] = 0.05 * Y[1]
    w = w.with_state(Y)
    o = Oracle(w)
    b0 = o.budget(w.Y)
    Y1 = o.step(w.Y, 5, dt=0.5 * o.dt_cfl(w.Y, 0.8))[0]
    b1 = o.budget(Y1)
    # dry air, the species total (the adjustment moves vapour and cloud) and sum(rho e + rho g z)
    assert b1[0] == pytest.approx(b0[0], rel=1e-13)
    assert b1[1:4].sum() == pytest.approx(b0[1:4].sum(), rel=1e-13)
    assert b1[-1] == pytest.approx(b0[-1], rel=1e-12)
    assert not np.allclose(Y1[3], w.Y[3])  # the rain moved


def test_kessler_step_conserves_mass_and_energy():
    w = dataclasses.replace(W.add_random_motion(W.moist_adjoint_bubble(n=12)),
                            w_term=(0.0, -5.0), kessler_k=K_JOVIAN)
    o = Oracle(w)
    b0 = o.budget(w.Y)
    Y1, _, rc = o.step(w.Y, 4, dt=o.dt_cfl(w.Y, 0.8))
    assert rc >= 0
    b1 = o.budget(Y1)
    assert b1[0] == pytest.approx(b0[0], rel=1e-13)
    assert b1[1:4].sum() == pytest.approx(b0[1:4].sum(), rel=1e-13)
    assert b1[-1] == pytest.approx(b0[-1], rel=1e-12)
    assert Y1[3].max() > 0  # rain formed from the cloud


def test_adjoint_refuses_sedimentation_and_microphysics():
    w, _, _ = rain_column()
    with pytest.raises(RuntimeError):
        Oracle(w).rhs_adjoint(w.Y, np.zeros_like(w.Y))
    w2 = dataclasses.replace(W.moist_bubble(n=8), kessler_k=K_JOVIAN)
    with pytest.raises(RuntimeError):
        Oracle(w2).step_adjoint(w2.Y, 0.1, np.zeros_like(w2.Y))
