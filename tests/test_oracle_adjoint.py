"""Pins of the oracle's discrete adjoint (the transpose of its own dry step) against central
finite differences of the oracle's forward routines: <mu, dL(Y)[v]> = <dL(Y)^T mu, v> and
the same for a whole SSP-RK3 step at fixed time step."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from oracle.oracle import weno5, weno5_gradient

from helpers import uniform_column


def test_weno5_gradient_matches_finite_differences():
    rs = np.random.default_rng(31)
    for _ in range(200):
        q = rs.normal(size=5) * 10.0 ** rs.uniform(-2, 2)
        eps = 10.0 ** rs.uniform(-8, -2)
        v, g = weno5_gradient(q, eps)
        assert v == pytest.approx(weno5(q, eps), rel=1e-14, abs=1e-14)
        for j in range(5):
            h = 1e-6 * max(abs(q[j]), np.abs(q).max() * 1e-3)
            qp, qm = q.copy(), q.copy()
            qp[j] += h
            qm[j] -= h
            fd = (weno5(qp, eps) - weno5(qm, eps)) / (2 * h)
            assert g[j] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())


def with_pressure_waves(w, amp=50.0, seed=7):
    """Add a smooth pressure perturbation (a few Fourier modes, amplitude ~amp Pa) through
    the energy, so that the WENO indicators of p' are far above eps and central differences
    stay in the linear regime of the nonlinear weights (at exact hydrostatic rest p' ~ 0)."""
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    z = np.arange(w.nz)[:, None, None] / w.nz
    y = np.arange(w.ny)[None, :, None] / max(w.ny, 1)
    x = np.arange(w.nx)[None, None, :] / w.nx
    pert = np.zeros((w.nz, w.ny, w.nx))
    for _ in range(3):
        kx, ky, kz = rs.integers(1, 3, size=3)
        ph = rs.uniform(0, 2 * np.pi, size=3)
        pert += np.sin(2 * np.pi * kx * x + ph[0]) * np.cos(np.pi * kz * z + ph[2]) * \
            (np.sin(2 * np.pi * ky * y + ph[1]) if w.ny > 1 else 1.0)
    Y[-1] += amp / (w.gamma_d - 1.0) * pert
    return w.with_state(Y)


def cases():
    return {
        "bubble_walls": with_pressure_waves(W.add_random_motion(W.warm_bubble(n=12))),
        "bubble_3d_periodic": with_pressure_waves(
            W.add_random_motion(W.dry_bubble_3d(nx=7, ny=6, nz=5))),
        "strip_periodic": with_pressure_waves(W.add_random_motion(uniform_column(
            9, 1000.0, lambda x: 1.0 + 0.1 * np.sin(2 * np.pi * x / 1000.0),
            lambda x: 3.0 + 0 * x, lambda x: 0 * x, nz=4))),
    }


def direction(w, rs):
    """Random perturbation of about 1e-3 of each field's variation across the domain."""
    v = rs.normal(size=w.Y.shape)
    for f in range(w.nv):
        v[f] *= 1e-3 * (np.ptp(w.Y[f]) + 1e-12)
    return v


@pytest.mark.parametrize("name", list(cases()))
def test_rhs_adjoint_dot_product(name):
    w = cases()[name]
    o = Oracle(w)
    rs = np.random.default_rng(32)
    for _ in range(3):
        v = direction(w, rs)
        mu = rs.normal(size=w.Y.shape)
        h = 1e-4
        fd = (o.rhs(w.Y + h * v) - o.rhs(w.Y - h * v)) / (2 * h)
        lhs = np.sum(mu * fd)
        rhs = np.sum(o.rhs_adjoint(w.Y, mu) * v)
        assert lhs == pytest.approx(rhs, rel=1e-6), (lhs, rhs)


@pytest.mark.parametrize("name", list(cases()))
def test_step_adjoint_dot_product(name):
    w = cases()[name]
    o = Oracle(w)
    dt = o.dt_cfl(w.Y, 0.8)
    rs = np.random.default_rng(33)
    for _ in range(2):
        v = direction(w, rs)
        lam = rs.normal(size=w.Y.shape)
        h = 1e-4
        fd = (o.step(w.Y + h * v, 1, dt=dt)[0] - o.step(w.Y - h * v, 1, dt=dt)[0]) / (2 * h)
        lhs = np.sum(lam * fd)
        rhs = np.sum(o.step_adjoint(w.Y, dt, lam) * v)
        assert lhs == pytest.approx(rhs, rel=1e-6), (lhs, rhs)


def test_adjoint_refuses_moist_and_viscous():
    for w in (W.moist_bubble(n=8), W.density_current(nx=16, nz=8)):
        with pytest.raises(RuntimeError):
            Oracle(w).rhs_adjoint(w.Y, np.zeros_like(w.Y))


def test_step_adjoint_at_rest_uses_the_average_at_zero_face_velocity():
    """From rest every face has u* = 0, a kink of the upwind flux; the adjoint takes the mean
    of both one-sided derivatives, which is what central differences measure."""
    w = W.warm_bubble(n=12)
    o = Oracle(w)
    dt = o.dt_cfl(w.Y, 0.8)
    rs = np.random.default_rng(34)
    # perturb temperature only (energy), as a theta perturbation would
    v = np.zeros(w.Y.shape)
    v[-1] = rs.normal(size=v[-1].shape) * 1e-2
    lam = rs.normal(size=w.Y.shape)

    def fd(h):
        d = (o.step(w.Y + h * v, 1, dt=dt)[0] - o.step(w.Y - h * v, 1, dt=dt)[0]) / (2 * h)
        return np.sum(lam * d)

    rich = (4.0 * fd(1e-3) - fd(2e-3)) / 3.0  # Richardson: removes the O(h^2) term
    assert rich == pytest.approx(np.sum(o.step_adjoint(w.Y, dt, lam) * v), rel=1e-6)
