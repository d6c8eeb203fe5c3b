"""Pins of the oracle's discrete adjoint (the transpose of its own step) against central
finite differences of the oracle's forward routines: <mu, dL(Y)[v]> = <dL(Y)^T mu, v>, the
same for a whole SSP-RK3 step at fixed time step, dry and moist, and the full Jacobian of the
saturation adjustment of single cells."""
import dataclasses

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


def direction(w, rs, energy_scale=None):
    """Random perturbation of about 1e-3 of each field's variation across the domain (for
    the energy, optionally 1e-3 of a given scale: a deep column's energy varies by ~1e7
    J/m^3 with height, far more than the pressure waves its WENO weights respond to)."""
    v = rs.normal(size=w.Y.shape)
    for f in range(w.nv):
        v[f] *= 1e-3 * (np.ptp(w.Y[f]) + 1e-12)
    if energy_scale is not None:
        v[-1] *= energy_scale / (np.ptp(w.Y[-1]) + 1e-12)
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


def test_adjoint_refuses_viscous():
    w = W.density_current(nx=16, nz=8)
    with pytest.raises(RuntimeError):
        Oracle(w).rhs_adjoint(w.Y, np.zeros_like(w.Y))


def tight(w):
    """The workload with the adjustment iterated to rounding (finite differences of its
    result then measure the derivative of the equilibrium, not the stopping rule)."""
    return dataclasses.replace(w, satadj_tol=1e-14, satadj_max_iter=200)


def with_condensate(w, seed=35):
    """Moist state with cloud and precipitation in every cell (fractions of the vapour) so
    that every tracer of the moist flux and primitive map carries a nonzero value."""
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    nvap, nc = len(w.vapors), w.ncond
    for i in range(nvap):
        for j in range(nc):
            Y[1 + nvap + i * nc + j] = Y[1 + i] * rs.uniform(0.02, 0.2, size=Y[1 + i].shape)
    return w.with_state(Y)


def moist_cases():
    return {
        "moist_bubble_walls": with_pressure_waves(W.add_random_motion(
            with_condensate(W.moist_bubble(n=10)))),
        "jovian_3d_periodic": with_pressure_waves(W.add_random_motion(
            with_condensate(W.crop(W.jovian(nx=6, ny=5, nz=8, seed=W.BASE_SEED + 51), 6, 5))),
            amp=5.0),
    }


# energy perturbation scale per moist case: the pressure waves' energy amplitude
MOIST_ENERGY_SCALE = {"moist_bubble_walls": None, "jovian_3d_periodic": 5.0 / 0.4}


@pytest.mark.parametrize("name", list(moist_cases()))
def test_moist_rhs_adjoint_dot_product(name):
    w = moist_cases()[name]
    o = Oracle(w)
    rs = np.random.default_rng(36)
    for _ in range(3):
        v = direction(w, rs, MOIST_ENERGY_SCALE[name])
        mu = rs.normal(size=w.Y.shape)

        def fd(h):
            return np.sum(mu * (o.rhs(w.Y + h * v) - o.rhs(w.Y - h * v)) / (2 * h))

        # the moist sum cancels between fields ~100x larger than the total and the tracer
        # weights are strongly nonlinear: Richardson's combination of two larger steps
        # removes the O(h^2) term while the rounding of the differences stays small
        lhs = (4.0 * fd(1e-3) - fd(2e-3)) / 3.0
        rhs = np.sum(o.rhs_adjoint(w.Y, mu) * v)
        assert lhs == pytest.approx(rhs, rel=1e-6), (lhs, rhs)


def satadj_cells(w, rs, n):
    """Cells of the workload with the species totals scaled by U(0.5, 2) (some end
    saturated with cloud, some not), random cloud fraction, precipitation and motion."""
    nvap, nc = len(w.vapors), w.ncond
    Y = w.Y.reshape(w.nv, -1)
    out = []
    for _ in range(n):
        y = Y[:, rs.integers(Y.shape[1])].copy()
        for i in range(nvap):
            tot = y[1 + i] * rs.uniform(0.5, 2.0)
            fc = rs.uniform(0, 0.5)
            y[1 + i] = tot * (1 - fc)
            y[1 + nvap + i * nc] = tot * fc
            y[1 + nvap + i * nc + 1] = tot * rs.uniform(0, 0.2)
        im0 = 1 + nvap + nvap * nc
        m = rs.normal(0, 5.0, w.nv - 1 - im0) * y[:im0].sum()
        y[-1] += 0.5 * np.sum(m * m) / y[:im0].sum()
        y[im0:-1] = m
        out.append(y)
    return out


@pytest.mark.parametrize("make", [lambda: W.moist_bubble(n=16),
                                  lambda: W.jovian(nx=4, ny=4, nz=32, seed=W.BASE_SEED + 50)],
                         ids=["earth_water", "jovian_h2o_nh3"])
def test_satadj_adjoint_is_the_transposed_jacobian(make):
    """Every column of the adjustment's Jacobian by central differences at the input, against
    the adjoint evaluated at the adjusted result; cells whose saturated set changes within
    the difference step (the kink) are skipped and counted."""
    w = tight(make())
    o = Oracle(w)
    nvap, nc = len(w.vapors), w.ncond
    rs = np.random.default_rng(37)
    checked, saturated = 0, 0
    for y in satadj_cells(w, rs, 60):
        yout, it = o.satadj_cell(y)
        assert it > 0
        sets = [tuple(yy[1 + nvap + i * nc] > 0 for i in range(nvap)) for yy in (yout,)]
        J = np.zeros((w.nv, w.nv))
        kink = False
        for t in range(w.nv):
            h = 1e-6 * max(abs(y[t]), 1e-3 * np.abs(y[:1 + nvap]).max())
            yp, ym = y.copy(), y.copy()
            yp[t] += h
            ym[t] -= h
            op, _ = o.satadj_cell(yp)
            om, _ = o.satadj_cell(ym)
            for yy in (op, om):
                if tuple(yy[1 + nvap + i * nc] > 0 for i in range(nvap)) != sets[0]:
                    kink = True
            J[:, t] = (op - om) / (2 * h)
        if kink:
            continue
        checked += 1
        saturated += any(sets[0])
        for _ in range(3):
            lam = rs.normal(size=w.nv) / np.maximum(np.abs(yout), 1e-30) ** 0
            want = J.T @ lam
            got = o.satadj_adjoint_cell(yout, lam)
            scale = np.abs(J.T).dot(np.abs(lam))
            assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-12), (got, want)
    assert checked >= 40 and saturated >= 10, (checked, saturated)


def supersaturated_bubble(n=10, seed=38):
    """Moist bubble whose vapour is raised by 1.05-1.3 in half of the cells (cloud forms in
    the first adjustment there), with pressure waves and random motion."""
    w = W.add_random_motion(W.moist_bubble(n=n))
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    mask = rs.uniform(size=Y[1].shape) < 0.5
    Y[1] = np.where(mask, Y[1] * rs.uniform(1.05, 1.3, size=Y[1].shape), Y[1])
    return tight(with_pressure_waves(w.with_state(Y)))


def test_moist_step_adjoint_dot_product():
    w = supersaturated_bubble()
    o = Oracle(w)
    dt = o.dt_cfl(w.Y, 0.8)
    Y1 = o.step(w.Y, 1, dt=dt)[0]
    ncloud = int(np.sum(Y1[2] > 0))
    assert ncloud > 10
    rs = np.random.default_rng(39)
    for _ in range(3):
        v = direction(w, rs)
        lam = rs.normal(size=w.Y.shape)
        h = 1e-4
        fd = (o.step(w.Y + h * v, 1, dt=dt)[0] - o.step(w.Y - h * v, 1, dt=dt)[0]) / (2 * h)
        lhs = np.sum(lam * fd)
        rhs = np.sum(o.step_adjoint(w.Y, dt, lam) * v)
        assert lhs == pytest.approx(rhs, rel=1e-6), (lhs, rhs)


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
