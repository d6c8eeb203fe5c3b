"""Discrete adjoint in the CUDA library, dry and moist, against the
oracle's adjoint (whose own pins are central differences of the oracle step), against central
differences of the library's forward run, between FP32 and FP64, and across checkpoint
spacings; and the gradients of the final kinetic energy and of a column's cloud mass with
respect to the initial potential temperature through torch.autograd against central
differences."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

from test_oracle_adjoint import with_pressure_waves

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()
    return t


def cases():
    return {
        "bubble_walls_ragged": with_pressure_waves(W.add_random_motion(W.warm_bubble(n=37))),
        "bubble_3d_periodic": with_pressure_waves(
            W.add_random_motion(W.dry_bubble_3d(nx=11, ny=9, nz=7))),
    }


def oracle_adjoint(w, nsteps, dt, lam):
    o = Oracle(w)
    states = [w.Y.copy()]
    for _ in range(nsteps - 1):
        states.append(o.step(states[-1], 1, dt=dt)[0])
    for Yn in reversed(states):
        lam = o.step_adjoint(Yn, dt, lam)
    return lam


@pytest.mark.parametrize("name", list(cases()))
def test_fp64_adjoint_matches_oracle(torch, name):
    from paper_1901_02955_gb300 import Context
    w = cases()[name]
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    nsteps = 5
    lam = np.random.default_rng(41).normal(size=w.Y.shape)
    ctx = Context(w, dtype="f64")
    ctx.set_state(w.Y)
    ctx.record(nsteps, ckpt_every=2, dt_fixed=dt)
    got = ctx.step_adjoint(nsteps, lam)
    want = oracle_adjoint(w, nsteps, dt, lam)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-10, err
    # the state after the adjoint is the recorded final state
    YN = Oracle(w).step(w.Y, nsteps, dt=dt)[0]
    assert np.linalg.norm(ctx.get_state() - YN) / np.linalg.norm(YN) < 1e-12


def test_checkpoint_spacing_does_not_change_the_adjoint(torch):
    from paper_1901_02955_gb300 import Context
    w = cases()["bubble_walls_ragged"]
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    lam = np.random.default_rng(42).normal(size=w.Y.shape)
    outs, finals = [], []
    for k in (1, 3, 7, 0):  # 0: every stage input kept, nothing recomputed
        ctx = Context(w, dtype="f64")
        ctx.set_state(w.Y)
        ctx.record(7, ckpt_every=k, dt_fixed=dt)
        outs.append(ctx.step_adjoint(7, lam))
        finals.append(ctx.get_state())
    for o, y in zip(outs[1:], finals[1:]):
        assert np.array_equal(outs[0], o)
        assert np.array_equal(finals[0], y)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_recorded_cfl_steps_same_with_and_without_recomputation(torch, dtype):
    """With the time step from the CFL rule at every step, the adjoint that reads the kept
    stage inputs and the one that recomputes them from checkpoints use the same recorded
    steps and give the same vector."""
    from paper_1901_02955_gb300 import Context
    w = cases()["bubble_3d_periodic"]
    ft = np.float32 if dtype == "f32" else np.float64
    lam = np.random.default_rng(44).normal(size=w.Y.shape).astype(ft)
    outs = []
    for k in (0, 2):
        ctx = Context(w, dtype=dtype)
        ctx.set_state(w.Y)
        ctx.record(5, ckpt_every=k)
        outs.append(ctx.step_adjoint(5, lam))
    assert np.array_equal(outs[0], outs[1])


def test_fp32_adjoint_tracks_fp64_adjoint(torch):
    from paper_1901_02955_gb300 import Context
    w = cases()["bubble_walls_ragged"]
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    lam = np.random.default_rng(43).normal(size=w.Y.shape)
    res = {}
    for dt_name in ("f64", "f32"):
        ctx = Context(w, dtype=dt_name)
        ctx.set_state(w.Y)
        ctx.record(4, ckpt_every=2, dt_fixed=dt)
        res[dt_name] = ctx.step_adjoint(4, lam.astype(np.float32 if dt_name == "f32" else np.float64))
    for f in range(w.nv):
        a, b = res["f32"][f].astype(np.float64), res["f64"][f]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-30, f


def test_adjoint_dot_product_with_forward_differences(torch):
    """<lambda, (Y_N(Y0 + h v) - Y_N(Y0 - h v)) / 2h> = <lambda_0, v> with the library's own
    FP64 forward run."""
    from paper_1901_02955_gb300 import Context
    w = cases()["bubble_walls_ragged"]
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    rs = np.random.default_rng(44)
    v = rs.normal(size=w.Y.shape)
    for f in range(w.nv):
        v[f] *= 1e-3 * np.ptp(w.Y[f])
    lam = rs.normal(size=w.Y.shape)
    nsteps = 6
    ctx = Context(w, dtype="f64")

    def run(Y):
        ctx.set_state(np.ascontiguousarray(Y))
        ctx.step(nsteps, dt_fixed=dt)
        return ctx.get_state()

    def fd(h):
        return np.sum(lam * (run(w.Y + h * v) - run(w.Y - h * v)) / (2 * h))

    rich = (4.0 * fd(1e-4) - fd(2e-4)) / 3.0
    ctx.set_state(w.Y)
    ctx.record(nsteps, ckpt_every=4, dt_fixed=dt)
    lam0 = ctx.step_adjoint(nsteps, lam)
    assert rich == pytest.approx(np.sum(lam0 * v), rel=1e-6)


def theta_gradient_check(torch, moving, tol, ndir=4):
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.autograd import SnapSteps, dry_state_from_theta, kinetic_energy
    w = W.warm_bubble(n=48)
    pk = torch.tensor(0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:]), dtype=torch.float64,
                      device="cuda")
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    T = w.Y[-1] * (w.gamma_d - 1.0) / (w.R_d * w.Y[0])  # at rest: p = (gamma - 1) rho e
    theta0 = torch.tensor(T * (1e5 / pk.cpu().numpy()[:, None, None]) ** kappa,
                          dtype=torch.float64, device="cuda")
    vel = None
    if moving:
        rs = np.random.default_rng(46)
        vel = torch.tensor(rs.uniform(-2.0, 2.0, size=(2,) + theta0.shape), device="cuda")
    ctx = Context(w, dtype="f64")
    dt = 0.5 * Oracle(w).dt_cfl(w.Y, 0.8)
    nsteps = 12
    vol = w.dx * w.dz

    def final(theta):
        Y0 = dry_state_from_theta(theta, pk, w.R_d, w.gamma_d, velocity=vel)
        return SnapSteps.apply(Y0.contiguous(), ctx, nsteps, 5, dt)

    def J(theta):
        return kinetic_energy(final(theta), vol)

    def ke_cells(Y):
        return 0.5 * (Y[1:-1] ** 2).sum(dim=0) / Y[0] * vol

    th = theta0.clone().requires_grad_(True)
    J(th).backward()
    grad = th.grad.detach()
    # g = grad . d over Gaussian directions d has standard deviation |grad|; a direction that
    # is nearly orthogonal to the gradient (|g| far below that) is held to the relative
    # tolerance of 1 % of the typical size, not of its own tiny derivative
    floor = 0.01 * float(grad.norm())
    rs = np.random.default_rng(45)
    for _ in range(ndir):
        d = torch.tensor(rs.normal(size=theta0.shape), device="cuda")
        with torch.no_grad():
            def fd(h):
                # cell by cell before the sum: J ~ 1e6 against differences ~ 1e-5, so the
                # difference of the two sums would carry the sums' rounding (~1e-10)
                return float((ke_cells(final(theta0 + h * d)) -
                              ke_cells(final(theta0 - h * d))).sum()) / (2 * h)
            rich = (4.0 * fd(1e-4) - fd(2e-4)) / 3.0
        g = float((grad * d).sum())
        assert abs(rich - g) <= tol * max(abs(g), floor), (rich, g)


def test_kinetic_energy_gradient_wrt_initial_theta_moving_flow(torch):
    """dJ/dtheta_0 through torch.autograd (initial-state map in torch, steps and their
    adjoint in the library) against central differences along random directions, for a
    bubble in a random flow (no face with u* = 0, so J is differentiable)."""
    theta_gradient_check(torch, moving=True, tol=1e-6, ndir=32)


def test_kinetic_energy_gradient_wrt_initial_theta_from_rest(torch):
    """From rest u* = 0 at nearly every face, where the upwind flux has a kink: J is not
    differentiable at theta_0. The adjoint takes the mean of the one-sided derivatives face
    by face; central differences average whole products of one-sided Jacobians, which
    differ at second order in the kink jumps (~1e-3 relative here)."""
    theta_gradient_check(torch, moving=False, tol=1e-4)


# ------------------------------------------------------------------------------------------
# moist (one vapour, cloud and rain, x-z): saturation adjustment after every stage
# ------------------------------------------------------------------------------------------
def moist_case(n=20):
    """Moist adjoint bubble (cloud forms in its core at the first adjustment) with random
    motion and pressure waves; the adjustment iterated to rounding."""
    w = with_pressure_waves(W.add_random_motion(W.moist_adjoint_bubble(n=n)))
    return dataclasses.replace(w, satadj_tol=1e-14, satadj_max_iter=200)


def test_moist_fp64_adjoint_matches_oracle(torch):
    from paper_1901_02955_gb300 import Context
    w = moist_case()
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    nsteps = 4
    lam = np.random.default_rng(51).normal(size=w.Y.shape)
    ctx = Context(w, dtype="f64")
    ctx.set_state(w.Y)
    ctx.record(nsteps, ckpt_every=3, dt_fixed=dt)
    got = ctx.step_adjoint(nsteps, lam)
    assert np.sum(ctx.get_state()[2] > 0) > 20  # cloud present in the final state
    want = oracle_adjoint(w, nsteps, dt, lam)
    for f in range(w.nv):
        err = np.linalg.norm(got[f] - want[f]) / np.linalg.norm(want)
        assert err < 1e-10, (f, err)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_moist_adjoint_same_with_and_without_recomputation(torch, dtype):
    from paper_1901_02955_gb300 import Context
    w = moist_case()
    ft = np.float32 if dtype == "f32" else np.float64
    lam = np.random.default_rng(52).normal(size=w.Y.shape).astype(ft)
    outs = []
    for k in (0, 2, 5):
        ctx = Context(w, dtype=dtype)
        ctx.set_state(w.Y)
        ctx.record(5, ckpt_every=k)
        outs.append(ctx.step_adjoint(5, lam))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_moist_fp32_adjoint_tracks_fp64_adjoint(torch):
    from paper_1901_02955_gb300 import Context
    w = moist_case()
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    lam = np.random.default_rng(53).normal(size=w.Y.shape)
    res = {}
    for dt_name in ("f64", "f32"):
        ctx = Context(w, dtype=dt_name)
        ctx.set_state(w.Y)
        ctx.record(4, ckpt_every=2, dt_fixed=dt)
        res[dt_name] = ctx.step_adjoint(4, lam.astype(np.float32 if dt_name == "f32" else np.float64))
    a, b = res["f32"].astype(np.float64), res["f64"]
    assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_cloud_mass_gradient_wrt_initial_theta(torch):
    """dJ/dtheta_0 of the cloud mass of the bubble's centre column after 12 steps (cloud
    forms in the supersaturated core at the first adjustment and changes with the
    temperature there), through torch.autograd, against Richardson-extrapolated central
    differences along 16 random directions, FP64, in a random flow."""
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.autograd import (SnapSteps, moist_state_from_theta,
                                                 column_cloud_mass)
    w = dataclasses.replace(W.moist_adjoint_bubble(n=48), satadj_tol=1e-14,
                            satadj_max_iter=200)
    vap = w.vapors[0]
    c_vd = w.R_d / (w.gamma_d - 1.0)
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    pk_np = 0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:])
    T = w.Y[-1] / (c_vd * w.Y[0] + vap.sigma_v * c_vd * w.Y[1])  # at rest, no condensate
    theta0 = torch.tensor(T * (1e5 / pk_np[:, None, None]) ** kappa, device="cuda")
    qv = torch.tensor(w.Y[1] / (w.Y[0] + w.Y[1]), device="cuda")
    pk = torch.tensor(pk_np, device="cuda")
    rs = np.random.default_rng(54)
    vel = torch.tensor(rs.uniform(-2.0, 2.0, size=(2,) + theta0.shape), device="cuda")
    ctx = Context(w, dtype="f64")
    dt = 0.5 * Oracle(w).dt_cfl(w.Y, 0.8)
    nsteps = 12

    def J(theta):
        Y0 = moist_state_from_theta(theta, pk, qv, w.R_d, w.gamma_d, vap.eps, vap.sigma_v,
                                    n_cond=w.ncond, velocity=vel)
        YN = SnapSteps.apply(Y0.contiguous(), ctx, nsteps, 5, dt)
        return column_cloud_mass(YN, w.dz, i=w.nx // 2)

    th = theta0.clone().requires_grad_(True)
    j0 = J(th)
    assert j0.item() > 0.0
    j0.backward()
    grad = th.grad.detach()
    assert float(grad.abs().max()) > 0.0
    for _ in range(16):
        d = torch.tensor(rs.normal(size=theta0.shape), device="cuda")
        with torch.no_grad():
            def fd(h):
                return (J(theta0 + h * d) - J(theta0 - h * d)).item() / (2 * h)
            rich = (4.0 * fd(1e-4) - fd(2e-4)) / 3.0
        assert rich == pytest.approx(float((grad * d).sum()), rel=1e-6)
