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
def test_overlapped_recomputation_repeats_bitwise(torch, dtype):
    """With several checkpoint segments the next segment is recomputed on a second stream
    while the current one is transposed; two adjoint runs over the same recording (the second
    reusing the streams and events of the first) and the run that keeps every stage input
    give the same vector bit for bit."""
    from paper_1901_02955_gb300 import Context
    w = cases()["bubble_walls_ragged"]
    dt = Oracle(w).dt_cfl(w.Y, 0.8)
    ft = np.float32 if dtype == "f32" else np.float64
    lam = np.random.default_rng(45).normal(size=w.Y.shape).astype(ft)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(w.Y)
    ctx.record(9, ckpt_every=2, dt_fixed=dt)
    a = ctx.step_adjoint(9, lam)
    b = ctx.step_adjoint(9, lam)
    ctx.set_state(w.Y)
    ctx.record(9, ckpt_every=0, dt_fixed=dt)
    c = ctx.step_adjoint(9, lam)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


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


def dry_theta_setup(torch, n, moving, seed=46):
    """Warm bubble on n x n cells as a potential-temperature field theta_0 on the reference
    pressure, optionally with a seeded random velocity field of +-2 m/s per component."""
    w = W.warm_bubble(n=n)
    pk = torch.tensor(0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:]), dtype=torch.float64,
                      device="cuda")
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    T = w.Y[-1] * (w.gamma_d - 1.0) / (w.R_d * w.Y[0])  # at rest: p = (gamma - 1) rho e
    theta0 = torch.tensor(T * (1e5 / pk.cpu().numpy()[:, None, None]) ** kappa,
                          dtype=torch.float64, device="cuda")
    vel = None
    if moving:
        rs = np.random.default_rng(seed)
        vel = torch.tensor(rs.uniform(-2.0, 2.0, size=(2,) + theta0.shape), device="cuda")
    return w, pk, theta0, vel


def directional_checks(torch, J_cells, theta0, grad, ndir, seed, h=1e-4):
    """Adjoint directional derivatives grad . d against central differences of J along ndir
    seeded Gaussian directions d. J_cells(theta) returns J's per-cell terms (summed after the
    difference: J is a large sum against differences of order h, so the difference of two
    sums would carry the sums' rounding). Returns per direction (g, rich, fd_h, fd_2h): the
    adjoint value, the Richardson extrapolation (4 fd_h - fd_2h) / 3 and the two central
    differences."""
    out = []
    rs = np.random.default_rng(seed)
    for _ in range(ndir):
        d = torch.tensor(rs.normal(size=tuple(theta0.shape)), device="cuda",
                         dtype=theta0.dtype)
        with torch.no_grad():
            def fd(hh):
                return float((J_cells(theta0 + hh * d) - J_cells(theta0 - hh * d)).sum()) / (2 * hh)
            f1, f2 = fd(h), fd(2 * h)
        out.append((float((grad * d).sum()), (4.0 * f1 - f2) / 3.0, f1, f2))
    return out


def smooth_along(f1, f2, rtol=1e-6, floor=0.0):
    """A central difference of a smooth J changes with h only at O(h^2) (relative ~1e-8 for
    h = 1e-4 K here); one whose stencil straddles a kink of J (an LMARS upwind switch at
    u* = 0, a cloud edge) changes at first order in the kink's jump. The two differences at
    h and 2h disagreeing beyond rtol therefore marks a direction along which J is not smooth
    within +-2h, where no derivative exists to compare with."""
    return abs(f1 - f2) <= rtol * max(abs(f1), floor)


def dry_ke_gradient(torch, n, nsteps, ckpt, ndir, moving, dtype="f64", dt=None, seed=45):
    """dJ/dtheta_0 of the final kinetic energy through torch.autograd (initial-state map in
    torch, steps and adjoint in the library) and its directional checks."""
    from paper_1901_02955_gb300 import Context
    from paper_1901_02955_gb300.autograd import SnapSteps, dry_state_from_theta, kinetic_energy
    w, pk, theta0, vel = dry_theta_setup(torch, n, moving)
    ctx = Context(w, dtype=dtype)
    if dt is None:
        dt = 0.5 * Oracle(w).dt_cfl(w.Y, 0.8)
    vol = w.dx * w.dz
    tdt = torch.float32 if dtype == "f32" else torch.float64

    def final(theta):
        Y0 = dry_state_from_theta(theta, pk, w.R_d, w.gamma_d, velocity=vel)
        return SnapSteps.apply(Y0.to(tdt).contiguous(), ctx, nsteps, ckpt, dt)

    def ke_cells(Y):
        Y = Y.double()
        return 0.5 * (Y[1:-1] ** 2).sum(dim=0) / Y[0] * vol

    th = theta0.clone().requires_grad_(True)
    kinetic_energy(final(th).double(), vol).backward()
    grad = th.grad.detach()
    checks = directional_checks(torch, lambda t: ke_cells(final(t)), theta0, grad, ndir,
                                seed) if ndir else []
    ctx.close()
    return grad, checks


def assert_directions(checks, grad, tol, min_smooth=1.0):
    """Every direction along which J is smooth within the differences' stencil agrees to tol
    (relative, with a floor of 1 % of |grad| for directions nearly orthogonal to it: g = grad
    . d over Gaussian d has standard deviation |grad|); at least min_smooth of them are
    smooth. Returns the fraction of directions that straddle a kink."""
    floor = 0.01 * float(grad.norm())
    smooth = [smooth_along(f1, f2, 1e-6, floor) for _, _, f1, f2 in checks]
    for (g, rich, f1, f2), ok in zip(checks, smooth):
        if ok:
            assert abs(rich - g) <= tol * max(abs(g), floor), (rich, g, f1, f2)
    frac_kink = 1.0 - sum(smooth) / len(smooth)
    assert 1.0 - frac_kink >= min_smooth, frac_kink
    return frac_kink


def theta_gradient_check(torch, moving, tol, ndir=4):
    grad, checks = dry_ke_gradient(torch, 48, 12, 5, ndir, moving)
    floor = 0.01 * float(grad.norm())
    for g, rich, _, _ in checks:
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
