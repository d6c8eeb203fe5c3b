"""Parity of the CUDA library (through the C ABI) with the FP64 oracle on seeded inputs.

Error of each field: relative L2 over the domain, ||GPU - oracle|| / ||reference||, with the
reference the larger of the oracle's and the input's norm of: the field itself for dry air,
vapours and energy; the species total (vapour + its condensates) for a condensate, the
quantity the saturation adjustment's stopping tolerance is relative to; and for each momentum
component the whole momentum vector or, if larger, ||rho|| x 1 m/s (a flow starting from rest
has momenta near zero after one step, where both sides only round the hydrostatic pressure,
~1e-16 x 1e5 Pa). Bounds: 1e-12 for the FP64 path; 1e-5 for the FP32 path, whose input is the
FP32-rounded state given to both sides."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

from helpers import uniform_column

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()


def Context(*a, **k):
    from paper_1901_02955_gb300 import Context as C
    return C(*a, **k)


def rounded(w, dtype):
    return w.Y.astype(np.float32).astype(np.float64) if dtype == "f32" else w.Y.copy()


def reference_fields(nv, nvap, ncond):
    """For each field, the fields whose joint norm is its error reference."""
    im0 = 1 + nvap + nvap * ncond
    ref = [[0]] + [[1 + i] for i in range(nvap)]
    for i in range(nvap):
        tot = [1 + i] + [1 + nvap + i * ncond + j for j in range(ncond)]
        ref += [tot for _ in range(ncond)]
    mom = list(range(im0, nv - 1))
    ref += [mom for _ in mom] + [[nv - 1]]
    return ref


def rel_errs(Yg, Yo, Y0, w=None):
    nv = Yo.shape[0]
    nvap = len(w.vapors) if w is not None else 0
    ncond = w.ncond if w is not None else 0
    if w is None:  # infer from the field count: dry
        nvap = ncond = 0
    out = []
    im0 = 1 + nvap + nvap * ncond
    rho_norm = np.linalg.norm(Yo[:im0].sum(axis=0))
    for f, ref in enumerate(reference_fields(nv, nvap, ncond)):
        den = max(np.linalg.norm(Yo[ref]), np.linalg.norm(Y0[ref]), 1e-300)
        if im0 <= f < nv - 1:
            den = max(den, rho_norm * 1.0)
        out.append(np.linalg.norm(Yg[f] - Yo[f]) / den)
    return np.array(out)


def cases():
    return {
        "warm_bubble_40": lambda: W.add_random_motion(W.warm_bubble(n=40)),
        "density_current_visc": lambda: W.add_random_motion(
            W.density_current(nx=70, nz=37, dtype="f64")),
        "moist_2d": lambda: W.add_random_motion(W.moist_bubble(nx=45, nz=35)),
        "jovian_3d": lambda: W.add_random_motion(W.jovian(nx=13, ny=11, nz=18)),
        "dry_3d": lambda: W.add_random_motion(W.dry_bubble_3d(nx=19, ny=10, nz=9)),
        "periodic_strip": lambda: W.add_random_motion(uniform_column(
            37, 1000.0, lambda x: 1.0 + 0.1 * np.sin(2 * np.pi * x / 1000.0),
            lambda x: 5.0 + 0 * x, lambda x: 0 * x, nz=5)),
        "minimum_3x3": lambda: W.add_random_motion(W.warm_bubble(n=3)),
    }


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", list(cases()))
def test_two_steps_match_oracle(name, dtype):
    w = cases()[name]()
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    dt = o.dt_cfl(Y0)
    Yo, _, rc = o.step(Y0, 2, dt=dt)
    assert rc >= 0
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ctx.step(2, dt_fixed=dt)
    Yg = ctx.get_state()
    err = rel_errs(Yg, Yo, Y0, w)
    assert np.all(err <= TOL[dtype]), dict(zip(w.field_names(), err))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", ["warm_bubble_40", "jovian_3d", "moist_2d"])
def test_cfl_steps_match_oracle(name, dtype):
    """Three steps, each with its own CFL time step from the state at step start."""
    w = cases()[name]()
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    Yo, dto, _ = o.step(Y0, 3, dt=0.0)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    dtg = ctx.step(3)
    assert dtg == pytest.approx(dto, rel=1e-12 if dtype == "f64" else 1e-5)
    err = rel_errs(ctx.get_state(), Yo, Y0, w)
    assert np.all(err <= TOL[dtype]), dict(zip(w.field_names(), err))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", list(cases()))
def test_dt_and_budget_match_oracle(name, dtype):
    w = cases()[name]()
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    assert ctx.compute_dt() == pytest.approx(o.dt_cfl(Y0), rel=1e-13 if dtype == "f64" else 1e-6)
    b = ctx.budget()
    bo = o.budget(Y0)
    np.testing.assert_allclose(b["total"], bo[:-1], rtol=1e-12 if dtype == "f64" else 1e-6,
                               atol=1e-12 * np.abs(bo[:-1]).max())
    assert b["energy_with_potential"] == pytest.approx(bo[-1], rel=1e-12 if dtype == "f64" else 1e-6)


def supersaturated(w, seed=5):
    """Random redistribution between vapour and cloud: some cells super-, some subsaturated."""
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    nvap, nc = len(w.vapors), w.ncond
    for i in range(nvap):
        f = rs.uniform(0.5, 1.8, size=Y[1 + i].shape)
        tot = Y[1 + i] * f
        cf = np.where(rs.uniform(size=tot.shape) < 0.5, rs.uniform(0, 0.4, size=tot.shape), 0.0)
        Y[1 + i] = tot * (1 - cf)
        Y[1 + nvap + i * nc] = tot * cf
    return w.with_state(Y)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("make", [lambda: W.moist_bubble(nx=33, nz=17),
                                  lambda: W.jovian(nx=9, ny=9, nz=40)])
def test_saturation_adjustment_kernel_matches_oracle(make, dtype):
    w = supersaturated(make())
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ctx.saturation_adjust()
    Yg = ctx.get_state()
    flat = Y0.reshape(o.nv, -1)
    want = np.stack([o.satadj_cell(flat[:, c])[0] for c in range(flat.shape[1])], axis=1)
    want = want.reshape(Y0.shape)
    err = rel_errs(Yg, want, Y0, w)
    assert np.all(err <= (1e-12 if dtype == "f64" else 1e-5)), dict(zip(w.field_names(), err))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ensemble_of_uneven_domains_matches_oracle(dtype):
    ws = [W.add_random_motion(W.moist_bubble(n=n, A=A, R=R), seed=W.BASE_SEED + n)
          for n, A, R in [(20, 0.5, 200.0), (33, 1.5, 300.0), (48, 1.0, 150.0)]]
    ctx = Context(ws, dtype=dtype)
    Y0s = [rounded(w, dtype) for w in ws]
    for d, Y0 in enumerate(Y0s):
        ctx.set_state(Y0, domain=d)
    ctx.step(2)
    for d, (w, Y0) in enumerate(zip(ws, Y0s)):
        Yo, _, _ = Oracle(w).step(Y0, 2, dt=0.0)
        err = rel_errs(ctx.get_state(domain=d), Yo, Y0, w)
        assert np.all(err <= TOL[dtype]), (d, err)


def test_graph_and_plain_launches_agree_bitwise():
    w = cases()["jovian_3d"]()
    outs = []
    for graph in (True, False, True):
        ctx = Context(w, dtype="f32")
        ctx.use_graph(graph)
        ctx.set_state(w.Y)
        ctx.step(3)
        outs.append(ctx.get_state())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_device_tensor_state_round_trip():
    import torch
    w = cases()["moist_2d"]()
    ctx = Context(w, dtype="f32")
    t = torch.from_numpy(w.Y).cuda()
    ctx.set_state(t)
    out = torch.empty_like(t)
    ctx.get_state(out=out)
    got = out.cpu().numpy()
    # FP32 storage: the energy is held as its departure from the level's reference, so the
    # round trip is at least as accurate as rounding each value to FP32
    np.testing.assert_allclose(got, w.Y, rtol=6e-8, atol=0)
    np.testing.assert_array_equal(got[:-1], w.Y[:-1].astype(np.float32).astype(np.float64))


def test_nonfinite_input_is_reported():
    from paper_1901_02955_gb300 import SnapError, capi
    w = W.warm_bubble(n=40)
    Y = w.Y.copy()
    Y[3, 5, 0, 7] = np.nan
    ctx = Context(w, dtype="f64")
    ctx.set_state(Y)
    with pytest.raises(SnapError) as e:
        ctx.step(1, dt_fixed=0.01)
    assert e.value.code == capi.ENONFINITE


def test_satadj_sweep_limit_is_reported():
    from paper_1901_02955_gb300 import SnapError, capi
    w = dataclasses.replace(supersaturated(W.moist_bubble(n=16)), satadj_max_iter=1)
    ctx = Context(w, dtype="f64")
    ctx.set_state(w.Y)
    with pytest.raises(SnapError) as e:
        ctx.saturation_adjust()
    assert e.value.code == capi.ENOCONV


@pytest.mark.parametrize("make", [lambda: W.jovian(nx=4, ny=4, nz=8),
                                  lambda: W.density_current(nx=16, nz=8)],
                         ids=["moist_3d", "viscous"])
def test_adjoint_entry_reports_not_supported(make):
    import ctypes
    from paper_1901_02955_gb300 import capi
    w = make()
    ctx = Context(w)
    buf = np.zeros(w.Y.shape)
    out = np.zeros(w.Y.shape)
    assert ctx.lib.snap_record(ctx._ptr, 1, 1, 0.0) == capi.ENOTSUP
    rc = ctx.lib.snap_step_adjoint(ctx._ptr, 1, ctypes.c_void_p(buf.ctypes.data),
                                   ctypes.c_void_p(out.ctypes.data), capi.F64, None)
    assert rc == capi.ENOTSUP


# ------------------------------------------------------------------------------------------
# full-size workloads in the launch configuration bench.py times
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_density_current_full_size_one_step(dtype):
    w = W.density_current(dtype=dtype)
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    dt = o.dt_cfl(Y0)
    Yo, _, _ = o.step(Y0, 1, dt=dt)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ctx.step(1, dt_fixed=dt)
    err = rel_errs(ctx.get_state(), Yo, Y0, w)
    assert np.all(err <= TOL[dtype]), dict(zip(w.field_names(), err))


def test_jovian_full_size_sampled_stage_and_conservation():
    """256 x 256 x 128 FP32: stage 0 at sampled cells against the oracle on 7-cell windows
    (a cell's stage result depends only on cells within 3 along each axis), and the
    horizontal-periodic, vertical-wall budget conserved over one step."""
    import torch
    w = W.jovian()
    Y0 = w.Y.astype(np.float32)
    Yd = Y0.astype(np.float64)
    ctx = Context(w, dtype="f32")
    ctx.set_state(Y0)
    b0 = ctx.budget()
    dt = ctx.compute_dt()
    ctx.stage(0, dt_fixed=dt)
    torch.cuda.synchronize()
    Y1 = ctx.buffer_view(slot=1).cpu().numpy().astype(np.float64)
    pk = 0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:])
    Y1[-1] += (pk / (w.gamma_d - 1.0))[:, None, None]  # stored layout -> total energy
    rs = np.random.default_rng(3)
    samples = []
    for _ in range(24):
        i, j = int(rs.integers(w.nx)), int(rs.integers(w.ny))
        k = int(rs.integers(3, w.nz - 3))
        ii = [(i + s) % w.nx for s in range(-3, 4)]
        jj = [(j + s) % w.ny for s in range(-3, 4)]
        win = Yd[:, k - 3:k + 4][:, :, jj][:, :, :, ii]
        ww = dataclasses.replace(w, nx=7, ny=7, nz=7, Y=np.ascontiguousarray(win),
                                 rho_bar=w.rho_bar[k - 3:k + 4],
                                 p_bar_face=w.p_bar_face[k - 3:k + 5])
        out, _ = Oracle(ww).stage(0, ww.Y, ww.Y, dt)
        samples.append((out[:, 3, 3, 3], Y1[:, k, j, i]))
    want = np.array([s[0] for s in samples])
    got = np.array([s[1] for s in samples])
    scale = np.maximum(np.abs(Yd).reshape(w.nv, -1).max(axis=1), np.abs(want).max(axis=0))
    for i in range(2):  # condensates are judged against their vapour's magnitude
        for j in range(2):
            scale[3 + 2 * i + j] = max(scale[3 + 2 * i + j], scale[1 + i])
    # momentum components against the momentum vector, floored at max(rho) x 1 m/s as in
    # rel_errs (the column starts at rest)
    scale[7:10] = max(scale[7:10].max(), scale[:7].sum() * 1.0)
    assert np.all(np.abs(got - want) <= 1e-5 * scale), np.abs(got - want).max(axis=0) / scale
    # one full step conserves dry air and rho e + rho g z (periodic x, y; walls in z)
    ctx.set_state(Y0)
    ctx.step(1, dt_fixed=dt)
    b1 = ctx.budget()
    assert b1["total"][0] == pytest.approx(b0["total"][0], rel=2e-6)
    assert b1["energy_with_potential"] == pytest.approx(b0["energy_with_potential"], rel=2e-6)
