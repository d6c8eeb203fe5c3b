"""Parity of the library's no-slip walls and fixed bottom temperature (the lower boundary of
Sec. 6) with the oracle, through the C ABI: a viscous dry x-z case (where the wall stress
and the heat flux act), a moist x-z bubble with no-slip walls on every side, and a crop of the
Jovian radiative-convective setup (Kessler microphysics, falling precipitation, cooling,
sponge, no-slip floor held at a fixed temperature). FP64 (1e-12) and FP32 (1e-5) by the
per-field relative L2 of the parity suite; conservation in a closed box; the adjoint's
refusal."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

from test_gpu_parity import TOL, rel_errs, rounded

pytestmark = pytest.mark.gpu


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


def with_rain(w, frac, seed=73):
    rs = np.random.default_rng(seed)
    Y = w.Y.copy()
    nvap, nc = len(w.vapors), w.ncond
    for i in range(nvap):
        Y[1 + nvap + i * nc + 1] = Y[1 + i] * rs.uniform(0.0, frac, size=Y[1].shape)
    return w.with_state(Y)


def cases():
    return {
        # Straka-like dry x-z strip with viscosity: no-slip floor 10 K warmer than the air
        "dry_viscous_noslip_hot_floor": lambda: dataclasses.replace(
            W.add_random_motion(W.density_current(nx=70, nz=37, dtype="f64")),
            bc=(W.REFLECT, W.NOSLIP, W.REFLECT, W.REFLECT, W.NOSLIP, W.REFLECT),
            T_bottom=310.0),
        "moist_2d_noslip_box": lambda: dataclasses.replace(
            W.add_random_motion(W.moist_bubble(nx=45, nz=35)), bc=(W.NOSLIP,) * 6),
        # the upper 200 km of the setup (0.1 bar to ~35 bar): cooling band and sponge inside
        "jovian_rce_crop": lambda: with_rain(
            W.add_random_motion(W.jovian_rce(nx=9, ny=7, nz=40, Lx=9 * 100e3 / 256,
                                             Ly=7 * 100e3 / 256, Lz=200e3)), 0.05),
    }


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", list(cases()))
def test_bottom_boundary_steps_match_oracle(name, dtype):
    w = cases()[name]()
    Y0 = rounded(w, dtype)
    o = Oracle(w)
    dt = o.dt_cfl(Y0)
    Yo, _, rc = o.step(Y0, 3, dt=dt)
    assert rc >= 0
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ctx.step(3, dt_fixed=dt)
    err = rel_errs(ctx.get_state(), Yo, Y0, w)
    assert np.all(err <= TOL[dtype]), dict(zip(w.field_names(), err))


def test_noslip_box_conserves_mass_and_energy():
    """Closed moist box with no-slip walls: dry air, each species total and the total of
    rho e + rho g z keep their sums (nothing crosses a wall)."""
    w = cases()["moist_2d_noslip_box"]()
    ctx = Context(w, dtype="f64")
    ctx.set_state(w.Y)
    b0 = ctx.budget()
    ctx.step(5)
    b1 = ctx.budget()
    assert b1["total"][0] == pytest.approx(b0["total"][0], rel=1e-13)
    assert sum(b1["total"][1:4]) == pytest.approx(sum(b0["total"][1:4]), rel=1e-12)
    assert b1["energy_with_potential"] == pytest.approx(b0["energy_with_potential"], rel=1e-12)


def test_adjoint_reports_not_supported_with_the_new_walls():
    from paper_1901_02955_gb300 import SnapError, capi
    for w in (dataclasses.replace(W.warm_bubble(n=16), bc=(W.REFLECT,) * 4 + (W.NOSLIP, W.REFLECT)),
              dataclasses.replace(W.warm_bubble(n=16), T_bottom=300.0)):
        ctx = Context(w, dtype="f64")
        ctx.set_state(w.Y)
        with pytest.raises(SnapError) as e:
            ctx.record(2, 1)
        assert e.value.code == capi.ENOTSUP
