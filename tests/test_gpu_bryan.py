"""The Bryan moist bubble (Sec. 5) on the GPU: steps of the saturated moist-adiabatic
background with its warm bubble against the oracle, and the library's equivalent potential
temperature diagnostic (App. A, Eq. theta_e) against the oracle's."""
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


def small():
    return W.add_random_motion(W.bryan_moist_bubble(nx=40, nz=24, Lx=4000.0, Lz=2400.0,
                                                    R=800.0, xc=2000.0, zc=800.0))


def Context(*a, **k):
    from paper_1901_02955_gb300 import Context as C
    return C(*a, **k)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_bryan_steps_match_oracle(dtype):
    w = small()
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


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_theta_e_matches_oracle(dtype):
    w = small()
    Y0 = rounded(w, dtype)
    ctx = Context(w, dtype=dtype)
    ctx.set_state(Y0)
    ctx.step(2)
    Yg = ctx.get_state()
    got = ctx.theta_e()
    want = Oracle(w).theta_e(Yg)
    assert got == pytest.approx(want, rel=1e-13 if dtype == "f64" else 2e-6)


def test_theta_e_refuses_other_species():
    from paper_1901_02955_gb300 import SnapError, capi
    w = W.jovian(nx=4, ny=4, nz=8)
    ctx = Context(w, dtype="f32")
    ctx.set_state(w.Y)
    with pytest.raises(SnapError) as e:
        ctx.theta_e()
    assert e.value.code == capi.ENOTSUP
