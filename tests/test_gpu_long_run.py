"""Long FP32 runs on the GPU: nothing drifts that must not. The SSP-RK3 combine weights are
applied so that they sum to exactly one in the arithmetic type (1/3 and 2/3 rounded to FP32
sum to 1 + 3e-8, which would scale the whole state every step); the density current reaches
900 s (Sec. 5.1) with a quiescent far field and a cold front where the scheme puts it."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()


def test_fp32_mass_and_energy_do_not_drift_over_4000_steps():
    from paper_1901_02955_gb300 import Context
    w = W.warm_bubble(n=64)
    ctx = Context(w, dtype="f32")
    ctx.set_state(w.Y.astype(np.float32))
    b0 = ctx.budget()
    ctx.step_async(4000)
    b1 = ctx.budget()
    assert abs(b1["total"][0] / b0["total"][0] - 1.0) < 2e-6
    assert abs(b1["energy_with_potential"] / b0["energy_with_potential"] - 1.0) < 2e-6
    ctx.close()


def test_density_current_at_900s_fp32():
    """Potential-temperature anomaly against the 300 K background at 900 s. The far field stays
    at 300 K (largest anomaly within 0.05 K; the paper reports 0.12 K with LMARS and 1.84 K with
    HLLC); the -15 K bubble has mixed to between -10 and -8 K; the -1 K front at the surface
    lies 14-15.5 km from the centre (the FP64 run of the same case: 0.007 K, -8.9 K, 14.7 km)."""
    from paper_1901_02955_gb300 import Context
    w = W.density_current(dtype="f32")
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    ctx = Context(w, dtype="f32")
    ctx.set_state(w.Y.astype(np.float32))
    t = 0.0
    while t < 900.0 - 1e-9:
        dt = min(ctx.compute_dt(), 900.0 - t)
        ctx.step(1, dt_fixed=dt)
        t += dt
    Y = ctx.get_state()
    ctx.close()
    rho = Y[0]
    p = (w.gamma_d - 1.0) * (Y[3] - 0.5 * (Y[1] ** 2 + Y[2] ** 2) / rho)
    dth = p / (rho * w.R_d) * (1e5 / p) ** kappa - 300.0
    cold = np.nonzero(dth[0, 0] < -1.0)[0]
    front = (cold.max() + 0.5) * w.dx
    assert -0.05 < dth.max() < 0.05, dth.max()
    assert -10.0 < dth.min() < -8.0, dth.min()
    assert 14000.0 < front < 15500.0, front
