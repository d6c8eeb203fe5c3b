"""The arithmetic-throughput probe (snap_probe_fma) measures a rate near the part's nominal
fused multiply-add peaks: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s, and
1.25 TFLOP/s in FP64 (clocks under load can sit below the maximum)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()


@pytest.mark.parametrize("dtype,nominal", [("f32", 80.5), ("f64", 1.25)])
def test_probe_rate_near_nominal(dtype, nominal):
    from paper_1901_02955_gb300 import capi
    t = capi.probe_fma(dtype)
    assert 0.3 * nominal < t < 1.15 * nominal, t
