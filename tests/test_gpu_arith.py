"""Arithmetic pieces of the stage kernels on given arguments, through the C ABI
(snap_check_rcp64, snap_check_weno): the FP64 kernels' reciprocal (Newton-Raphson from the
approximate hardware reciprocal) against IEEE division, and the kernels' WENO5 face states of
Sec. 4.2 (FP64, FP32 scalar and the packed two-variable FP32 form) against the Jiang-Shu
formula written out here in FP64 from its textbook definition: indicators
13/12 (second difference)^2 + 1/4 (first-difference combination)^2, linear weights
(0.1, 0.6, 0.3), candidates (1/3, -7/6, 11/6), (-1/6, 5/6, 1/3), (1/3, 5/6, -1/6), and the right
state as the mirror of the window."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02955_gb300 import build
    build.build()
    return t


def jiang_shu_left(a, b, c, d, e, eps):
    b0 = 13.0 / 12.0 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2
    b1 = 13.0 / 12.0 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2
    b2 = 13.0 / 12.0 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2
    q0 = a / 3.0 - 7.0 / 6.0 * b + 11.0 / 6.0 * c
    q1 = -b / 6.0 + 5.0 / 6.0 * c + d / 3.0
    q2 = c / 3.0 + 5.0 / 6.0 * d - e / 6.0
    w0, w1, w2 = 0.1 / (eps + b0) ** 2, 0.6 / (eps + b1) ** 2, 0.3 / (eps + b2) ** 2
    return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2)


def windows(seed=11, n=60000):
    """Smooth ramps and parabolas, jumps at every position of the window, random windows and
    constant ones, at scales from 1e-3 to 1e5 and with offsets large against the variation."""
    rs = np.random.default_rng(seed)
    k = np.arange(5) - 2.0
    W = []
    m = n // 6
    W.append(rs.normal(size=(m, 1)) + rs.normal(size=(m, 1)) * k + 0.1 * rs.normal(size=(m, 1)) * k ** 2)
    jump = np.zeros((m, 5))
    pos = rs.integers(1, 5, size=m)
    jump[np.arange(5)[None, :] >= pos[:, None]] = 1.0
    W.append(rs.normal(size=(m, 1)) + rs.normal(size=(m, 1)) * jump)
    W.append(rs.normal(size=(m, 5)))
    W.append(np.repeat(rs.normal(size=(m, 1)), 5, axis=1))
    W.append(1e3 + 1e-2 * rs.normal(size=(m, 5)))
    W.append(rs.normal(size=(n - 5 * m, 5)) * rs.choice([1e-3, 1.0, 1e2], size=(n - 5 * m, 1)))
    X = np.concatenate(W)
    return X * rs.choice([1e-3, 1.0, 1e3, 1e5], size=(len(X), 1))


def run_weno(torch, X, dtype, packed, eps):
    from paper_1901_02955_gb300 import capi
    tdt = torch.float64 if dtype == "f64" else torch.float32
    win = torch.tensor(X, dtype=tdt, device="cuda").contiguous()
    out = torch.empty((len(X), 2), dtype=tdt, device="cuda")
    capi.check_weno(dtype, packed, win.data_ptr(), out.data_ptr(), len(X), eps)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def reference(X, eps):
    left = jiang_shu_left(*X.T, eps)
    right = jiang_shu_left(*X[:, ::-1].T, eps)
    return np.stack([left, right], axis=1)


def test_fp64_reciprocal_matches_ieee_division(torch):
    from paper_1901_02955_gb300 import capi
    rs = np.random.default_rng(3)
    n = 1 << 20
    x = np.ldexp(1.0 + rs.random(n), rs.integers(-1000, 1000, n)) * rs.choice([-1.0, 1.0], n)
    x[:4] = [1.0, -3.0, 7.0, 0.1]
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    capi.check_rcp64(xd.data_ptr(), yd.data_ptr(), n)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ours, ieee = y[0::2], y[1::2]
    assert np.array_equal(ieee, 1.0 / x)
    assert np.all(np.abs(ours - ieee) <= np.spacing(np.abs(ieee)))  # within one ulp
    assert ours[0] == 1.0 and ours[3] == 1.0 / 0.1


def test_fp64_weno_matches_jiang_shu(torch):
    X = windows()
    eps = 1e-6
    got = run_weno(torch, X, "f64", False, eps)
    want = reference(X, eps)
    scale = np.abs(X).max(axis=1, keepdims=True)
    err = np.abs(got - want) / scale
    assert err.max() <= 1e-13, err.max()
    # constant windows reproduce the constant exactly; the two states lie within the window
    const = np.all(X == X[:, :1], axis=1)
    assert np.array_equal(got[const, 0], X[const, 2]) and np.array_equal(got[const, 1], X[const, 2])


@pytest.mark.parametrize("packed", [False, True])
def test_fp32_weno_matches_jiang_shu(torch, packed):
    X = windows(seed=12).astype(np.float32)
    eps = 1e-6
    got = run_weno(torch, X, "f32", packed, eps)
    want = reference(X.astype(np.float64), eps)
    scale = np.abs(X.astype(np.float64)).max(axis=1, keepdims=True)
    err = np.abs(got - want) / scale
    assert err.max() <= 4e-6, err.max()


def test_fp32_packed_and_scalar_forms_agree(torch):
    """The same operations in the same order, two lanes at a time: equal to within a few
    units of FP32 rounding of the window's scale (each field always takes the same form, so
    the kernels do not rely on the two being bitwise equal)."""
    X = windows(seed=13).astype(np.float32)
    a = run_weno(torch, X, "f32", True, 1e-6)
    b = run_weno(torch, X, "f32", False, 1e-6)
    scale = np.abs(X.astype(np.float64)).max(axis=1, keepdims=True)
    assert np.all(np.abs(a - b) <= 4 * np.finfo(np.float32).eps * scale)
    assert np.mean(a == b) > 0.99


def test_check_entry_points_reject_bad_arguments(torch):
    from paper_1901_02955_gb300 import SnapError, capi
    with pytest.raises(SnapError) as e:
        capi.check_weno("f64", True, 0, 0, 2, 1e-6)
    assert e.value.code == capi.EINVAL
    with pytest.raises(SnapError) as e:
        capi.check_rcp64(0, 0, 4)
    assert e.value.code == capi.EINVAL
    capi.check_rcp64(0, 0, 0)  # nothing to do
