"""Pins of the oracle's WENO5 interpolant (Sec. 4.2, Eq. weno5) against the paper's printed
coefficients and against what the mathematics fixes (exactness, order, Jiang-Shu weights
from their integral definition, the ENO property)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.oracle import weno5, weno5_poly, weno5_weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "weno5_coefficients.txt")


def golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, *vals = line.split()
        rows[name] = [Fraction(v) for v in vals]
    return rows


def cell_avg_poly(coef, lo, hi):
    """Exact average over [lo, hi] of sum coef[n] x^n."""
    P = np.polynomial.polynomial.Polynomial(coef).integ()
    return (P(hi) - P(lo)) / (hi - lo)


def stencil_avgs(f_avg, x_face, h):
    """Cell averages of the 5 cells i-3..i+1 around the face x_face = x_{i-1/2}."""
    return np.array([f_avg(x_face + (s - 1) * h, x_face + s * h) for s in range(-2, 3)])


def test_golden_rows_are_consistent():
    g = golden()
    comb = [sum(g["linear"][k] * g[f"stencil{k}"][m] for k in range(3)) for m in range(5)]
    assert comb == g["poly"]


def test_poly_matches_paper_coefficients():
    g = golden()
    for m in range(5):
        e = np.zeros(5)
        e[m] = 1.0
        assert weno5_poly(e) == pytest.approx(float(g["poly"][m]), rel=0, abs=1e-16)


def test_candidates_match_paper_given_weights():
    g = golden()
    rs = np.random.default_rng(1)
    for _ in range(200):
        q = rs.normal(size=5) * 10.0 ** rs.uniform(-3, 3)
        w = weno5_weights(q)
        want = sum(w[k] * sum(float(g[f"stencil{k}"][m]) * q[m] for m in range(5))
                   for k in range(3))
        assert weno5(q) == pytest.approx(want, rel=1e-13, abs=1e-13 * np.abs(q).max())


def test_linear_weights_reduce_to_poly():
    rs = np.random.default_rng(2)
    for _ in range(50):
        q = rs.normal(size=5)
        w = weno5_weights(q, eps=1e30)
        np.testing.assert_allclose(w, [0.1, 0.6, 0.3], rtol=1e-14)
        assert weno5(q, eps=1e30) == pytest.approx(weno5_poly(q), rel=1e-13, abs=1e-14)


def jiang_shu_beta(q, k):
    """beta_k = sum_{l=1,2} h^(2l-1) int_cell (d^l p_k/dx^l)^2 dx (Jiang & Shu 1996), where
    p_k is the quadratic with the cell averages of stencil k and the integral runs over the
    cell left of the face (cell i-1); h = 1, cell i-1 = [-1, 0]."""
    cells = {0: (0, 1, 2), 1: (1, 2, 3), 2: (2, 3, 4)}[k]
    A = np.zeros((3, 3))
    for r, c in enumerate(cells):
        lo, hi = c - 3.0, c - 2.0
        for n in range(3):
            A[r, n] = (hi ** (n + 1) - lo ** (n + 1)) / (n + 1)
    coef = np.linalg.solve(A, q[list(cells)])
    P = np.polynomial.polynomial.Polynomial(coef)
    xs, ws = np.polynomial.legendre.leggauss(8)
    x = -0.5 + 0.5 * xs
    total = 0.0
    for l in (1, 2):
        d = P.deriv(l)
        total += np.sum(0.5 * ws * d(x) ** 2)
    return total


def test_weights_match_jiang_shu_integral_definition():
    rs = np.random.default_rng(3)
    d = np.array([0.1, 0.6, 0.3])
    for _ in range(300):
        scale = 10.0 ** rs.uniform(-4, 3)
        q = rs.normal(size=5) * scale
        eps = 10.0 ** rs.uniform(-8, -2)
        b = np.array([jiang_shu_beta(q, k) for k in range(3)])
        a = d / (eps + b) ** 2
        np.testing.assert_allclose(weno5_weights(q, eps), a / a.sum(), rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_exact_for_quadratics_any_weights(deg):
    rs = np.random.default_rng(10 + deg)
    for _ in range(100):
        coef = rs.normal(size=deg + 1) * 10.0 ** rs.uniform(-2, 2, size=deg + 1)
        x0, h = rs.uniform(-2, 2), 10.0 ** rs.uniform(-2, 0)
        q = stencil_avgs(lambda a, b: cell_avg_poly(coef, a, b), x0, h)
        exact = np.polynomial.polynomial.polyval(x0, coef)
        for eps in (1e-12, 1e-6, 1.0, 1e6):
            got = weno5(q, eps)
            assert got == pytest.approx(exact, rel=1e-11, abs=1e-11 * np.abs(q).max())


@pytest.mark.parametrize("deg", [3, 4])
def test_poly_exact_for_quartics(deg):
    rs = np.random.default_rng(20 + deg)
    for _ in range(100):
        coef = rs.normal(size=deg + 1)
        x0, h = rs.uniform(-1, 1), 10.0 ** rs.uniform(-2, -0.5)
        q = stencil_avgs(lambda a, b: cell_avg_poly(coef, a, b), x0, h)
        exact = np.polynomial.polynomial.polyval(x0, coef)
        assert weno5_poly(q) == pytest.approx(exact, rel=1e-10, abs=1e-10 * np.abs(q).max())
        assert weno5(q, 1e30) == pytest.approx(exact, rel=1e-10, abs=1e-10 * np.abs(q).max())


def test_fifth_order_on_smooth_monotone_data():
    """Face value of A exp(sin x) at x = 0.3 (f' != 0) from exact cell averages; A large so
    the nonlinear weights are active (beta >> eps)."""
    A = 1000.0
    xs, ws = np.polynomial.legendre.leggauss(12)

    def f_avg(a, b):
        x = 0.5 * (a + b) + 0.5 * (b - a) * xs
        return np.sum(0.5 * ws * A * np.exp(np.sin(x)))

    x0 = 0.3
    # asymptotic range: the weights approach the linear ones as O(h^2), so coarser grids
    # show a pre-asymptotic mix; finer ones reach rounding (~1e-13 A)
    hs = [0.2 / 2 ** n for n in range(4, 7)]
    err = [abs(weno5(stencil_avgs(f_avg, x0, h)) - A * np.exp(np.sin(x0))) for h in hs]
    order = [np.log2(err[n] / err[n + 1]) for n in range(len(err) - 1)]
    assert min(order) >= 4.75, (err, order)


def test_eno_property_at_a_jump():
    # jump between Q_{i-1} and Q_i: the left state uses the smooth stencil 0 and keeps the
    # left value
    assert abs(weno5([0.0, 0.0, 0.0, 1.0, 1.0])) < 1e-9
    assert abs(weno5([1.0, 1.0, 1.0, 0.0, 0.0]) - 1.0) < 1e-9
    # jump between Q_{i-3} and Q_{i-2}: stencils 1 and 2 are smooth, value is the right one
    assert abs(weno5([0.0, 1.0, 1.0, 1.0, 1.0]) - 1.0) < 1e-9
    # the linear interpolant overshoots at the same jump, WENO does not
    assert weno5_poly([0.0, 0.0, 0.0, 1.0, 1.0]) == pytest.approx(0.4)
