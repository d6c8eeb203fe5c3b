"""Pins of the equivalent potential temperature (App. A, Eq. theta_e) and of the moist-adiabat
initialisation (Eq. mgrad integrated in the workload generator): theta_e reduces to the dry
potential temperature without water, and the reversible saturated moist adiabat, built from
Li (2018)'s gradient, keeps Emanuel's theta_e constant (two independent published formulas
that must agree along the same process)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def test_dry_limit_is_the_potential_temperature():
    w = W.moist_bubble(n=8)
    Y = w.Y.copy()
    Y[0] += Y[1]
    Y[1:4] = 0.0  # all water removed, the same density and energy
    o = Oracle(w)
    te = o.theta_e(Y)
    X, T, _ = o.cons_to_prim(Y.reshape(w.nv, -1)[:, 0])
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    for c in range(5):
        y = Y.reshape(w.nv, -1)[:, c]
        Xc, Tc, _ = o.cons_to_prim(y)
        assert te.reshape(-1)[c] == pytest.approx(Tc * (1e5 / Xc[-1]) ** kappa, rel=1e-13)


@pytest.mark.parametrize("r_t", [0.012, 0.020])
def test_moist_adiabat_background_has_uniform_theta_e(r_t):
    w = W.bryan_moist_bubble(nx=8, nz=100, Lx=800.0, A=0.0, r_t=r_t)
    te = Oracle(w).theta_e(w.Y)
    assert w.Y[2].min() > 0.0  # saturated with cloud at every level
    assert np.ptp(te) <= 1e-9 * te.mean()


def test_bubble_raises_theta_e_where_it_is_warmer():
    w = W.bryan_moist_bubble(nx=40, nz=20, Lx=4000.0, Lz=2000.0, R=800.0, xc=2000.0, zc=800.0)
    te = Oracle(w).theta_e(w.Y)
    anomaly = te - te[:, :, :1]
    assert anomaly.max() > 1.0 and anomaly.min() >= -1e-9
