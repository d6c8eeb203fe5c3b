"""Hand-built workloads for the scheme pins (inputs only)."""
import dataclasses

import numpy as np

import workloads as W


def uniform_column(nx, L, rho_fn, u_fn, w_fn, p0=1e5, nz=3, gamma=1.4, R=287.0, nu=0.0,
                   periodic_x=True):
    """x-z strip without gravity, uniform in z: density rho_fn(x), velocities u_fn(x),
    w_fn(x), uniform pressure p0 (dry ideal gas)."""
    dx = L / nx
    x = (np.arange(nx) + 0.5) * dx
    rho = rho_fn(x) * np.ones((nz, 1, nx))
    u = u_fn(x) * np.ones((nz, 1, nx))
    w = w_fn(x) * np.ones((nz, 1, nx))
    Y = np.zeros((4, nz, 1, nx))
    Y[0] = rho
    Y[1] = rho * u
    Y[2] = rho * w
    Y[3] = p0 / (gamma - 1.0) + 0.5 * rho * (u * u + w * w)
    bc = (W.PERIODIC if periodic_x else W.REFLECT,) * 2 + (W.REFLECT,) * 4
    return W.Workload(name=f"strip_{nx}", nx=nx, ny=1, nz=nz, dx=dx, dy=dx, dz=dx, bc=bc,
                      grav=0.0, gamma_d=gamma, R_d=R, vapors=[], ncond=0,
                      rho_bar=np.ones(nz), p_bar_face=np.full(nz + 1, p0), Y=Y, nu=nu)


def no_gravity(w):
    """Same state and parameters with g = 0 and a flat reference pressure (the mean of the
    workload's reference, so pressure perturbations stay small)."""
    pm = float(np.mean(w.p_bar_face))
    return dataclasses.replace(w, grav=0.0, p_bar_face=np.full(w.nz + 1, pm),
                               rho_bar=np.full(w.nz, float(np.mean(w.rho_bar))))
