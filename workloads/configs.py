"""Seeded synthetic initial states shaped like the paper's test problems.

This module builds INPUTS only: the conserved state Y, the fixed hydrostatic
reference profile and the physical parameters of each workload. It contains
none of the scheme (no reconstruction, Riemann flux, update or saturation
adjustment). Both the oracle and the CUDA library receive exactly what is
built here.

Physical set-up used to make the inputs (each stated where it is applied):
  * equation of state p = (rho_d R_d + sum_i rho_i R_i) T            (Sec. 2, Eq. eos)
  * total energy rho e = (rho_d c_vd + sum rho_i c_vi + ...) T + K + A (Sec. 2, Eq. energy)
  * potential temperature T = theta (p / p0)^(R_d / c_pd)             (App. C, Eq. theta, dry)
  * saturation vapour pressure from the integrated Clausius-Clapeyron
    relation, used only to cap initial vapour at saturation          (App. D)
  * a discretely hydrostatic background: p_{k+1/2} = p_{k-1/2} - g rho_k dz
    with the cell pressure p_k the mean of its two face pressures; the
    initial pressure of every cell equals the reference p_k, so a state
    without perturbation is at rest to rounding in the scheme.

Field order of Y follows the paper's conserved vector (App. B):
  (rho_d, rho_i [n_vapor], rho_ij [n_vapor x n_cond, grouped by vapour],
   rho u, [rho v if ny > 1], rho w, rho e),
stored as Y[field, k, j, i] with i (x) fastest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

from . import rng

RHAT = 8.3144598  # universal gas constant, J/(mol K) (App. A, symbol table)

REFLECT = 0   # free-slip wall
PERIODIC = 1
NOSLIP = 2    # wall whose ghost cells reverse every velocity component

BASE_SEED = 190102955


@dataclasses.dataclass
class Condensate:
    sigma_v: float  # c_ij / c_vd
    L_ref: float  # latent heat of forming this condensate at the vapour's T_ref, J/kg


@dataclasses.dataclass
class Vapor:
    name: str
    eps: float  # m_i / m_d
    sigma_v: float  # c_v,i / c_vd
    T_ref: float  # reference temperature (triple point), K
    p_ref: float  # saturation vapour pressure over condensate (i,1) at T_ref, Pa
    cond: List[Condensate]  # j = 1 cloud, j = 2 precipitation


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    bc: tuple  # (x-, x+, y-, y+, z-, z+), REFLECT, PERIODIC or NOSLIP
    grav: float
    gamma_d: float
    R_d: float
    vapors: List[Vapor]
    ncond: int
    rho_bar: np.ndarray  # (nz,) reference density of each level
    p_bar_face: np.ndarray  # (nz+1,) reference pressure at each level face
    Y: np.ndarray  # (nv, nz, ny, nx) float64
    cfl: float = 0.8
    nu: float = 0.0
    nsteps: int = 1
    satadj_max_iter: int = 20
    satadj_tol: float = 1e-12
    weno_eps: float = 1e-6
    dtype: str = "f64"
    seed: int = BASE_SEED
    # terminal velocity of condensate phase j of every vapour (m/s, negative falls); the
    # Kessler rates (k1 condensation, k2 autoconversion, k3 accretion, k4 evaporation, 1/s);
    # an empty kessler_k switches the microphysics off
    w_term: tuple = ()
    kessler_k: tuple = ()
    kessler_max_iter: int = 30
    kessler_tol: float = 1e-12
    # forcing of the Jovian simulation: body cooling (rate K/s, p_lo, p_hi) and sponge
    # (tau0 s, p0 Pa) by the reference pressure of each level; empty: off
    cooling: tuple = ()
    sponge: tuple = ()
    # lower boundary of the Jovian simulation: temperature held by the ghost cells below the
    # bottom wall, K (0: off)
    T_bottom: float = 0.0

    @property
    def nvapor(self) -> int:
        return len(self.vapors)

    @property
    def nmom(self) -> int:
        return 3 if self.ny > 1 else 2

    @property
    def nv(self) -> int:
        return 1 + self.nvapor + self.nvapor * self.ncond + self.nmom + 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def field_names(self) -> List[str]:
        names = ["rho_d"] + [f"rho_{v.name}" for v in self.vapors]
        for v in self.vapors:
            names += [f"rho_{v.name}_c{j + 1}" for j in range(self.ncond)]
        names += ["rho_u"] + (["rho_v"] if self.ny > 1 else []) + ["rho_w", "rho_e"]
        return names

    def with_state(self, Y: np.ndarray) -> "Workload":
        return dataclasses.replace(self, Y=np.ascontiguousarray(Y, dtype=np.float64))


# --------------------------------------------------------------------------
# species tables used by the workloads (inputs, not method arithmetic)
# --------------------------------------------------------------------------
M_H2O = 18.01528e-3  # kg/mol
M_NH3 = 17.03052e-3


def _vapor(name, m_vapor, m_dry, c_vd, c_cond, L_ref, T_ref, p_ref, ncond=2):
    """Vapour whose gas has c_v = 3 R (non-linear polyatomic molecule)."""
    R_i = RHAT / m_vapor
    c_vi = 3.0 * R_i
    return Vapor(name=name, eps=m_vapor / m_dry, sigma_v=c_vi / c_vd, T_ref=T_ref, p_ref=p_ref,
                 cond=[Condensate(sigma_v=c_cond / c_vd, L_ref=L_ref) for _ in range(ncond)])


def earth_water(R_d=287.0, gamma_d=1.4) -> Vapor:
    """Water over liquid: triple point 273.16 K / 611.657 Pa, L = 2.5008e6 J/kg, c_liq = 4218 J/(kg K)."""
    m_d = RHAT / R_d
    c_vd = R_d / (gamma_d - 1.0)
    return _vapor("H2O", M_H2O, m_d, c_vd, 4218.0, 2.5008e6, 273.16, 611.657)


def jovian_species(R_d, gamma_d) -> List[Vapor]:
    """H2O over liquid and NH3 over ice (triple point 195.4 K / 6060 Pa, L = 1.8e6 J/kg,
    c_ice = 2300 J/(kg K)); approximate handbook-style constants chosen for the workload."""
    m_d = RHAT / R_d
    c_vd = R_d / (gamma_d - 1.0)
    return [_vapor("H2O", M_H2O, m_d, c_vd, 4218.0, 2.5008e6, 273.16, 611.657),
            _vapor("NH3", M_NH3, m_d, c_vd, 2300.0, 1.8e6, 195.4, 6060.0)]


# --------------------------------------------------------------------------
# set-up physics (initial-state construction only)
# --------------------------------------------------------------------------
def _sat_pressure(v: Vapor, R_d: float, gamma_d: float, T):
    """Integrated Clausius-Clapeyron saturation pressure over condensate (v,1) (App. D)."""
    c_vd = R_d / (gamma_d - 1.0)
    R_i = R_d / v.eps
    c_pi = v.sigma_v * c_vd + R_i
    dc = v.cond[0].sigma_v * c_vd - c_pi
    beta = (v.cond[0].L_ref + dc * v.T_ref) / (R_i * v.T_ref)
    delta = dc / R_i
    t = np.asarray(T, dtype=np.float64) / v.T_ref
    return v.p_ref * np.exp(beta * (1.0 - 1.0 / t) - delta * np.log(t))


def _gas_densities(p, T, R_d, gamma_d, vapors, x_vap, cap_T=None):
    """Dry and vapour densities of a cloud-free gas at (p, T).

    x_vap[i]: target molar fraction of vapour i (or None: use a partial pressure given by
    cap_T, see callers). Each vapour partial pressure is capped at saturation at T."""
    p = np.asarray(p, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    pv = []
    for i, v in enumerate(vapors):
        target = x_vap[i](p, T)
        pv.append(np.minimum(target, _sat_pressure(v, R_d, gamma_d, T)))
    pd = p - sum(pv) if pv else p
    rho_d = pd / (R_d * T)
    rho_v = [pv[i] / ((R_d / v.eps) * T) for i, v in enumerate(vapors)]
    return rho_d, rho_v


def _hydrostatic_column(nz, dz, g, p_anchor, anchor_top, rho_of):
    """Discretely hydrostatic reference: p_{k+1/2} = p_{k-1/2} - g rho_k dz and
    rho_k = rho_of(k, p_k) with p_k the mean of the two face pressures."""
    pf = np.zeros(nz + 1)
    rho = np.zeros(nz)
    order = range(nz - 1, -1, -1) if anchor_top else range(nz)
    if anchor_top:
        pf[nz] = p_anchor
    else:
        pf[0] = p_anchor
    for k in order:
        pface = pf[k + 1] if anchor_top else pf[k]
        sgn = 1.0 if anchor_top else -1.0
        r = rho_of(k, pface)
        for _ in range(200):
            r_new = rho_of(k, pface + sgn * 0.5 * g * r * dz)
            if abs(r_new - r) <= 1e-16 * abs(r_new):
                r = r_new
                break
            r = r_new
        rho[k] = r
        if anchor_top:
            pf[k] = pf[k + 1] + g * r * dz
        else:
            pf[k + 1] = pf[k] - g * r * dz
    return rho, pf


def _assemble(nx, ny, nz, rho_d, rho_v, T, R_d, gamma_d, vapors, ncond):
    """Conserved state of a motionless, cloud-free gas (Eq. energy with K = A = 0)."""
    c_vd = R_d / (gamma_d - 1.0)
    nmom = 3 if ny > 1 else 2
    nv = 1 + len(vapors) * (1 + ncond) + nmom + 1
    Y = np.zeros((nv, nz, ny, nx))
    Y[0] = rho_d
    cv = c_vd * rho_d
    for i, v in enumerate(vapors):
        Y[1 + i] = rho_v[i]
        cv = cv + v.sigma_v * c_vd * rho_v[i]
    Y[nv - 1] = cv * T
    return Y


def _cell_centres(n, d):
    return (np.arange(n) + 0.5) * d


def _dry_theta_state(name, nx, nz, Lx, Lz, theta0, p0, perturb, R_d=287.0, gamma_d=1.4,
                     g=9.81, bc=(REFLECT,) * 6, **kw):
    """x-z plane: isentropic background theta0 at surface pressure p0 plus a
    theta perturbation applied at fixed pressure (density changes only)."""
    dx, dz = Lx / nx, Lz / nz
    kappa = (gamma_d - 1.0) / gamma_d  # R_d / c_pd

    def rho_of(k, p):
        return p / (R_d * theta0 * (p / p0) ** kappa)

    rho_bar, pf = _hydrostatic_column(nz, dz, g, p0, False, rho_of)
    pk = 0.5 * (pf[:-1] + pf[1:])
    x = _cell_centres(nx, dx)[None, :]
    z = _cell_centres(nz, dz)[:, None]
    theta = theta0 + perturb(x, z)
    T = theta * (pk[:, None] / p0) ** kappa
    rho = pk[:, None] / (R_d * T)
    Y = _assemble(nx, 1, nz, rho[:, None, :], [], T[:, None, :], R_d, gamma_d, [], 0)
    return Workload(name=name, nx=nx, ny=1, nz=nz, dx=dx, dy=dx, dz=dz, bc=tuple(bc), grav=g,
                    gamma_d=gamma_d, R_d=R_d, vapors=[], ncond=0, rho_bar=rho_bar, p_bar_face=pf,
                    Y=Y, **kw)


def cosine_bubble(A, xc, zc, rx, rz=None):
    """theta' = A cos^2(pi L / 2) for L <= 1, L the scaled distance to the centre."""
    rz = rx if rz is None else rz

    def f(x, z):
        L = np.sqrt(((x - xc) / rx) ** 2 + ((z - zc) / rz) ** 2)
        return np.where(L <= 1.0, A * np.cos(0.5 * np.pi * np.minimum(L, 1.0)) ** 2, 0.0)

    return f


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def warm_bubble(n=128, L=1000.0, nsteps=100, dtype="f64", A=0.5, R=250.0, xc=500.0, zc=260.0):
    """2-D dry warm bubble: 1 km box, theta = 300 K, p_s = 1e5 Pa, +0.5 K cosine bubble
    of radius 250 m at (500 m, 260 m), reflecting walls (shaped like the Robert bubble, Sec. 5.2)."""
    return _dry_theta_state(f"warm_bubble_{n}x{n}", n, n, L, L, 300.0, 1e5,
                            cosine_bubble(A, xc, zc, R), nsteps=nsteps, dtype=dtype)


def density_current(nx=1024, nz=256, nsteps=None, dtype="f32", nu=75.0):
    """2-D dry density current (Straka, Sec. 5.1): 25.6 km x 6.4 km half domain with a
    mirror wall at x = 0, theta = 300 K, -15 K cosine bubble of radii 4 km x 2 km centred
    at (0, 3 km), viscosity 75 m^2/s."""
    w = _dry_theta_state(f"density_current_{nx}x{nz}", nx, nz, 25600.0, 6400.0, 300.0, 1e5,
                         cosine_bubble(-15.0, 0.0, 3000.0, 4000.0, 2000.0), dtype=dtype, nu=nu)
    if nsteps is not None:
        w.nsteps = nsteps
    return w


def rest_state(nx=32, nz=32, L=1000.0, nsteps=100, dtype="f64"):
    """Isentropic atmosphere at rest (no perturbation)."""
    return _dry_theta_state(f"rest_{nx}x{nz}", nx, nz, L, L * nz / nx, 300.0, 1e5,
                            lambda x, z: 0.0 * x * z, nsteps=nsteps, dtype=dtype)


def isothermal_rest(nx=16, nz=32, T0=250.0, L=1000.0, p0=1e5, R_d=287.0, gamma_d=1.4,
                    g=9.81, nsteps=100, dtype="f64"):
    """Isothermal dry atmosphere at rest on a discretely hydrostatic profile."""
    dx = L / nx
    dz = dx
    rho_bar, pf = _hydrostatic_column(nz, dz, g, p0, False, lambda k, p: p / (R_d * T0))
    pk = 0.5 * (pf[:-1] + pf[1:])
    T = np.full((nz, 1, nx), T0)
    rho = pk[:, None, None] / (R_d * T)
    Y = _assemble(nx, 1, nz, rho, [], T, R_d, gamma_d, [], 0)
    return Workload(name=f"isothermal_{nx}x{nz}", nx=nx, ny=1, nz=nz, dx=dx, dy=dx, dz=dz,
                    bc=(REFLECT,) * 6, grav=g, gamma_d=gamma_d, R_d=R_d, vapors=[], ncond=0,
                    rho_bar=rho_bar, p_bar_face=pf, Y=Y, nsteps=nsteps, dtype=dtype)


def dry_bubble_3d(nx=32, ny=24, nz=20, L=1000.0, A=0.5, R=250.0, nsteps=10, dtype="f64",
                  theta0=300.0, p0=1e5, R_d=287.0, gamma_d=1.4, g=9.81):
    """3-D dry warm bubble: isentropic theta0 background, spherical cosine bubble at the
    centre of the lower half, periodic x and y, walls in z."""
    dx = dy = dz = L / nx
    kappa = (gamma_d - 1.0) / gamma_d

    def rho_of(k, p):
        return p / (R_d * theta0 * (p / p0) ** kappa)

    rho_bar, pf = _hydrostatic_column(nz, dz, g, p0, False, rho_of)
    pk = 0.5 * (pf[:-1] + pf[1:])
    x = _cell_centres(nx, dx)[None, None, :]
    y = _cell_centres(ny, dy)[None, :, None]
    z = _cell_centres(nz, dz)[:, None, None]
    r = np.sqrt((x - nx * dx / 2) ** 2 + (y - ny * dy / 2) ** 2 + (z - nz * dz / 3) ** 2) / R
    theta = theta0 + np.where(r <= 1.0, A * np.cos(0.5 * np.pi * np.minimum(r, 1.0)) ** 2, 0.0)
    T = theta * (pk[:, None, None] / p0) ** kappa
    rho = pk[:, None, None] / (R_d * T)
    Y = _assemble(nx, ny, nz, rho, [], T, R_d, gamma_d, [], 0)
    return Workload(name=f"dry_bubble_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                    bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC, REFLECT, REFLECT), grav=g,
                    gamma_d=gamma_d, R_d=R_d, vapors=[], ncond=0, rho_bar=rho_bar, p_bar_face=pf,
                    Y=Y, nsteps=nsteps, dtype=dtype)


def jovian(nx=256, ny=256, nz=128, Lx=100e3, Ly=100e3, Lz=150e3, nsteps=500, dtype="f32",
           seed=BASE_SEED + 3, noise_K=0.1, q_deep=(0.040, 0.0027), p_top=1e5):
    """3-D moist Jovian-like column (Sec. 6): H2/He gas with mu = 2.3 g/mol, c_p = 3.5 R;
    dry adiabat theta = 166 K referenced at 1 bar, the top face at p_top (1 bar by default);
    H2O and NH3 vapour with deep mass mixing ratios 40 and 2.7 g/kg capped at saturation; no
    condensate initially; seeded white-noise temperature perturbation (sigma 0.1 K);
    periodic x/y, walls in z. The grid spacing is Lx/nx etc., so a crop (smaller nx, ny at
    the same spacing) is made by scaling Lx, Ly with nx, ny."""
    R_d = RHAT / 2.3e-3
    gamma_d = 1.4
    g = 24.79
    p0, theta0 = 1e5, 166.0
    kappa = (gamma_d - 1.0) / gamma_d
    vapors = jovian_species(R_d, gamma_d)
    dx, dy, dz = Lx / nx, Ly / ny, Lz / nz
    qd = 1.0 - sum(q_deep)
    denom = qd + sum(q / v.eps for q, v in zip(q_deep, vapors))
    x_deep = [(q / v.eps) / denom for q, v in zip(q_deep, vapors)]
    x_fn = [(lambda xv: (lambda p, T: xv * p))(xv) for xv in x_deep]

    def T_of(p):
        return theta0 * (p / p0) ** kappa

    def rho_of(k, p):
        T = T_of(p)
        rd, rv = _gas_densities(p, T, R_d, gamma_d, vapors, x_fn)
        return float(rd + sum(rv))

    rho_bar, pf = _hydrostatic_column(nz, dz, g, p_top, True, rho_of)
    pk = 0.5 * (pf[:-1] + pf[1:])
    Tbar = T_of(pk)
    dT = noise_K * rng.normal(seed, nx * ny * nz).reshape(nz, ny, nx)
    T = Tbar[:, None, None] + dT
    P = np.broadcast_to(pk[:, None, None], T.shape)
    rd, rv = _gas_densities(P, T, R_d, gamma_d, vapors, x_fn)
    Y = _assemble(nx, ny, nz, rd, rv, T, R_d, gamma_d, vapors, 2)
    return Workload(name=f"jovian_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                    bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC, REFLECT, REFLECT), grav=g,
                    gamma_d=gamma_d, R_d=R_d, vapors=vapors, ncond=2, rho_bar=rho_bar,
                    p_bar_face=pf, Y=Y, nsteps=nsteps, dtype=dtype, seed=seed)


def jovian_rce(nx=256, ny=256, nz=128, Lx=100e3, Ly=100e3, Lz=332e3, p_top=1e4, nsteps=500,
               dtype="f32", seed=BASE_SEED + 6, noise_K=0.1, cool_K_per_day=1.0):
    """The Jovian radiative-convective setup of Sec. 6 on the column above: the top face at
    0.1 bar and 332 km of depth put the bottom near 200 bar and 750 K on the dry adiabat
    (the paper holds 800 K at 200 bar). Kessler microphysics with the paper's constants and
    precipitation falling at 20 m/s; a body cooling of cool_K_per_day between 2 and 0.2 bar;
    a sponge above 0.2 bar relaxing the horizontal winds on 1e4 s (p/p0)^2; a no-slip bottom
    wall whose ghost cells hold the bottom level's initial horizontal-mean temperature (the
    fixed-temperature lower boundary). Periodic x and y, a free-slip top."""
    w = jovian(nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz, nsteps=nsteps, dtype=dtype,
               seed=seed, noise_K=noise_K, p_top=p_top)
    pk0 = 0.5 * (w.p_bar_face[0] + w.p_bar_face[1])
    T_bot = 166.0 * (pk0 / 1e5) ** ((w.gamma_d - 1.0) / w.gamma_d)
    return dataclasses.replace(
        w, name=f"jovian_rce_{nx}x{ny}x{nz}",
        bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC, NOSLIP, REFLECT),
        kessler_k=(1e9, 1e-4, 0.0, 1e-2), w_term=(0.0, -20.0),
        cooling=(cool_K_per_day / 86400.0, 2e4, 2e5), sponge=(1e4, 2e4), T_bottom=float(T_bot))


def moist_bubble(n=64, L=1000.0, A=0.5, R=250.0, xc=500.0, zc=450.0, rh=0.9, nsteps=200,
                 dtype="f32", seed=BASE_SEED + 4, theta0=300.0, p0=1e5, nx=None, nz=None):
    """2-D moist warm bubble: Earth air (R_d = 287, gamma 1.4), theta = 300 K background with
    water vapour at relative humidity `rh` of the background temperature, capped at
    saturation of the perturbed temperature; cloud and rain start at 0; walls."""
    nx = n if nx is None else nx
    nz = n if nz is None else nz
    R_d, gamma_d, g = 287.0, 1.4, 9.81
    kappa = (gamma_d - 1.0) / gamma_d
    vap = earth_water(R_d, gamma_d)
    dx, dz = L / nx, L / nz

    def rh_fn(p, T):
        return rh * _sat_pressure(vap, R_d, gamma_d, T)

    def rho_of(k, p):
        T = theta0 * (p / p0) ** kappa
        rd, rv = _gas_densities(p, T, R_d, gamma_d, [vap], [rh_fn])
        return float(rd + rv[0])

    rho_bar, pf = _hydrostatic_column(nz, dz, g, p0, False, rho_of)
    pk = 0.5 * (pf[:-1] + pf[1:])
    Tbar = theta0 * (pk / p0) ** kappa
    x = _cell_centres(nx, dx)[None, :]
    z = _cell_centres(nz, dz)[:, None]
    theta = theta0 + cosine_bubble(A, xc, zc, R)(x, z)
    T = theta * (pk[:, None] / p0) ** kappa
    pv_bg = rh * _sat_pressure(vap, R_d, gamma_d, Tbar)[:, None] * np.ones_like(T)
    fixed = [(lambda arr: (lambda p, TT: arr))(pv_bg)]
    P = pk[:, None] * np.ones_like(T)
    rd, rv = _gas_densities(P, T, R_d, gamma_d, [vap], fixed)
    Y = _assemble(nx, 1, nz, rd[:, None, :], [rv[0][:, None, :]], T[:, None, :], R_d, gamma_d,
                  [vap], 2)
    return Workload(name=f"moist_bubble_{nx}x{nz}", nx=nx, ny=1, nz=nz, dx=dx, dy=dx, dz=dz,
                    bc=(REFLECT,) * 6, grav=g, gamma_d=gamma_d, R_d=R_d, vapors=[vap], ncond=2,
                    rho_bar=rho_bar, p_bar_face=pf, Y=Y, nsteps=nsteps, dtype=dtype, seed=seed)


def moist_adjoint_bubble(n=256, rh=0.95, rh_core=1.05, A=0.5, R=250.0, xc=500.0, zc=260.0,
                         dtype="f64", nsteps=400):
    """Moist variant of the adjoint bubble: the warm bubble of the first workload (+A K,
    radius R at (xc, zc) on an n x n grid over 1 km) in Earth air with water vapour at
    relative humidity rh of the background, and at rh_core of saturation at the perturbed
    temperature inside the bubble (pressure unchanged), so that the first saturation
    adjustment forms cloud there; cloud and rain start at 0; walls."""
    w = moist_bubble(n=n, A=A, R=R, xc=xc, zc=zc, rh=rh, nsteps=nsteps, dtype=dtype)
    vap = w.vapors[0]
    kappa = (w.gamma_d - 1.0) / w.gamma_d
    pk = 0.5 * (w.p_bar_face[:-1] + w.p_bar_face[1:])
    x = _cell_centres(w.nx, w.dx)[None, :]
    z = _cell_centres(w.nz, w.dz)[:, None]
    shape = cosine_bubble(A, xc, zc, R)(x, z)
    T = (300.0 + shape) * (pk[:, None] / 1e5) ** kappa
    core = shape > 0.0
    pv = rh_core * _sat_pressure(vap, w.R_d, w.gamma_d, T)
    P = pk[:, None] * np.ones_like(T)
    rho_d = (P - pv) / (w.R_d * T)
    rho_v = pv / ((w.R_d / vap.eps) * T)
    Y = w.Y.copy()
    Yc = _assemble(w.nx, 1, w.nz, rho_d[:, None, :], [rho_v[:, None, :]], T[:, None, :],
                   w.R_d, w.gamma_d, [vap], w.ncond)
    Y[:, core[:, None, :]] = Yc[:, core[:, None, :]]
    w = w.with_state(Y)
    w.name = f"moist_adjoint_bubble_{n}x{n}"
    return w


def _moist_adiabat(T0, p0, r_t, R_d, gamma_d, vap, p_top, n=40000):
    """Reversible saturated moist adiabat of Appendix A (Eq. mgrad): ln T against ln p for air
    carrying one condensing species with total water r_t per unit mass of dry air, integrated
    by classical RK4 in ln p from (T0, p0) up to p_top. Vapour is at saturation over the
    condensate (the App. D Clausius-Clapeyron integral), cloud the rest of r_t; where r_t is
    below saturation the latent terms vanish (the dry gradient of Eq. dgrad). Returns
    (ln p ascending, T) for interpolation."""
    c_vd = R_d / (gamma_d - 1.0)
    c_pd = gamma_d * c_vd
    R_v = R_d / vap.eps
    c_pv = vap.sigma_v * c_vd + R_v
    c_l = vap.cond[0].sigma_v * c_vd
    dc = c_l - c_pv  # Eq. latent
    beta = (vap.cond[0].L_ref + dc * vap.T_ref) / (R_v * vap.T_ref)
    delta = dc / R_v

    def slope(lnp, T):
        p = np.exp(lnp)
        t = T / vap.T_ref
        es = vap.p_ref * np.exp(beta * (1.0 - 1.0 / t) - delta * np.log(t))
        r_s = vap.eps * es / (p - es)
        r_v = min(r_s, r_t)
        r_c = r_t - r_v
        a = r_v / vap.eps
        lam = (vap.cond[0].L_ref - dc * (T - vap.T_ref)) / (R_v * T) if r_s < r_t else 0.0
        num = (1.0 + a) * (1.0 + a * lam)
        den = c_pd / R_d * (1.0 + r_v * c_pv / c_pd + r_c * c_l / c_pd) + a * lam * lam + (a * lam) ** 2
        return T * num / den  # dT / d ln p

    lnp = np.linspace(np.log(p0), np.log(p_top), n)
    h = lnp[1] - lnp[0]
    T = np.empty(n)
    T[0] = T0
    for m in range(n - 1):
        x, y = lnp[m], T[m]
        k1 = slope(x, y)
        k2 = slope(x + h / 2, y + h / 2 * k1)
        k3 = slope(x + h / 2, y + h / 2 * k2)
        k4 = slope(x + h, y + h * k3)
        T[m + 1] = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return lnp[::-1].copy(), T[::-1].copy()


def _saturated_parcel(T, p, r_t, R_d, gamma_d, vap):
    """Densities (rho_d, rho_v, rho_c) of air at (T, p) with total water r_t per unit dry
    air, the vapour at saturation over the condensate or all of r_t if that is less."""
    c_vd = R_d / (gamma_d - 1.0)
    R_v = R_d / vap.eps
    es = _sat_pressure(vap, R_d, gamma_d, T)
    r_s = vap.eps * es / (p - es)
    e = np.where(r_s < r_t, es, p * r_t / (vap.eps + r_t))
    rho_d = (p - e) / (R_d * T)
    rho_v = e / (R_v * T)
    rho_c = np.maximum(r_t * rho_d - rho_v, 0.0)
    del c_vd
    return rho_d, rho_v, rho_c


def bryan_moist_bubble(nx=200, nz=100, Lx=20e3, Lz=10e3, T_s=289.85, p_s=1e5, r_t=0.020,
                       A=2.0, R=2000.0, xc=10e3, zc=2000.0, dtype="f64", nsteps=5000):
    """Bryan moist bubble (Sec. 5, after Bryan & Fritsch 2002): a saturated environment on
    the reversible moist adiabat from 289.85 K and 1 bar, total water fixed at all levels,
    20 km x 10 km at 100 m; a bubble warmer by A cos^2(pi L/2) (L the distance from its
    centre over R) at fixed pressure, saturated at its own temperature (more vapour, less
    cloud); Earth air and water (cloud and rain slots, rain 0); walls. The background is
    discretely hydrostatic and neutral to moist convection."""
    R_d, gamma_d, g = 287.0, 1.4, 9.81
    vap = earth_water(R_d, gamma_d)
    dx, dz = Lx / nx, Lz / nz
    lnp, Tad = _moist_adiabat(T_s, p_s, r_t, R_d, gamma_d, vap, p_top=0.2 * p_s)

    def T_of(p):
        return np.interp(np.log(p), lnp, Tad)

    def rho_of(k, p):
        rd, rv, rc = _saturated_parcel(T_of(p), p, r_t, R_d, gamma_d, vap)
        return float(rd + rv + rc)

    rho_bar, pf = _hydrostatic_column(nz, dz, g, p_s, False, rho_of)
    pk = 0.5 * (pf[:-1] + pf[1:])
    x = _cell_centres(nx, dx)[None, :]
    z = _cell_centres(nz, dz)[:, None]
    T = T_of(pk)[:, None] + cosine_bubble(A, xc, zc, R)(x, z)
    P = pk[:, None] * np.ones_like(T)
    rd, rv, rc = _saturated_parcel(T, P, r_t, R_d, gamma_d, vap)
    Y = _assemble_condensed(nx, 1, nz, rd[:, None, :], rv[:, None, :], rc[:, None, :],
                            T[:, None, :], R_d, gamma_d, vap)
    return Workload(name=f"bryan_moist_bubble_{nx}x{nz}", nx=nx, ny=1, nz=nz, dx=dx, dy=dx,
                    dz=dz, bc=(REFLECT,) * 6, grav=g, gamma_d=gamma_d, R_d=R_d, vapors=[vap],
                    ncond=2, rho_bar=rho_bar, p_bar_face=pf, Y=Y, nsteps=nsteps, dtype=dtype)


def _assemble_condensed(nx, ny, nz, rho_d, rho_v, rho_c, T, R_d, gamma_d, vap):
    """Conserved state at rest of dry air, one vapour and its cloud (rain 0): rho e =
    (c_vd rho_d + c_v rho_v + c_l rho_c) T + mu_c rho_c, mu_c = -(L^r + (c_l - c_pv) T^r)
    (Sec. 2, Eqs. energy and muij)."""
    c_vd = R_d / (gamma_d - 1.0)
    c_pv = vap.sigma_v * c_vd + R_d / vap.eps
    c_l = vap.cond[0].sigma_v * c_vd
    mu_c = -(vap.cond[0].L_ref + (c_l - c_pv) * vap.T_ref)
    nmom = 3 if ny > 1 else 2
    Y = np.zeros((1 + 1 + 2 + nmom + 1, nz, ny, nx))
    Y[0], Y[1], Y[2] = rho_d, rho_v, rho_c
    Y[-1] = (c_vd * rho_d + vap.sigma_v * c_vd * rho_v + c_l * rho_c) * T + mu_c * rho_c
    return Y


def ensemble(sizes=(64, 128, 256, 512), per_size=24, seed=BASE_SEED + 4, nsteps=200):
    """Ensemble of 2-D moist bubbles of uneven sizes on 1 km boxes: amplitude ~ U(0.2, 2) K
    and radius ~ U(150, 400) m drawn per member from the seeded stream."""
    members = []
    nmem = len(sizes) * per_size
    u = rng.uniform(seed, 2 * nmem)
    m = 0
    for n in sizes:
        for _ in range(per_size):
            A = 0.2 + 1.8 * u[2 * m]
            R = 150.0 + 250.0 * u[2 * m + 1]
            members.append(moist_bubble(n=n, A=A, R=R, zc=450.0, nsteps=nsteps, seed=seed + m))
            m += 1
    return members


def adjoint_bubble(n=256, dtype="f64", nsteps=400):
    """2-D dry warm bubble of the first workload on an n x n grid."""
    w = warm_bubble(n=n, nsteps=nsteps, dtype=dtype)
    w.name = f"adjoint_bubble_{n}x{n}"
    return w


# --------------------------------------------------------------------------
# generic perturbations for parity tests
# --------------------------------------------------------------------------
def add_random_motion(w: Workload, amp_u=2.0, seed=BASE_SEED + 99) -> Workload:
    """Add a seeded random velocity field (m/s) at fixed temperature: momentum and the
    kinetic part of the total energy change; densities are unchanged."""
    Y = w.Y.copy()
    nv = w.nv
    im0 = 1 + w.nvapor * (1 + w.ncond)
    rho = Y[:im0].sum(axis=0)
    n = w.ncells
    ke = np.zeros_like(rho)
    for m in range(w.nmom):
        u = amp_u * (2.0 * rng.uniform(seed, n, offset=m * n) - 1.0).reshape(rho.shape)
        Y[im0 + m] = rho * u
        ke += 0.5 * rho * u * u
    Y[nv - 1] += ke
    return w.with_state(Y)


def crop(w: Workload, nx: int, ny: int, i0: int = 0, j0: int = 0) -> Workload:
    """Horizontal crop of a workload (keeps all levels and the reference profile)."""
    Y = w.Y[:, :, j0:j0 + ny, i0:i0 + nx]
    return dataclasses.replace(w, nx=nx, ny=ny, Y=np.ascontiguousarray(Y),
                               name=f"{w.name}_crop{nx}x{ny}")
