"""ctypes binding of the C oracle (snap_oracle.c) -- test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snap_oracle.c")
_HDR = os.path.join(_HERE, "snap_oracle.h")

MAXV = 4
MAXC = 2


def lib_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (plain -O2, no fast-math).
    SNAP_ORACLE_LIB names a prebuilt library to load instead (the mutation test uses it to
    run the pins against deliberately broken copies of the oracle)."""
    alt = os.environ.get("SNAP_ORACLE_LIB")
    if alt:
        return alt
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


class _Grid(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("bc", C.c_int * 6),
        ("grav", C.c_double), ("gamma_d", C.c_double), ("Rd", C.c_double),
        ("nvap", C.c_int), ("ncond", C.c_int),
        ("eps", C.c_double * MAXV), ("sig_v", C.c_double * MAXV),
        ("Tref", C.c_double * MAXV), ("pref", C.c_double * MAXV),
        ("sig_c", (C.c_double * MAXC) * MAXV), ("Lref", (C.c_double * MAXC) * MAXV),
        ("rho_bar", C.POINTER(C.c_double)), ("p_bar_face", C.POINTER(C.c_double)),
        ("nu", C.c_double),
        ("satadj", C.c_int), ("satadj_max_iter", C.c_int), ("satadj_tol", C.c_double),
        ("weno_eps", C.c_double),
        ("gravity_energy_pointwise", C.c_int),
        ("w_term", C.c_double * MAXC),
        ("kessler", C.c_int), ("kessler_k", C.c_double * 4),
        ("kessler_max_iter", C.c_int), ("kessler_tol", C.c_double),
        ("cool_rate", C.c_double), ("cool_p_lo", C.c_double), ("cool_p_hi", C.c_double),
        ("sponge_tau0", C.c_double), ("sponge_p0", C.c_double),
        ("T_bottom", C.c_double),
    ]


_D = C.POINTER(C.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _load():
    lib = C.CDLL(build())
    G = C.POINTER(_Grid)
    lib.orc_nvar.argtypes = [G]
    lib.orc_weno5.argtypes = [_D, C.c_double]
    lib.orc_weno5.restype = C.c_double
    lib.orc_weno5_poly.argtypes = [_D]
    lib.orc_weno5_poly.restype = C.c_double
    lib.orc_weno5_weights.argtypes = [_D, C.c_double, _D]
    lib.orc_cons_to_prim.argtypes = [G, _D, _D, _D, _D]
    lib.orc_prim_to_cons.argtypes = [G, _D, _D]
    lib.orc_sat_pressure.argtypes = [G, C.c_int, C.c_double]
    lib.orc_sat_pressure.restype = C.c_double
    lib.orc_lmars.argtypes = [G, _D, _D, C.c_int, C.c_double, _D, _D, _D]
    lib.orc_satadj_cell.argtypes = [G, _D, C.c_int, C.c_double]
    lib.orc_satadj_bisect.argtypes = [G, _D]
    lib.orc_rhs.argtypes = [G, _D, _D]
    lib.orc_rk3_combine.argtypes = [C.c_int, C.c_long, _D, _D, _D, C.c_double, _D]
    lib.orc_stage.argtypes = [G, C.c_int, _D, _D, C.c_double, _D]
    lib.orc_step.argtypes = [G, _D, C.c_int, C.c_double, C.c_double, _D]
    lib.orc_dt_cfl.argtypes = [G, _D, C.c_double]
    lib.orc_dt_cfl.restype = C.c_double
    lib.orc_budget.argtypes = [G, _D, _D]
    lib.orc_weno5_gradient.argtypes = [_D, C.c_double, _D]
    lib.orc_weno5_gradient.restype = C.c_double
    lib.orc_rhs_adjoint.argtypes = [G, _D, _D, _D]
    lib.orc_step_adjoint.argtypes = [G, _D, C.c_double, _D, _D]
    lib.orc_satadj_adjoint_cell.argtypes = [G, _D, _D, _D]
    lib.orc_kessler_cell.argtypes = [G, _D, C.c_double]
    lib.orc_theta_e.argtypes = [G, _D, _D]
    return lib


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


def grid_from_workload(w, satadj: Optional[bool] = None, nu: Optional[float] = None,
                       grav: Optional[float] = None, energy_pointwise: bool = False):
    """Fill the oracle's grid description from a workloads.Workload."""
    g = _Grid()
    g.nx, g.ny, g.nz = w.nx, w.ny, w.nz
    g.dx, g.dy, g.dz = w.dx, w.dy, w.dz
    for s in range(6):
        g.bc[s] = int(w.bc[s])
    g.grav = w.grav if grav is None else grav
    g.gamma_d, g.Rd = w.gamma_d, w.R_d
    g.nvap, g.ncond = len(w.vapors), w.ncond
    for i, v in enumerate(w.vapors):
        g.eps[i], g.sig_v[i], g.Tref[i], g.pref[i] = v.eps, v.sigma_v, v.T_ref, v.p_ref
        for j in range(w.ncond):
            g.sig_c[i][j] = v.cond[j].sigma_v
            g.Lref[i][j] = v.cond[j].L_ref
    keep = (np.ascontiguousarray(w.rho_bar, dtype=np.float64),
            np.ascontiguousarray(w.p_bar_face, dtype=np.float64))
    g.rho_bar, g.p_bar_face = _ptr(keep[0]), _ptr(keep[1])
    g.nu = w.nu if nu is None else nu
    g.satadj = int((len(w.vapors) > 0 and w.ncond > 0) if satadj is None else satadj)
    g.satadj_max_iter, g.satadj_tol = w.satadj_max_iter, w.satadj_tol
    g.weno_eps = w.weno_eps
    g.gravity_energy_pointwise = int(energy_pointwise)
    for j, wt in enumerate(getattr(w, "w_term", ())):
        g.w_term[j] = wt
    kk = tuple(getattr(w, "kessler_k", ()))
    g.kessler = int(len(kk) == 4)
    for r, kv in enumerate(kk):
        g.kessler_k[r] = kv
    g.kessler_max_iter = getattr(w, "kessler_max_iter", 30)
    g.kessler_tol = getattr(w, "kessler_tol", 1e-12)
    cool = tuple(getattr(w, "cooling", ()))  # (rate K/s, p_lo, p_hi)
    if cool:
        g.cool_rate, g.cool_p_lo, g.cool_p_hi = cool
    sponge = tuple(getattr(w, "sponge", ()))  # (tau0 s, p0 Pa)
    if sponge:
        g.sponge_tau0, g.sponge_p0 = sponge
    g.T_bottom = float(getattr(w, "T_bottom", 0.0))
    return g, keep


class Oracle:
    """The oracle bound to one workload's grid and parameters."""

    def __init__(self, w, **kw):
        self.w = w
        self.grid, self._keep = grid_from_workload(w, **kw)
        self.lib = _lib()
        self.nv = self.lib.orc_nvar(C.byref(self.grid))
        self.shape = (self.nv, w.nz, w.ny, w.nx)

    # -- pointwise -------------------------------------------------------------------
    def cons_to_prim(self, Yc):
        Yc = np.ascontiguousarray(Yc, dtype=np.float64)
        X = np.zeros(self.nv)
        T = np.zeros(1)
        gam = np.zeros(1)
        self.lib.orc_cons_to_prim(C.byref(self.grid), _ptr(Yc), _ptr(X), _ptr(T), _ptr(gam))
        return X, T[0], gam[0]

    def prim_to_cons(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.zeros(self.nv)
        self.lib.orc_prim_to_cons(C.byref(self.grid), _ptr(X), _ptr(Y))
        return Y

    def sat_pressure(self, i, T):
        return self.lib.orc_sat_pressure(C.byref(self.grid), i, T)

    def lmars(self, XL, XR, d, pref):
        XL = np.ascontiguousarray(XL, dtype=np.float64)
        XR = np.ascontiguousarray(XR, dtype=np.float64)
        F = np.zeros(self.nv)
        us = np.zeros(1)
        ps = np.zeros(1)
        self.lib.orc_lmars(C.byref(self.grid), _ptr(XL), _ptr(XR), d, pref, _ptr(F), _ptr(us),
                           _ptr(ps))
        return F, us[0], ps[0]

    def satadj_cell(self, Yc, max_iter=None, tol=None):
        Yc = np.array(Yc, dtype=np.float64)
        it = self.lib.orc_satadj_cell(C.byref(self.grid), _ptr(Yc),
                                      self.w.satadj_max_iter if max_iter is None else max_iter,
                                      self.w.satadj_tol if tol is None else tol)
        return Yc, it

    def satadj_bisect(self, Yc):
        Yc = np.array(Yc, dtype=np.float64)
        rc = self.lib.orc_satadj_bisect(C.byref(self.grid), _ptr(Yc))
        return Yc, rc

    # -- whole grid ----------------------------------------------------------------------
    def rhs(self, Y):
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.shape)
        rc = self.lib.orc_rhs(C.byref(self.grid), _ptr(Y), _ptr(out))
        if rc:
            raise RuntimeError(f"orc_rhs failed: {rc}")
        return out

    def stage(self, stage, Yn, Ys, dt):
        Yn = np.ascontiguousarray(Yn, dtype=np.float64).reshape(self.shape)
        Ys = np.ascontiguousarray(Ys, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.shape)
        rc = self.lib.orc_stage(C.byref(self.grid), stage, _ptr(Yn), _ptr(Ys), dt, _ptr(out))
        if rc < -1:
            raise RuntimeError(f"orc_stage failed: {rc}")
        return out, rc

    def step(self, Y, nsteps=1, dt=0.0, cfl=None):
        Y = np.array(Y, dtype=np.float64).reshape(self.shape)
        dt_last = np.zeros(1)
        rc = self.lib.orc_step(C.byref(self.grid), _ptr(Y), nsteps, dt,
                               self.w.cfl if cfl is None else cfl, _ptr(dt_last))
        if rc < -1:
            raise RuntimeError(f"orc_step failed: {rc}")
        return Y, dt_last[0], rc

    def dt_cfl(self, Y, cfl=None):
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.shape)
        return self.lib.orc_dt_cfl(C.byref(self.grid), _ptr(Y), self.w.cfl if cfl is None else cfl)

    def rhs_adjoint(self, Y, mu):
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.shape)
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.shape)
        rc = self.lib.orc_rhs_adjoint(C.byref(self.grid), _ptr(Y), _ptr(mu), _ptr(out))
        if rc:
            raise RuntimeError(f"orc_rhs_adjoint failed: {rc}")
        return out

    def theta_e(self, Y):
        """Equivalent potential temperature of every cell (App. A, Eq. theta_e)."""
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.shape[1:])
        rc = self.lib.orc_theta_e(C.byref(self.grid), _ptr(Y), _ptr(out))
        if rc:
            raise RuntimeError(f"orc_theta_e failed: {rc}")
        return out

    def kessler_cell(self, Yc, dt):
        """Sec. 3 Kessler scheme on one cell (backward Euler over dt): (Y, iterations)."""
        Yc = np.array(Yc, dtype=np.float64)
        it = self.lib.orc_kessler_cell(C.byref(self.grid), _ptr(Yc), dt)
        return Yc, it

    def satadj_adjoint_cell(self, Yout, lam_out):
        """(dYout/dYin)^T lam_out of the saturation adjustment of one cell at its result."""
        Yout = np.array(Yout, dtype=np.float64)
        lam_out = np.array(lam_out, dtype=np.float64)
        out = np.zeros_like(lam_out)
        rc = self.lib.orc_satadj_adjoint_cell(C.byref(self.grid), _ptr(Yout), _ptr(lam_out),
                                              _ptr(out))
        if rc:
            raise RuntimeError(f"orc_satadj_adjoint_cell failed: {rc}")
        return out

    def step_adjoint(self, Yn, dt, lam_out):
        Yn = np.ascontiguousarray(Yn, dtype=np.float64).reshape(self.shape)
        lam_out = np.ascontiguousarray(lam_out, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.shape)
        rc = self.lib.orc_step_adjoint(C.byref(self.grid), _ptr(Yn), dt, _ptr(lam_out), _ptr(out))
        if rc:
            raise RuntimeError(f"orc_step_adjoint failed: {rc}")
        return out

    def budget(self, Y):
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.shape)
        out = np.zeros(self.nv + 1)
        self.lib.orc_budget(C.byref(self.grid), _ptr(Y), _ptr(out))
        return out


def rk3_combine(stage, Yn, Ys, L, dt):
    lib = _lib()
    Yn = np.ascontiguousarray(Yn, dtype=np.float64)
    Ys = np.ascontiguousarray(Ys, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    out = np.zeros_like(Yn)
    lib.orc_rk3_combine(stage, Yn.size, _ptr(Yn), _ptr(Ys), _ptr(L), dt, _ptr(out))
    return out


def weno5(q, eps=1e-6):
    q = np.ascontiguousarray(q, dtype=np.float64)
    return _lib().orc_weno5(_ptr(q), eps)


def weno5_poly(q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    return _lib().orc_weno5_poly(_ptr(q))


def weno5_gradient(q, eps=1e-6):
    q = np.ascontiguousarray(q, dtype=np.float64)
    g = np.zeros(5)
    v = _lib().orc_weno5_gradient(_ptr(q), eps, _ptr(g))
    return v, g


def weno5_weights(q, eps=1e-6):
    q = np.ascontiguousarray(q, dtype=np.float64)
    w = np.zeros(3)
    _lib().orc_weno5_weights(_ptr(q), eps, _ptr(w))
    return w
