"""ctypes binding of the C ABI in include/snap.h (argument marshalling only).

Every step of the numerical method runs in the CUDA library libsnap_gb300.so; this module
only fills descriptors and passes pointers. Importing it without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnap_gb300.so")

MAX_VAPOR = 4
MAX_COND = 2
MAX_FIELDS = 24

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ENOCONV, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
REFLECT, PERIODIC, NOSLIP, HALO = 0, 1, 2, 3
F64, F32 = 0, 1

# every function declared in include/snap.h
EXPORTS = ["snap_init_grid", "snap_set_state", "snap_get_state", "snap_step", "snap_step_async",
           "snap_step_io",
           "snap_stage", "snap_check", "snap_reset_flags", "snap_budget_compute",
           "snap_compute_dt", "snap_saturation_adjust", "snap_record", "snap_step_adjoint",
           "snap_set_stream",
           "snap_use_graph", "snap_set_tile_variant", "snap_use_persistent", "snap_autotune",
           "snap_set_barrier_test", "snap_link_halo", "snap_halo_buffer", "snap_halo_pack",
           "snap_set_class_tile_variant", "snap_get_class_info",
           "snap_get_info", "snap_buffer_pointer", "snap_budget_noalloc", "snap_theta_e",
           "snap_probe_fma", "snap_check_rcp64", "snap_check_weno",
           "snap_free", "snap_last_error", "snap_status_string"]


class Species(C.Structure):
    _fields_ = [("eps", C.c_double), ("sigma_v", C.c_double), ("T_ref", C.c_double),
                ("p_ref", C.c_double), ("sigma_c", C.c_double * MAX_COND),
                ("L_ref", C.c_double * MAX_COND)]


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("bc", C.c_int * 6), ("grav", C.c_double), ("gamma_d", C.c_double),
                ("R_d", C.c_double), ("n_vapor", C.c_int), ("n_cond", C.c_int),
                ("species", Species * MAX_VAPOR),
                ("rho_bar", C.POINTER(C.c_double)), ("p_bar_face", C.POINTER(C.c_double)),
                ("dtype", C.c_int), ("cfl", C.c_double), ("nu", C.c_double),
                ("satadj", C.c_int), ("satadj_max_iter", C.c_int), ("satadj_tol", C.c_double),
                ("weno_eps", C.c_double),
                ("w_term", C.c_double * MAX_COND),
                ("kessler", C.c_int), ("kessler_k", C.c_double * 4),
                ("kessler_max_iter", C.c_int), ("kessler_tol", C.c_double),
                ("cool_rate", C.c_double), ("cool_p_lo", C.c_double), ("cool_p_hi", C.c_double),
                ("sponge_tau0", C.c_double), ("sponge_p0", C.c_double),
                ("T_bottom", C.c_double)]


class Budget(C.Structure):
    _fields_ = [("nfields", C.c_int), ("total", C.c_double * MAX_FIELDS),
                ("energy_with_potential", C.c_double), ("dt_last", C.c_double),
                ("flags", C.c_uint), ("satadj_max_sweeps", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_domains", C.c_int), ("nfields", C.c_int), ("ncells_total", C.c_longlong),
                ("state_bytes", C.c_longlong), ("tile", C.c_int * 3), ("tiles_total", C.c_int),
                ("kernel_launches_per_step", C.c_int), ("tile_variant", C.c_int),
                ("n_tile_variants", C.c_int), ("persistent", C.c_int),
                ("persistent_grid", C.c_int), ("n_size_classes", C.c_int),
                ("per_class_tiles", C.c_int)]


class SnapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_LIB = None


def load(path: Optional[str] = None) -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.snap_init_grid.argtypes = [C.POINTER(P), C.POINTER(GridDesc), C.c_int]
    lib.snap_set_state.argtypes = [P, C.c_int, P, C.c_int, C.c_int, P]
    lib.snap_get_state.argtypes = [P, C.c_int, P, C.c_int, C.c_int, P]
    lib.snap_step.argtypes = [P, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(Budget)]
    lib.snap_step_async.argtypes = [P, C.c_int, C.c_double]
    lib.snap_step_io.argtypes = [P, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double]
    lib.snap_stage.argtypes = [P, C.c_int, C.c_double]
    lib.snap_check.argtypes = [P, C.POINTER(C.c_uint)]
    lib.snap_reset_flags.argtypes = [P]
    lib.snap_budget_compute.argtypes = [P, C.c_int, C.POINTER(Budget)]
    lib.snap_compute_dt.argtypes = [P, C.c_int, C.POINTER(C.c_double)]
    lib.snap_saturation_adjust.argtypes = [P, C.c_int]
    lib.snap_step_adjoint.argtypes = [P, C.c_int, P, P, C.c_int, P]
    lib.snap_record.argtypes = [P, C.c_int, C.c_int, C.c_double]
    lib.snap_set_stream.argtypes = [P, P]
    lib.snap_use_graph.argtypes = [P, C.c_int]
    lib.snap_get_info.argtypes = [P, C.POINTER(Info)]
    lib.snap_set_tile_variant.argtypes = [P, C.c_int]
    lib.snap_use_persistent.argtypes = [P, C.c_int]
    lib.snap_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.snap_set_barrier_test.argtypes = [P, C.c_longlong, C.c_int]
    lib.snap_link_halo.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.snap_set_class_tile_variant.argtypes = [P, C.c_int, C.c_int]
    lib.snap_get_class_info.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.snap_halo_buffer.argtypes = [P, C.c_int, C.c_int, C.POINTER(P)]
    lib.snap_halo_pack.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P]
    lib.snap_buffer_pointer.argtypes = [P, C.c_int, C.c_int, C.POINTER(P)]
    lib.snap_probe_fma.argtypes = [C.c_int, C.POINTER(C.c_double), P]
    lib.snap_check_rcp64.argtypes = [P, P, C.c_longlong, P]
    lib.snap_check_weno.argtypes = [C.c_int, C.c_int, P, P, C.c_longlong, C.c_double, P]
    lib.snap_budget_noalloc.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_double, P, P]
    lib.snap_theta_e.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.c_int]
    lib.snap_free.argtypes = [P]
    lib.snap_free.restype = None
    lib.snap_last_error.argtypes = [P]
    lib.snap_last_error.restype = C.c_char_p
    lib.snap_status_string.argtypes = [C.c_int]
    lib.snap_status_string.restype = C.c_char_p
    _LIB = lib
    return lib


def desc_from_workload(w, dtype: Optional[str] = None, satadj: Optional[bool] = None):
    """GridDesc of a workloads.Workload (the arrays it points to are returned to keep alive)."""
    d = GridDesc()
    d.nx, d.ny, d.nz = w.nx, w.ny, w.nz
    d.dx, d.dy, d.dz = w.dx, w.dy, w.dz
    for s in range(6):
        d.bc[s] = int(w.bc[s])
    d.grav, d.gamma_d, d.R_d = w.grav, w.gamma_d, w.R_d
    d.n_vapor, d.n_cond = len(w.vapors), w.ncond
    for i, v in enumerate(w.vapors):
        sp = d.species[i]
        sp.eps, sp.sigma_v, sp.T_ref, sp.p_ref = v.eps, v.sigma_v, v.T_ref, v.p_ref
        for j in range(w.ncond):
            sp.sigma_c[j] = v.cond[j].sigma_v
            sp.L_ref[j] = v.cond[j].L_ref
    keep = (np.ascontiguousarray(w.rho_bar, dtype=np.float64),
            np.ascontiguousarray(w.p_bar_face, dtype=np.float64))
    d.rho_bar = keep[0].ctypes.data_as(C.POINTER(C.c_double))
    d.p_bar_face = keep[1].ctypes.data_as(C.POINTER(C.c_double))
    dt = w.dtype if dtype is None else dtype
    d.dtype = F32 if dt == "f32" else F64
    d.cfl, d.nu = w.cfl, w.nu
    d.satadj = int((len(w.vapors) > 0 and w.ncond > 0) if satadj is None else satadj)
    d.satadj_max_iter, d.satadj_tol = w.satadj_max_iter, w.satadj_tol
    d.weno_eps = w.weno_eps
    for j, wt in enumerate(getattr(w, "w_term", ())):
        d.w_term[j] = wt
    kk = tuple(getattr(w, "kessler_k", ()))
    d.kessler = int(len(kk) == 4)
    for r, kv in enumerate(kk):
        d.kessler_k[r] = kv
    d.kessler_max_iter = getattr(w, "kessler_max_iter", 30)
    d.kessler_tol = getattr(w, "kessler_tol", 1e-12)
    cool = tuple(getattr(w, "cooling", ()))
    if cool:
        d.cool_rate, d.cool_p_lo, d.cool_p_hi = cool
    sponge = tuple(getattr(w, "sponge", ()))
    if sponge:
        d.sponge_tau0, d.sponge_p0 = sponge
    d.T_bottom = float(getattr(w, "T_bottom", 0.0))
    return d, keep


class Context:
    """One library context (snap_ctx) over one or more domains."""

    def __init__(self, workloads: Sequence, dtype: Optional[str] = None,
                 satadj: Optional[bool] = None):
        self.lib = load()
        ws = list(workloads) if isinstance(workloads, (list, tuple)) else [workloads]
        self.workloads = ws
        descs, self._keep = [], []
        for w in ws:
            d, k = desc_from_workload(w, dtype, satadj)
            descs.append(d)
            self._keep.append(k)
        arr = (GridDesc * len(descs))(*descs)
        self._ptr = C.c_void_p()
        rc = self.lib.snap_init_grid(C.byref(self._ptr), arr, len(descs))
        if rc:
            raise SnapError(rc, self.lib.snap_last_error(None).decode())
        self.f32 = descs[0].dtype == F32
        self.np_dtype = np.float32 if self.f32 else np.float64

    def _check(self, rc):
        if rc:
            raise SnapError(rc, self.lib.snap_last_error(self._ptr).decode())
        return rc

    def close(self):
        if self._ptr:
            self.lib.snap_free(self._ptr)
            self._ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state --------------------------------------------------------------------------
    def _sized(self, Y, domain, what):
        w = self.workloads[domain]
        n = w.nv * w.nz * w.ny * w.nx
        if (Y.size if isinstance(Y, np.ndarray) else Y.numel()) != n:
            raise ValueError(f"{what}: expected {n} values (nv, nz, ny, nx) = "
                             f"{(w.nv, w.nz, w.ny, w.nx)} for domain {domain}")
        return Y

    def set_state(self, Y, domain=0, stream=None):
        """Y: numpy array (host) or torch tensor (CUDA or CPU), float32 or float64."""
        ptr, dt, dev = _buffer(self._sized(Y, domain, "set_state"))
        return self._check(self.lib.snap_set_state(self._ptr, domain, ptr, dt, dev, stream))

    def get_state(self, domain=0, out=None, dtype=np.float64, stream=None):
        w = self.workloads[domain]
        if out is None:
            out = np.empty((w.nv, w.nz, w.ny, w.nx), dtype=dtype)
        ptr, dt, dev = _buffer(self._sized(out, domain, "get_state"))
        self._check(self.lib.snap_get_state(self._ptr, domain, ptr, dt, dev, stream))
        return out

    # -- stepping -----------------------------------------------------------------------
    def step(self, nsteps=1, dt_fixed=0.0):
        dt = C.c_double(0.0)
        self._check(self.lib.snap_step(self._ptr, nsteps, dt_fixed, C.byref(dt), None))
        return dt.value

    def step_async(self, nsteps=1, dt_fixed=0.0):
        return self._check(self.lib.snap_step_async(self._ptr, nsteps, dt_fixed))

    def step_io(self, Y=None, out=None, nsteps=1, dt_fixed=0.0, domain=0):
        """snap_step_io: optionally load Y, advance nsteps, optionally write the result into
        out (numpy array or torch tensor of the state's shape, float32 or float64; the same
        type as Y when both are given). Returns out."""
        ptr_in, dt_in, ptr_out, dt_out = None, None, None, None
        if Y is not None:
            ptr_in, dt_in, _ = _buffer(self._sized(Y, domain, "step_io"))
        if out is not None:
            ptr_out, dt_out, _ = _buffer(self._sized(out, domain, "step_io"))
        if dt_in is not None and dt_out is not None and dt_in != dt_out:
            raise ValueError("step_io: Y and out must have the same type")
        dt = dt_in if dt_in is not None else (dt_out if dt_out is not None else
                                                 (F32 if self.f32 else F64))
        self._check(self.lib.snap_step_io(self._ptr, domain, ptr_in, ptr_out, dt, nsteps,
                                          dt_fixed))
        return out

    def stage(self, stage, dt_fixed=0.0):
        return self._check(self.lib.snap_stage(self._ptr, stage, dt_fixed))

    def check(self):
        f = C.c_uint(0)
        rc = self.lib.snap_check(self._ptr, C.byref(f))
        return rc, f.value

    def reset_flags(self):
        return self._check(self.lib.snap_reset_flags(self._ptr))

    def budget(self, domain=0):
        b = Budget()
        self._check(self.lib.snap_budget_compute(self._ptr, domain, C.byref(b)))
        n = b.nfields
        return {"total": np.array(b.total[:n]), "energy_with_potential": b.energy_with_potential,
                "dt_last": b.dt_last, "flags": b.flags, "satadj_max_sweeps": b.satadj_max_sweeps}

    def theta_e(self, domain=0):
        """Equivalent potential temperature of every cell (snap_theta_e), FP64 numpy array
        shaped (nz, ny, nx)."""
        w = self.workloads[domain]
        out = np.empty((w.nz, w.ny, w.nx), dtype=np.float64)
        self._check(self.lib.snap_theta_e(self._ptr, domain,
                                          out.ctypes.data_as(C.POINTER(C.c_double)), 0))
        return out

    def compute_dt(self, domain=0):
        dt = C.c_double(0.0)
        self._check(self.lib.snap_compute_dt(self._ptr, domain, C.byref(dt)))
        return dt.value

    def saturation_adjust(self, domain=0):
        return self._check(self.lib.snap_saturation_adjust(self._ptr, domain))

    def record(self, nsteps, ckpt_every=20, dt_fixed=0.0):
        """Forward run kept for the adjoint (see snap_record)."""
        return self._check(self.lib.snap_record(self._ptr, nsteps, ckpt_every, dt_fixed))

    def step_adjoint(self, nsteps, lam_final, out=None):
        """lambda_init = (dY_N/dY_0)^T lambda_final for the last recorded run; lam_final is a
        numpy array or torch tensor in the state layout."""
        if out is None:
            out = np.empty_like(lam_final) if isinstance(lam_final, np.ndarray) else \
                lam_final.new_empty(lam_final.shape)
        pin, dt_in, _ = _buffer(lam_final)
        pout, dt_out, _ = _buffer(out)
        if dt_in != dt_out:
            raise TypeError("lam_final and out must have the same dtype")
        self._check(self.lib.snap_step_adjoint(self._ptr, nsteps, pin, pout, dt_in, None))
        return out

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        h = getattr(stream, "cuda_stream", stream)
        return self._check(self.lib.snap_set_stream(self._ptr, h))

    def use_graph(self, enable=True):
        return self._check(self.lib.snap_use_graph(self._ptr, int(enable)))

    def info(self):
        i = Info()
        self._check(self.lib.snap_get_info(self._ptr, C.byref(i)))
        return {"n_domains": i.n_domains, "nfields": i.nfields, "ncells_total": i.ncells_total,
                "state_bytes": i.state_bytes, "tile": tuple(i.tile), "tiles_total": i.tiles_total,
                "kernel_launches_per_step": i.kernel_launches_per_step,
                "tile_variant": i.tile_variant, "n_tile_variants": i.n_tile_variants,
                "persistent": i.persistent, "persistent_grid": i.persistent_grid,
                "n_size_classes": i.n_size_classes, "per_class_tiles": i.per_class_tiles,
                "classes": [self.class_info(c) for c in range(i.n_size_classes)]}

    def class_info(self, cls):
        nd, cells, var = C.c_int(0), C.c_int(0), C.c_int(0)
        tile = (C.c_int * 3)()
        self._check(self.lib.snap_get_class_info(self._ptr, cls, C.byref(nd), C.byref(cells),
                                                 tile, C.byref(var)))
        return {"domains": nd.value, "cells": cells.value, "tile": tuple(tile),
                "variant": var.value}

    def set_class_tile_variant(self, cls, variant):
        return self._check(self.lib.snap_set_class_tile_variant(self._ptr, cls, variant))

    def set_tile_variant(self, variant):
        return self._check(self.lib.snap_set_tile_variant(self._ptr, variant))

    def use_persistent(self, mode=True):
        """Launch mode of a step: 0/False three launches, 1/True one persistent launch with
        grid barriers, 2 the resident step (see snap_use_persistent)."""
        return self._check(self.lib.snap_use_persistent(self._ptr, int(mode)))

    def set_barrier_test(self, spin_cycles=0, absent_cta=-1):
        """Test aid of the persistent step's grid barrier (see snap_set_barrier_test)."""
        return self._check(self.lib.snap_set_barrier_test(self._ptr, int(spin_cycles),
                                                          int(absent_cta)))

    def autotune(self, steps=5):
        ms = C.c_double(0.0)
        choice = C.c_int(0)
        self._check(self.lib.snap_autotune(self._ptr, steps, C.byref(ms), C.byref(choice)))
        if choice.value < 0:
            return {"ms_per_step": ms.value, "variant": None, "persistent": 0,
                    "per_class": [self.class_info(c)["variant"]
                                  for c in range(self.info()["n_size_classes"])]}
        return {"ms_per_step": ms.value, "variant": choice.value // 3,
                "persistent": choice.value % 3}

    # -- slab decomposition (SNAP_HALO sides) ---------------------------------------------
    def link_halo(self, domain, side, nbr):
        """Ghost columns of `side` (0: x-, 1: x+) read from domain nbr (see snap_link_halo)."""
        return self._check(self.lib.snap_link_halo(self._ptr, domain, side, nbr))

    def halo_view(self, domain=0, side=0):
        """Zero-copy torch view (nfields, nz, ny, 3) of a side's ghost buffer, which the caller
        fills before each stage (see snap_halo_buffer)."""
        import torch
        p = C.c_void_p()
        self._check(self.lib.snap_halo_buffer(self._ptr, domain, side, C.byref(p)))
        w = self.workloads[domain]
        return _device_view((w.nv, w.nz, w.ny, 3), self.f32, p.value)

    def halo_pack(self, domain, side, slot, out, stream=None):
        """The three columns next to `side` of state buffer `slot` into the device tensor out
        (see snap_halo_pack)."""
        if not (out.is_cuda and out.is_contiguous()):
            raise ValueError("out must be a contiguous CUDA tensor")
        return self._check(self.lib.snap_halo_pack(self._ptr, domain, side, slot,
                                                   C.c_void_p(out.data_ptr()), stream))

    def buffer_pointer(self, domain=0, slot=0):
        p = C.c_void_p()
        self._check(self.lib.snap_buffer_pointer(self._ptr, domain, slot, C.byref(p)))
        return p.value

    def buffer_view(self, domain=0, slot=0):
        """Zero-copy torch view of a device state buffer (see snap_buffer_pointer)."""
        w = self.workloads[domain]
        return _device_view((w.nv, w.nz, w.ny, w.nx), self.f32,
                            self.buffer_pointer(domain, slot))


def _device_view(shape, f32, ptr):
    """torch tensor over device memory the library owns (no copy)."""
    import torch

    class _Dev:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4" if f32 else "<f8",
                                    "data": (ptr, False), "version": 2}

    return torch.as_tensor(_Dev(), device="cuda")


def _buffer(Y):
    """(pointer, dtype code, on_device) of a numpy array or torch tensor."""
    if isinstance(Y, np.ndarray):
        if not Y.flags["C_CONTIGUOUS"]:
            raise ValueError("state array must be C-contiguous")
        if Y.dtype == np.float64:
            return C.c_void_p(Y.ctypes.data), F64, 0
        if Y.dtype == np.float32:
            return C.c_void_p(Y.ctypes.data), F32, 0
        raise TypeError("state must be float32 or float64")
    import torch  # torch tensors: plumbing only (memory and streams)
    if not Y.is_contiguous():
        raise ValueError("state tensor must be contiguous")
    code = {torch.float64: F64, torch.float32: F32}[Y.dtype]
    return C.c_void_p(Y.data_ptr()), code, int(Y.is_cuda)


def check_rcp64(x_ptr, y_ptr, n, stream=None):
    """Device pointers: y[2i] = the FP64 kernels' reciprocal of x[i], y[2i+1] = 1 / x[i]
    (see snap_check_rcp64)."""
    rc = load().snap_check_rcp64(x_ptr, y_ptr, n, stream)
    if rc:
        raise SnapError(rc, "snap_check_rcp64 failed")


def check_weno(dtype, packed, win_ptr, out_ptr, n, eps, stream=None):
    """Device pointers: the kernels' WENO5 face states of n five-value windows (see
    snap_check_weno)."""
    rc = load().snap_check_weno(F32 if dtype == "f32" else F64, int(packed), win_ptr, out_ptr,
                                n, eps, stream)
    if rc:
        raise SnapError(rc, "snap_check_weno failed")


def probe_fma(dtype="f32", stream=None):
    """Achieved fused multiply-add rate of the device in TFLOP/s (see snap_probe_fma)."""
    lib = load()
    t = C.c_double(0.0)
    rc = lib.snap_probe_fma(F32 if dtype == "f32" else F64, C.byref(t), stream)
    if rc:
        raise SnapError(rc, "snap_probe_fma failed")
    return t.value
