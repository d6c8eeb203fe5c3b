"""GB300 (sm_103a) implementation of one explicit finite-volume step of the SNAP model
(Li & Chen 2019): WENO5 reconstruction, LMARS flux, flux divergence with gravity, SSP-RK3
stage combine and saturation adjustment, fused in CUDA kernels behind the C ABI of
include/snap.h. This package is the thin Python binding of that library."""
from .capi import (Context, SnapError, load, desc_from_workload, LIB_PATH, EXPORTS, F32, F64,
                   REFLECT, PERIODIC, HALO)

__all__ = ["Context", "SnapError", "load", "desc_from_workload", "LIB_PATH", "EXPORTS", "F32",
           "F64", "REFLECT", "PERIODIC", "HALO"]
