"""Plain FP64 CPU oracle of the SNAP finite-volume step (test infrastructure).

Only tests, the smoke check and the CPU-baseline leg of the benchmark may import this
package. It shares no code with the CUDA library. See snap_oracle.c for the passages of
the paper each routine follows.
"""
from .oracle import (Oracle, build, grid_from_workload, lib_path)

__all__ = ["Oracle", "build", "grid_from_workload", "lib_path"]
