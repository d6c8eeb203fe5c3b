"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

Holds no part of the numerical scheme: only initial states, reference profiles and
physical parameters of the workloads.
"""
from .configs import (REFLECT, PERIODIC, NOSLIP, RHAT, BASE_SEED, Condensate, Vapor, Workload,
                      warm_bubble, density_current, rest_state, isothermal_rest, dry_bubble_3d,
                      jovian, jovian_rce, moist_bubble, ensemble, adjoint_bubble, moist_adjoint_bubble,
                      bryan_moist_bubble,
                      add_random_motion, crop, cosine_bubble, earth_water, jovian_species)
from . import rng

__all__ = ["REFLECT", "PERIODIC", "NOSLIP", "RHAT", "BASE_SEED", "Condensate", "Vapor", "Workload",
           "warm_bubble", "density_current", "rest_state", "isothermal_rest", "dry_bubble_3d",
           "jovian", "jovian_rce", "moist_bubble", "ensemble", "adjoint_bubble", "moist_adjoint_bubble",
           "bryan_moist_bubble",
           "add_random_motion", "crop", "cosine_bubble", "earth_water", "jovian_species", "rng"]
