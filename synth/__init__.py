"""Seeded synthetic catalogue generators shared by the oracle tests and the GPU path.

This package draws random inputs only (positions, weights, the expected number
density at each position, and the geometry of the analysis box).  It contains none
of the estimator's arithmetic: no mesh assignment, no Fourier transform of the
density field, no binning.
"""
from .catalogs import (Catalog, Geometry, poisson_cube, poisson_shell, zeldovich_cone,
                       zeldovich_cube, batched_cube_specs, on_node_catalog, paper_cap,
                       workload)

__all__ = ["Catalog", "Geometry", "poisson_cube", "poisson_shell", "zeldovich_cone",
           "zeldovich_cube", "batched_cube_specs", "on_node_catalog", "paper_cap", "workload"]
