"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package holds input construction only: quadtree leaf-cell lists for the
benchmark meshes (octree lists and 3D initial states in ``perk_inputs.octree``), analytic initial conditions, and seeded random draws. It
holds none of the method's arithmetic (no DGSEM operator, no flux, no
Runge-Kutta coefficient), so both the product library and the oracle can take
their inputs from here without sharing any of the computation under test.
"""

from .meshes import (  # noqa: F401
    Cell,
    uniform_cells,
    refine_cells,
    morton_sort,
    vortex_two_level_cells,
    kh_band_cells,
    nested_band_cells,
    three_level_band_cells,
)
from .initial import (  # noqa: F401
    GAMMA,
    isentropic_vortex,
    kelvin_helmholtz,
    shear_layer,
    prim_to_cons,
    nodal_state,
    node_coordinates,
    smooth_random_state,
    SEED,
)
