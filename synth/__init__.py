"""Seeded synthetic lattices shaped like the paper's slicing workloads.

The paper's models (Teddy ... Kitten-HR, Table 4) are not available, so these
generators stand in for their shapes: strut-graph lattices of 1e3 to 1e8
struts, struts of 0.05-0.5 mm radius, images of 4e4 to 1.6e7 pixels per layer.
This module holds no arithmetic of the method (no kernel, no field, no
contour); both the CUDA path and the CPU oracle take their inputs from here.
Random numbers come from numpy's Philox counter-based generator, seeded with
2101050310 + the configuration index (+ the lattice index in a batch).
"""
from .lattices import (  # noqa: F401
    SEED_BASE,
    adaptive_graded,
    batched_set,
    config,
    cubic_bcc,
    freudenthal,
    graded_density,
    lattice_bbox,
    rng,
)
from .tets import density_config, graded_target_grid, kuhn_tet_mesh  # noqa: F401,E402
