"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws inputs: tetrahedral voxel meshes, per-tet material
parameters, Dirichlet masks, initial states and synthetic sparse bases.  It
holds none of the solver's arithmetic (no rest-shape quantities, masses,
energies or bases built by the paper's construction), so that the oracle and
the CUDA path, which both consume these inputs, share no computation.
"""
from .meshes import (  # noqa: F401
    Mesh,
    kuhn_voxel_mesh,
    lattice_mask,
    voronoi_cells,
    random_tet_mesh,
)
from .workloads import (  # noqa: F401
    Scene,
    cube_scene,
    beam_scene,
    lattice_scene,
    batched_lattice_scenes,
    tiny_scene,
    two_block_scene,
    lattice_stack_scene,
    random_sparse_basis,
    mlp_init,
)
