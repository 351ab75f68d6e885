"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the numerical method: it only builds meshes
(vertex coordinates, vertex ids, boundary tags), per-element material tables,
point-source and receiver descriptions, all from explicit seeds.  Both the
CUDA library (through its C-ABI) and the FP64 oracle consume these arrays.
"""
from .mesh import Mesh, kuhn_box_mesh, periodic_cube_mesh
from .workloads import (
    FIELD_NAMES, rock_material, two_layer_material, uniform_material,
    dip_slip_source, receiver_grid, workload_c1, workload_c2, workload_c4, workload_small_layered,
    workload_riemann, workload_adjoint,
)

__all__ = [
    "Mesh", "kuhn_box_mesh", "periodic_cube_mesh", "FIELD_NAMES", "rock_material",
    "two_layer_material", "uniform_material", "dip_slip_source", "receiver_grid",
    "workload_c1", "workload_c2", "workload_c4", "workload_small_layered", "workload_riemann", "workload_adjoint",
]
