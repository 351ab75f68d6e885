"""GB300-native ADER-DG step for 3-D waves in a continuum-damage (CDM) rock.

The compute path is libdg (C-ABI in include/dg.h, CUDA kernels for sm_103a in
csrc/); this package holds its in-tree build and a thin ctypes binding.
"""
from .build import LIB_PATH, build
from .dg import (DGError, Solver, host_chunks, load_library, misfit_function, n_modes, reference_table,
                 revolve_cost, revolve_plan, torch_allocator)

__all__ = ["LIB_PATH", "build", "DGError", "Solver", "host_chunks", "load_library", "misfit_function", "n_modes",
           "reference_table", "revolve_cost", "revolve_plan", "torch_allocator"]
