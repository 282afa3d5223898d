"""GB300-native hybridised DG IMEX stage solver for the incompressible Euler equations
(arXiv 2410.09790): a C-ABI CUDA library (include/hdg.h) and its Python binding."""
from .hdg import (Context, HdgError, load, hdg_default_params, hdg_mesh_counts, hdg_reference_rule,
                  hdg_reference_basis, TABLEAUS, Server, hdg_batch_step, hdg_estimate_bytes, make_params)

__all__ = ['Context', 'HdgError', 'load', 'hdg_default_params', 'hdg_mesh_counts', 'hdg_reference_rule',
           'hdg_reference_basis', 'TABLEAUS', 'Server', 'hdg_batch_step', 'hdg_estimate_bytes', 'make_params']
