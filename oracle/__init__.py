"""Plain FP64 CPU oracle of the hybridised DG IMEX method (TEST INFRASTRUCTURE ONLY).

Only tests/, the smoke check and the benchmark's CPU baseline leg may import this package.
It shares no code with the CUDA path; the two meet only in the exchange format (nodal values
at the equispaced lattice of each cell / facet of the canonical mesh, oracle/mesh.py).
"""
from .element import LagrangeTri, Lagrange1D, triangle_quadrature, line_quadrature, lattice, lattice_1d
from .mesh import Mesh, dof_counts
from .hdg import HDG
from .bdm import bdm_project
from .tableaus import TABLEAUS, Tableau
from .solve import Oracle
from .tracer import Tracer
