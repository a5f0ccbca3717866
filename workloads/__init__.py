"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates problem data*: the basic tetrahedral mesh T (coordinates,
elements, Dirichlet and Neumann face lists, as in Section 2 "Data structure" of the paper)
and the PDE data of eq. (1.1) as plain functions of position (kappa, c, f, u_D, g_N, and the
exact solution used to manufacture them).  It holds none of the HDG method's arithmetic:
no quadrature, no basis, no local solver.  Both the oracle and the CUDA path evaluate
these functions at their own quadrature nodes.
"""

from .mesh import (boundary_faces, kuhn_coarse_interpolation, kuhn_cube, kuhn_grid_points,  # noqa: F401
                   kuhn_interpolation, kuhn_p1_hierarchy)
from .problems import PROBLEMS, Problem, get_problem  # noqa: F401
