"""Oracle: a plain, slow, float64 CPU restatement of the iHDG method.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check in
__graft_entry__.py and the CPU-baseline leg of bench.py may import or run it.  The CUDA
library never calls it, shares no code, tables or constants with it, and must fail loudly
rather than fall back to it.

Contents:
  refelem   GLL / Gauss / Lagrange reference-element tables
  mesh      uniform box meshes, faces and neighbours
  ihdg      the upwind HDG local problems (transport, convection-diffusion, linearized
            shallow water), Algorithm 1, and a static-condensation direct solve
  krylov    restarted GMRES (Saad and Schultz) and GMRES around the iHDG sweep

Every function is pinned by tests under tests/ against closed forms, brute force, the
direct HDG solve, polynomial exactness, manufactured-solution convergence rates and the
contraction results the paper states (Theorem 1 and the remark after it).
"""
from .mesh import BoxMesh
from .refelem import RefElement, gll_nodes, gauss_rule, lagrange_matrix, lagrange_deriv_matrix
from .ihdg import (Discretisation, Transport, TransportVar, ConvDiff, ShallowWater, ShallowWaterCN,
                   STATUS_OK, STATUS_NOT_CONVERGED, STATUS_DIVERGED)
from .krylov import gmres, ihdg_gmres
