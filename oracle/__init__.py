"""CPU oracle for the sixth-order compact Helmholtz method (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package.  It shares no code with the CUDA path.
"""
from .helm6_oracle import (Problem, scheme_coefficients, sommerfeld_coefficients, apply_A,
                           apply_Ap, axis_matrix, rhs, lift_dirichlet, Preconditioner, gmres,
                           sks, chebyshev, dirichlet_ratio_bounds, psi_order, dense_matrix,
                           solve_dense, solve, exchange)
from . import sources
