"""CPU FP64 oracle for the matrix-free Q_p Helmholtz operator and its Jacobi-PCG solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library and its Python binding) never calls it and shares no code with it.

The oracle computes the plain definitions of the paper's Section 3 with no sum
factorization: explicit element matrices

    A^K_ij = sum_q w_q detJ_q ( alpha phi_i phi_j + nu_q (J^-T grad phi_i).(J^-T grad phi_j) )

(mass, Eq. (vectorMass); stiffness, Eqs. (localStiffness)-(localStiffnessQuadrature)),
with the 3D basis built from full tensor products of 1D Lagrange polynomials
on the Gauss-Lobatto points and tensor Gauss quadrature (Sec. 3.1), the
element-sum assembly of the action (Sec. 3.1), and the textbook preconditioned
conjugate gradient method (Sec. 5, Sec. 5.3) with a Jacobi (diagonal)
preconditioner.

Readings of the paper used here (where it is silent or ambiguous):
  * J_ij = dx_i/dxi_j, so the stiffness coefficient is nu w detJ J^-1 J^-T
    (the paper's J^-T |J| J^-1 is the transposed-Jacobian convention);
  * reference cube [-1,1]^3, n_q = p + 2 Gauss points per direction;
  * trilinear element maps from 8 vertices (a subset of Q_p isoparametric maps);
  * Dirichlet rows eliminated symmetrically: A_c = P A P + (I - P), P zeroing
    Dirichlet DoFs; the right-hand side is masked, b_c = P b;
  * CG stops when ||r_k||_2 <= rtol ||b_c||_2 (recurrence residual, x0 = 0).

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, exact polynomial integrals, invariants and brute force.
"""
from .basis import gll_nodes, gauss_rule, lagrange_values, lagrange_derivatives, legendre
from .fem import StructuredMesh, Mesh, Operator, ReferenceElement, load_vector, l2_error, trilinear_map
from .solve import jacobi_pcg, jacobi_pcg_nullspace

__all__ = [
    "gll_nodes", "gauss_rule", "lagrange_values", "lagrange_derivatives", "legendre",
    "StructuredMesh", "Mesh", "Operator", "ReferenceElement", "load_vector", "l2_error",
    "trilinear_map", "jacobi_pcg", "jacobi_pcg_nullspace",
]
