"""Oracle gradients of L = 1/2 (u - u*)^T M (u - u*) where A_c(nu) u = P b(f).

Not a method of the paper (which solves forward problems only); the oracle
restates the adjoint method from its definitions, using the paper's operator
(Sec. 3.1) and the element matrices of ``fem``:

  * forward:  A_c u = P b,  b_i = sum_K sum_q w_q detJ_q f_q phi_i(xi_q)   (load vector)
  * loss:     L = 1/2 d^T M d,  d = u - u*,  M the (unconstrained) mass matrix
  * adjoint:  A_c lam = P M d        (A_c symmetric)
  * dL/df_q = w_q detJ_q sum_i phi_i(xi_q) lam_i          (b linear in f)
  * dL/dnu_q = -lam_K^T (dA^K/dnu_q) u_K
             = -w_q detJ_q (J^-T grad phi . lam_K) . (J^-T grad phi . u_K)   at point q of element K.

Pinned in tests/test_oracle_adjoint.py by central finite differences of L.
"""
from __future__ import annotations

import numpy as np

from .fem import Operator, load_vector, trilinear_map


def solve_dense(op, rhs):
    """A_c x = P rhs by a dense solve of the assembled constrained matrix (small meshes)."""
    A = op.assembled(constrained=True)
    return np.linalg.solve(A, np.where(op.mesh.dirichlet, 0.0, rhs))


def loss(mesh, alpha, nu_q, f_q, u_target):
    """L and the forward solution u."""
    op = Operator(mesh, alpha, nu_q)
    u = solve_dense(op, load_vector(mesh, f_q))
    d = u - u_target
    Md = Operator(mesh, 1.0, 0.0).apply(d)
    return 0.5 * d @ Md, u


def gradients(mesh, alpha, nu_q, f_q, u_target):
    """(L, dL/dnu (E, Q), dL/df (E, Q), u, lam)."""
    op = Operator(mesh, alpha, nu_q)
    u = solve_dense(op, load_vector(mesh, f_q))
    d = u - u_target
    g = Operator(mesh, 1.0, 0.0).apply(d)
    L = 0.5 * d @ g
    lam = solve_dense(op, g)
    dnu, df = point_gradients(mesh, u, lam)
    return L, dnu, df, u, lam


def point_gradients(mesh, u, lam, elems=None):
    """(dL/dnu, dL/df) at the quadrature points of ``elems`` (default: all) from u and lam.

    Dirichlet entries of u and lam enter as given (zero for solutions of A_c).
    """
    ref = mesh.ref
    es = np.arange(mesh.n_elem) if elems is None else np.asarray(elems)
    _, J = trilinear_map(mesh.vertices[mesh.elem_vert[es]], ref.xi)
    detJ = np.linalg.det(J)                                   # (e, Q)
    Jinv = np.linalg.inv(J)
    wdet = ref.w[None, :] * detJ
    R = np.stack([mesh.element_dofs(e) for e in es]) if mesh.restriction is None else mesh.restriction[es]
    uE, lE = u[R], lam[R]                                     # (e, N)
    # physical gradients at every point: (J^-T dphi)^T coefficient vectors
    gphys = np.einsum("qnd,eqdk->eqnk", ref.dPhi, Jinv)       # (e, Q, N, 3)
    gu = np.einsum("eqnk,en->eqk", gphys, uE)
    gl = np.einsum("eqnk,en->eqk", gphys, lE)
    dnu = -wdet * np.einsum("eqk,eqk->eq", gl, gu)
    df = wdet * (lE @ ref.Phi.T)                              # (e, Q)
    return dnu, df
