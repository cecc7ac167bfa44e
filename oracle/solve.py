"""Jacobi-preconditioned conjugate gradients for the oracle (Sec. 5 and Sec. 5.3).

Textbook PCG (Hestenes-Stiefel form) on the constrained system
A_c x = P b with A_c = P A P + (I - P) and the preconditioner
z = diag(A_c)^-1 r.  Stopping rule: ||r_k||_2 <= rtol ||P b||_2 on the
recurrence residual, starting from x0 = 0.
"""
from __future__ import annotations

import numpy as np


def jacobi_pcg(op, b, rtol=1e-10, max_it=10000):
    """Return (x, iterations, final relative recurrence residual, converged)."""
    mesh = op.mesh
    bc = np.where(mesh.dirichlet, 0.0, np.asarray(b, dtype=np.float64))
    dinv = 1.0 / op.diagonal(constrained=True)
    x = np.zeros(mesh.n_dof)
    r = bc.copy()
    bnorm = np.linalg.norm(bc)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for it in range(1, max_it + 1):
        Ap = op.apply(p, constrained=True)
        pAp = p @ Ap
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        a = rz / pAp
        x += a * p
        r -= a * Ap
        rel = np.linalg.norm(r) / bnorm
        if rel <= rtol:
            return x, it, rel, True
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_it, rel, False


def jacobi_pcg_nullspace(op, b, rtol=1e-10, max_it=10000):
    """Jacobi-PCG for the pure-Neumann Poisson problem (no Dirichlet DoFs, alpha = 0).

    The operator K has the constants as null space (Sec. 5.3).  Following the
    paper: the right-hand side is made orthogonal to the null space, every
    preconditioner application is followed by an orthogonalization against it,
    and the solution is closed with the mean-zero condition int p dx = 0
    (Sec. 4.2, Eq. (meanZero)), i.e. m1 . x = 0 with m1_i = int phi_i dx.

    Returns (x, iterations, final relative recurrence residual, converged).
    """
    from .fem import Operator
    mesh = op.mesh
    n = mesh.n_dof
    b = np.asarray(b, dtype=np.float64)
    bc = b - b.mean()                        # orthogonal to the constants
    d = op.diagonal()
    x = np.zeros(n)
    r = bc.copy()
    bnorm = np.linalg.norm(bc)
    m1 = Operator(mesh, 1.0, 0.0).apply(np.ones(n))   # m1_i = int phi_i dx
    if bnorm == 0.0:
        return x, 0, 0.0, True

    def precond(v):
        z = v / d
        return z - z.mean()                  # orthogonalization step

    z = precond(r)
    p = z.copy()
    rz = r @ z
    rel = 1.0
    for it in range(1, max_it + 1):
        Ap = op.apply(p)
        pAp = p @ Ap
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        a = rz / pAp
        x += a * p
        r -= a * Ap
        rel = np.linalg.norm(r) / bnorm
        if rel <= rtol:
            break
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    x -= (m1 @ x) / m1.sum()                 # mean-zero closure
    return x, it, rel, rel <= rtol
