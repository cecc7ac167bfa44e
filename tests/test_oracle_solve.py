"""Oracle Jacobi-PCG (Sec. 5, Sec. 5.3) pinned to a dense solve and to p+1 convergence (Sec. 7.2 criterion)."""
import numpy as np
import pytest

import synthetic as S
from oracle import fem
from oracle.solve import jacobi_pcg
from tests.oracle_pins import mms_errors


def test_pcg_matches_dense_solve():
    n = (3, 3, 2)
    V = S.structured_vertices(*n, 0.1, 21)
    mesh = fem.StructuredMesh(*n, 2, 4, V, S.structured_elem_vert(*n))
    op = fem.Operator(mesh, 1.0, 0.5)
    b = S.random_vector(mesh.n_dof, 8)
    x, its, rel, conv = jacobi_pcg(op, b, 1e-12)
    assert conv and rel <= 1e-12
    Ac = op.assembled(constrained=True)
    bc = np.where(mesh.dirichlet, 0.0, b)
    xd = np.linalg.solve(Ac, bc)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert np.linalg.norm(Ac @ x - bc) <= 2e-12 * np.linalg.norm(bc)
    # Jacobi PCG on an SPD system of size m converges in at most m steps
    assert its <= (~mesh.dirichlet).sum()


def test_pcg_zero_rhs_and_stopping_rule():
    n = (2, 2, 2)
    mesh = fem.StructuredMesh(*n, 3, 5, S.structured_vertices(*n, 0.1, 2), S.structured_elem_vert(*n))
    op = fem.Operator(mesh, 1.0, 1.0)
    x, its, rel, conv = jacobi_pcg(op, np.zeros(mesh.n_dof))
    assert conv and its == 0 and not x.any()
    b = S.random_vector(mesh.n_dof, 1)
    for tol in (1e-4, 1e-8, 1e-10):
        x, its, rel, conv = jacobi_pcg(op, b, tol)
        r = np.where(mesh.dirichlet, 0, b) - op.apply(x, constrained=True)
        assert conv and rel <= tol
        assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(np.where(mesh.dirichlet, 0, b)) + 1e-14


@pytest.mark.parametrize("p,perturb", [(2, 0.0), (2, 0.1), (3, 0.0), (3, 0.1)])
def test_mms_converges_at_order_p_plus_1(p, perturb):
    errs = mms_errors(p, [2, 4, 8], perturb)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] >= p + 1 - 0.3, (errs, rates)
