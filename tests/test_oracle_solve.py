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


def _neumann_mesh(N, p, perturb=0.1, seed=5):
    V = S.structured_vertices(N, N, N, perturb, seed)
    return fem.StructuredMesh(N, N, N, p, p + 2, V, S.structured_elem_vert(N, N, N), dirichlet_boundary=False)


def test_neumann_poisson_matches_pseudoinverse():
    """Pure Neumann: the orthogonalized PCG gives the minimum-norm solution shifted to int x = 0."""
    from oracle.solve import jacobi_pcg_nullspace
    mesh = _neumann_mesh(2, 2)
    op = fem.Operator(mesh, 0.0, 1.0)
    b = S.random_vector(mesh.n_dof, 31)
    x, its, rel, conv = jacobi_pcg_nullspace(op, b, 1e-12)
    assert conv
    K = op.assembled()
    bp = b - b.mean()
    xd = np.linalg.pinv(K) @ bp
    m1 = fem.Operator(mesh, 1.0, 0.0).apply(np.ones(mesh.n_dof))
    xd -= (m1 @ xd) / m1.sum()
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert abs(m1 @ x) <= 1e-12 * np.abs(m1).sum() * np.abs(x).max()
    assert np.linalg.norm(K @ x - bp) <= 1e-10 * np.linalg.norm(bp)


@pytest.mark.parametrize("p", [2, 3])
def test_neumann_mms_converges_at_order_p_plus_1(p):
    """u = cos(pi x) cos(pi y) cos(pi z): zero normal derivative on the cube and zero mean."""
    from oracle.solve import jacobi_pcg_nullspace
    uex = lambda X: np.cos(np.pi * X[..., 0]) * np.cos(np.pi * X[..., 1]) * np.cos(np.pi * X[..., 2])
    errs = []
    for N in (2, 4, 8):
        mesh = _neumann_mesh(N, p, 0.1, 1910)
        op = fem.Operator(mesh, 0.0, 1.0)
        b = fem.load_vector(mesh, 3 * np.pi ** 2 * uex(mesh.qpoint_coords()))
        x, its, rel, conv = jacobi_pcg_nullspace(op, b, 1e-12, 5000)
        assert conv
        errs.append(fem.l2_error(mesh, x, uex))
    errs = np.array(errs)
    assert np.log2(errs[-2] / errs[-1]) >= p + 1 - 0.3, errs
