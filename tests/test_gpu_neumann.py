"""Pure-Neumann Poisson (the projection method's pressure step, Sec. 4.2 / Sec. 5.3) and partial
Dirichlet boundaries, through the C ABI, vs the CPU oracle."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def cos3(X):
    return np.cos(np.pi * X[..., 0]) * np.cos(np.pi * X[..., 1]) * np.cos(np.pi * X[..., 2])


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


@pytest.mark.parametrize("p,shape", [(2, (3, 3, 2)), (3, (3, 3, 3)), (5, (2, 2, 2))])
@pytest.mark.parametrize("mixed", [False, True])
def test_neumann_poisson_matches_oracle(hx, p, shape, mixed):
    from oracle import fem
    from oracle.solve import jacobi_pcg_nullspace
    V, EV, om = case(shape, p, dirichlet=False)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    b = S.random_vector(om.n_dof, 13)
    if mixed:
        x, info = op.solve_mixed(to_dev(b), rtol=1e-10)
    else:
        x, info = op.solve(to_dev(b), rtol=1e-10)
        assert info["true_rel_residual"] <= 1.01e-10
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xo, its, rel, conv = jacobi_pcg_nullspace(fem.Operator(om, 0.0, 1.0), b, 1e-12)
    xs = x.cpu().numpy()
    assert rel_err(xs, xo) <= 1e-8
    m1 = fem.Operator(om, 1.0, 0.0).apply(np.ones(om.n_dof))
    assert abs(m1 @ xs) <= 1e-12 * np.abs(xs).max()


def test_neumann_manufactured_solution(hx):
    from oracle import fem
    p, shape = 4, (4, 4, 4)
    V, EV, om = case(shape, p, dirichlet=False)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    b = op.load_vector(to_dev(3 * np.pi ** 2 * cos3(mesh.qpoint_coords().cpu().numpy())))
    x, info = op.solve(b, rtol=1e-10)
    assert fem.l2_error(om, x.cpu().numpy(), cos3) < 5e-4


@pytest.mark.parametrize("faces", [3, 16 | 32, 1])
def test_partial_dirichlet_faces(hx, faces):
    from oracle import fem
    p, shape = 3, (3, 2, 2)
    V, EV, om = case(shape, p, dirichlet=False)
    gx, gy, gz = p * shape[0] + 1, p * shape[1] + 1, p * shape[2] + 1
    K, J, I = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    sel = [(1, I == 0), (2, I == gx - 1), (4, J == 0), (8, J == gy - 1), (16, K == 0), (32, K == gz - 1)]
    om.dirichlet = np.zeros(om.n_dof, bool)
    for bit, m in sel:
        if faces & bit:
            om.dirichlet |= m
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=faces)
    op = hx.Operator(mesh, 0.0, 1.0)
    oop = fem.Operator(om, 0.0, 1.0)
    xv = S.random_vector(om.n_dof, 3)
    y = op.apply(to_dev(xv), constrained=True).cpu().numpy()
    np.testing.assert_allclose(y, oop.apply(xv, constrained=True), rtol=0, atol=1e-12 * np.abs(y).max())
    b = S.random_vector(om.n_dof, 4)
    x, info = op.solve(to_dev(b), rtol=1e-12)
    xd = np.linalg.solve(oop.assembled(constrained=True), np.where(om.dirichlet, 0.0, b))
    assert rel_err(x.cpu().numpy(), xd) <= 1e-9
