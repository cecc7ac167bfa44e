"""Degenerate and edge cases through the C ABI, vs the CPU oracle: every DoF Dirichlet, a
right-hand side living on Dirichlet DoFs only, max_it = 0, a single element of every order
(one block holding fewer elements than it can), and a single-element pure-Neumann Poisson solve
with each preconditioner."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

PRECS = ["JACOBI", "LOR", "LOR_MC", "LOR_MG"]


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


def _set(hx, op, name):
    op.set_preconditioner(getattr(hx, "HX_PREC_" + name), 1 if name == "LOR_MG" else 4)


def test_every_dof_dirichlet(hx):
    """Q1 on one element with all six faces fixed: A_c = P A P + (I - P) = I, so the constrained
    apply returns its input, P b = 0, and every solver returns x = 0 without iterating."""
    from oracle import fem
    V, EV, om = case((1, 1, 1), 1, q=3, perturb=0.1, seed=5)
    assert om.dirichlet.all()
    mesh = hx.Mesh.box(1, 1, 1, 1, 3, V, dirichlet_faces=63)
    op = hx.Operator(mesh, 2.0, 0.5)
    x = S.random_vector(8, 3)
    assert rel_err(op.apply(to_dev(x), constrained=True).cpu().numpy(), x) <= 1e-15
    assert rel_err(op.apply(to_dev(x)).cpu().numpy(), fem.Operator(om, 2.0, 0.5).apply(x)) <= 1e-12
    b = to_dev(S.random_vector(8, 4))
    for name in PRECS:
        _set(hx, op, name)
        u, info = op.solve(b, rtol=1e-10)
        assert info["status"] == 0 and info["iterations"] == 0 and not u.any(), name
    op.set_preconditioner(hx.HX_PREC_JACOBI)
    u, info = op.solve_mixed(b, rtol=1e-10)
    assert info["status"] == 0 and not u.any()


def test_rhs_on_dirichlet_dofs_only(hx):
    """b != 0 only where DoFs are fixed: P b = 0, so x = 0 at once (FP64, mixed, batched)."""
    p, shape = 2, (3, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=63)
    op = hx.Operator(mesh, 1.0, 1.0)
    b = to_dev(np.where(om.dirichlet, S.random_vector(om.n_dof, 5), 0.0))
    u, info = op.solve(b, rtol=1e-10)
    assert info["status"] == 0 and info["iterations"] == 0 and not u.any()
    u, info = op.solve_mixed(b, rtol=1e-10)
    assert info["status"] == 0 and not u.any()
    x = torch.zeros_like(b)
    infos = hx.Batch([op], [b], [x], rtol=1e-10).solve()
    assert infos[0]["status"] == 0 and not x.any()


def test_zero_iterations_allowed(hx):
    """max_it = 0 with a non-zero residual: NOT_CONVERGED after 0 iterations, x left at zero."""
    p, shape = 2, (2, 2, 2)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    u, info = op.solve(to_dev(S.random_vector(om.n_dof, 6)), rtol=1e-10, max_it=0, raise_on_fail=False)
    assert info["status"] == hx.HX_ERR_NOT_CONVERGED and info["iterations"] == 0 and not u.any()


@pytest.mark.parametrize("p", range(1, 9))
def test_single_element_every_order(hx, p):
    """One element: the operator's only block holds one element of the several it is sized for
    (FP64, and the constrained FP32 operator, whose factor copy then covers a single element)."""
    from oracle import fem
    for q in (p + 1, p + 2):
        V, EV, om = case((1, 1, 1), p, q=q, perturb=0.2, seed=60 + p)
        mesh = hx.Mesh.structured(1, 1, 1, p, q, V)
        oop = fem.Operator(om, 1.5, 0.8)
        x = S.random_vector(om.n_dof, 61)
        for gm in (hx.HX_GEOM_STORED, hx.HX_GEOM_ONTHEFLY):
            op = hx.Operator(mesh, 1.5, 0.8, geom_mode=gm)
            y = op.apply(to_dev(x)).cpu().numpy()
            assert rel_err(y, oop.apply(x)) <= 1e-12, (q, gm)
            x32 = x.astype(np.float32)       # the FP32 operator is the constrained A_c
            ref32 = oop.apply(x32.astype(np.float64), constrained=True)
            kinds = [hx.HX_F32_COLLOCATED, hx.HX_F32_DIRECT] + ([hx.HX_F32_DIRECT_STAGED] if gm == 0 else [])
            for kind in kinds:
                op.set_f32_kernel(kind)
                y32 = op.apply_f32(torch.as_tensor(x32, device="cuda")).double().cpu().numpy()
                assert rel_err(y32, ref32) <= 2e-5, (q, gm, kind)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("name", PRECS)
def test_single_element_neumann_poisson(hx, p, name):
    """Pure Neumann on one element (alpha = 0, no fixed DoF): the mean-zero solution of the
    singular system, with each preconditioner (at p = 4 the multigrid has two levels, 5 -> 3)."""
    from oracle import fem
    from oracle.solve import jacobi_pcg_nullspace
    V, EV, om = case((1, 1, 1), p, perturb=0.15, seed=70 + p, dirichlet=False)
    mesh = hx.Mesh.box(1, 1, 1, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    _set(hx, op, name)
    b = S.random_vector(om.n_dof, 71)
    u, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    uo = jacobi_pcg_nullspace(fem.Operator(om, 0.0, 1.0), b, 1e-13)[0]
    assert rel_err(u.cpu().numpy(), uo) <= 1e-8
