"""Preconditioners of the PCG solves through the C ABI, vs the CPU oracle: the collocated
Gauss-Lobatto mass (Sec. 5.1)."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


@pytest.mark.parametrize("p", range(1, 9))
def test_collocated_mass_matches_oracle(hx, p):
    from oracle import precond
    shape = (3, 2, 2) if p <= 5 else (2, 2, 1)
    V, EV, om = case(shape, p, perturb=0.15, seed=300 + p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 3.5, 0.1)
    d = op.collocated_mass().cpu().numpy()
    assert rel_err(d, precond.collocated_mass_diagonal(om, 3.5)) <= 1e-13


def test_precond_apply_is_the_inverse_diagonal(hx):
    from oracle import fem, precond
    p, shape = 4, (3, 3, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 2.0, 0.3)
    r = S.uniform_pm1(17, om.n_dof)
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    dj = fem.Operator(om, 2.0, 0.3).diagonal()
    assert rel_err(z, np.where(om.dirichlet, r, r / dj)) <= 1e-13
    op.set_preconditioner(hx.HX_PREC_COLLOCATED_MASS)
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    dm = precond.collocated_mass_diagonal(om, 2.0)
    assert rel_err(z, np.where(om.dirichlet, r, r / dm)) <= 1e-13
    op.set_preconditioner(hx.HX_PREC_JACOBI)
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    assert rel_err(z, np.where(om.dirichlet, r, r / dj)) <= 1e-13


def _mass_solve(hx, shape, p, prec):
    V = S.structured_vertices(*shape, 0.1, 1910)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1.0, 0.0)
    op.set_preconditioner(prec)
    b = to_dev(S.uniform_pm1(23, mesh.n_dof))
    x, info = op.solve(b, rtol=1e-10)
    assert info["status"] == 0 and info["true_rel_residual"] <= 1.01e-10
    return x, info["iterations"]


def test_collocated_mass_iterations_bounded_in_h_and_p(hx):
    """Mass solves: the collocated mass keeps CG iterations bounded as h and p change (Sec. 5.1).
    On affine elements the preconditioned spectrum lies in [(p / (2p + 1))^3, 1], so
    kappa <= 27 and CG needs at most about sqrt(27) / 2 ln(2 / 1e-10) ~ 62 iterations."""
    its = {}
    for p in (2, 4, 8):
        for N in (4, 8, 16):
            if p == 8 and N == 16:
                continue
            x_m, its[(p, N)] = _mass_solve(hx, (N, N, N), p, hx.HX_PREC_COLLOCATED_MASS)
            x_j, _ = _mass_solve(hx, (N, N, N), p, hx.HX_PREC_JACOBI)
            assert rel_err(x_m.cpu().numpy(), x_j.cpu().numpy()) <= 1e-8
    assert max(its.values()) <= 70, its


@pytest.mark.parametrize("mixed", [False, True])
def test_helmholtz_with_collocated_mass_matches_oracle(hx, mixed):
    """A mass-dominated Helmholtz solve (alpha = 1000, nu = 1e-2) preconditioned by alpha Mc."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    p, shape = 3, (4, 4, 4)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1000.0, 1e-2)
    op.set_preconditioner(hx.HX_PREC_COLLOCATED_MASS)
    b = S.random_vector(om.n_dof, 29)
    if mixed:
        x, info = op.solve_mixed(to_dev(b), rtol=1e-10)
    else:
        x, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["true_rel_residual"] <= 1.01e-10
    xo, _, _, _ = jacobi_pcg(fem.Operator(om, 1000.0, 1e-2), b, 1e-12)
    assert rel_err(x.cpu().numpy(), xo) <= 1e-8


def test_collocated_mass_needs_positive_alpha(hx):
    p, shape = 2, (2, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 0.0, 1.0)
    with pytest.raises(hx.HxError) as ei:
        op.set_preconditioner(hx.HX_PREC_COLLOCATED_MASS)
    assert ei.value.status == -1
    with pytest.raises(hx.HxError):
        op.set_preconditioner(7)
    op.set_coefficients(1.0, 1.0)
    op.set_preconditioner(hx.HX_PREC_COLLOCATED_MASS)
    op.solve(to_dev(S.uniform_pm1(3, om.n_dof)))
    with pytest.raises(hx.HxError):
        op.set_coefficients(0.0, 1.0)
