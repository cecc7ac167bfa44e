"""Full-size meshes of the FP64 scaling sweep (the launch configuration the benchmark times):
sampled entries vs the oracle computed row by row, plus a size-independent property."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, lor_row_oracle, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

SWEEP = [(2, 160), (4, 96), (8, 48)]


@pytest.mark.parametrize("p,N", SWEEP)
def test_fullsize_apply_sampled(p, N):
    hx = require_gpu()
    from oracle import fem
    V, EV, om = case((N, N, N), p, lazy=True)
    mesh = hx.Mesh.structured(N, N, N, p, p + 2, V)
    alpha, nu = 1000.0, 1e-2
    op = hx.Operator(mesh, alpha, nu)
    assert mesh.n_dof == (p * N + 1) ** 3
    x = S.random_vector(mesh.n_dof, 3032)
    y = op.apply(to_dev(x), constrained=True).cpu().numpy()
    oop = fem.Operator(om, alpha, nu, cache=False)
    g = np.unique(np.concatenate([S.permutation(mesh.n_dof, 7)[:40], [0, mesh.n_dof - 1, mesh.n_dof // 2]]))
    ref = oop.apply_rows(x, g, constrained=True)
    np.testing.assert_allclose(y[g], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    del op
    # size-independent property: 1^T M 1 = volume of the unit cube
    opm = hx.Operator(mesh, 1.0, 0.0)
    one = torch.ones(mesh.n_dof, dtype=torch.float64, device="cuda")
    assert abs(float(opm.apply(one).sum()) - 1.0) < 1e-11


@pytest.mark.parametrize("p,N", [(4, 96)])
def test_fullsize_fp32_apply_sampled(p, N):
    """The FP32 operator of the mixed-precision solver at the benchmark's size (factors staged by
    the bulk copy): sampled rows within the FP32 rounding of the FP64 rows (a few q^3 terms of
    relative size 2^-24 each)."""
    hx = require_gpu()
    from oracle import fem
    V, EV, om = case((N, N, N), p, lazy=True)
    mesh = hx.Mesh.structured(N, N, N, p, p + 2, V)
    op = hx.Operator(mesh, 1000.0, 1e-2)
    x = S.random_vector(mesh.n_dof, 3033)
    y = op.apply_f32(to_dev(x).float()).double().cpu().numpy()
    oop = fem.Operator(om, 1000.0, 1e-2, cache=False)
    g = np.unique(np.concatenate([S.permutation(mesh.n_dof, 8)[:40], [0, mesh.n_dof - 1, mesh.n_dof // 2]]))
    ref = oop.apply_rows(x, g, constrained=True)
    np.testing.assert_allclose(y[g], ref, rtol=0, atol=2e-5 * np.abs(ref).max())


# the two solves of the preconditioner benchmark: the projection step's pure-Neumann pressure
# Poisson (64^3, p = 5) and the Helmholtz problem of the headline (96^3, p = 4)
PRECOND_CASES = [(5, 64, 0.0, 1.0, False), (4, 96, 1000.0, 1e-2, True)]


@pytest.mark.parametrize("p,N,alpha,nu,dirichlet", PRECOND_CASES)
def test_fullsize_lor_sampled_rows_and_symmetry(p, N, alpha, nu, dirichlet):
    """HX_PREC_LOR_MC at the benchmark's sizes: sampled rows of the assembled alpha Mc + nu K_LOR
    vs the oracle (each row from its patch of elements), and two properties of the Chebyshev
    apply that hold at any size: P = p(D^-1 A) D^-1 is linear and symmetric (u.P v = v.P u),
    which a misplaced column of its sliced-ELL copy would break.

    Row tolerance 1e-12 of the row's largest entry: the oracle forms each sub-element's Jacobian
    from differences of mapped node coordinates, sub-elements 1/(pN) ~ 3e-3 wide in a unit cube,
    so each difference carries a relative error of about eps pN ~ 4e-14 (the library evaluates
    the element map at the sub-element's points instead); J^-1 and detJ amplify that a few
    times (observed 1.5e-13 on a corner row at 64^3, p = 5)."""
    hx = require_gpu()
    V, EV, om = case((N, N, N), p, lazy=True, dirichlet=dirichlet)
    mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    op = hx.Operator(mesh, alpha, nu)
    op.set_preconditioner(hx.HX_PREC_LOR_MC, 16)
    n = mesh.n_dof
    ro, col, val = op.lor_csr()
    ro_h = ro.cpu().numpy()
    g_all = np.unique(np.concatenate([S.permutation(n, 9)[:30], [0, n - 1, n // 2, (p * N + 1) ** 2 + 1]]))
    for g in g_all:
        a, b = int(ro_h[g]), int(ro_h[g + 1])
        cols, vals = col[a:b].cpu().numpy().astype(np.int64), val[a:b].cpu().numpy()
        oc, ov = lor_row_oracle(om, g, alpha, nu)
        union = np.union1d(cols, oc)
        mine, ref = np.zeros(len(union)), np.zeros(len(union))
        mine[np.searchsorted(union, cols)] = vals
        ref[np.searchsorted(union, oc)] = ov
        np.testing.assert_allclose(mine, ref, rtol=0, atol=1e-12 * np.abs(ref).max(), err_msg=f"row {g}")
    del ro, col, val
    u = to_dev(S.uniform_pm1(91, n))
    v = to_dev(S.uniform_pm1(92, n))
    Pu, Pv = op.precond_apply(u), op.precond_apply(v)
    lhs, rhs = float(torch.dot(u, Pv)), float(torch.dot(v, Pu))
    assert abs(lhs - rhs) <= 1e-11 * float(u.norm() * Pv.norm()), (lhs, rhs)
    Pw = op.precond_apply(2.0 * u - 3.0 * v)
    assert float((Pw - (2.0 * Pu - 3.0 * Pv)).norm()) <= 1e-12 * float(Pw.norm())
