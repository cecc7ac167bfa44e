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


# ---------------------------------------------------------------------------
# low-order refined preconditioner (Sec. 5.2)
# ---------------------------------------------------------------------------
def _dense(row_off, col, val, n):
    ro, c, v = row_off.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(ro))
    A[rows, c] = v
    for g in range(n):
        assert np.all(np.diff(c[ro[g]:ro[g + 1]]) > 0)    # sorted, distinct
    return A


@pytest.mark.parametrize("p,dirichlet", [(1, True), (2, True), (3, True), (3, False), (5, True), (8, True)])
def test_lor_matrix_matches_oracle(hx, p, dirichlet):
    from oracle import precond
    shape = (3, 2, 2) if p <= 3 else (2, 2, 1)
    V, EV, om = case(shape, p, perturb=0.15, seed=400 + p, dirichlet=dirichlet)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    op = hx.Operator(mesh, 2.5, 0.7)
    A = _dense(*op.lor_csr(), om.n_dof)
    Ao = precond.lor_operator(om, 2.5, 0.7).assembled(constrained=True)
    assert np.abs(A - Ao).max() <= 1e-13 * np.abs(Ao).max()
    # pattern: exactly the structural non-zeros of the oracle matrix (27 per interior row)
    assert np.array_equal(A != 0, Ao != 0) or np.all(np.abs(Ao[(A != 0) != (Ao != 0)]) <= 1e-14 * np.abs(Ao).max())


@pytest.mark.parametrize("p", [2, 3])
def test_lor_on_unstructured_mesh(hx, p):
    """Valence-5 central edge: LOR rows of 33 entries (sliced-ELL slices wider than 27 and a
    partial load batch) vs the oracle: the matrix, the Chebyshev apply of both mass forms, and
    the LOR-PCG solution."""
    from oracle import fem, precond
    from oracle.solve import jacobi_pcg
    from tests.unstructured import star_prism
    V, EV, om = star_prism(p)
    mesh = hx.Mesh.general(p, p + 2, V, EV, om.n_dof, om.restriction.astype(np.int32),
                           om.dirichlet.astype(np.uint8))
    op = hx.Operator(mesh, 2.0, 0.7)
    op.set_preconditioner(hx.HX_PREC_LOR, 5)
    ro, col, val = op.lor_csr()
    assert int(np.diff(ro.cpu().numpy()).max()) == 33
    A = _dense(ro, col, val, om.n_dof)
    Ao = precond.lor_operator(om, 2.0, 0.7).assembled(constrained=True)
    assert np.abs(A - Ao).max() <= 1e-13 * np.abs(Ao).max()
    r = np.where(om.dirichlet, 0.0, S.uniform_pm1(71, om.n_dof))
    assert rel_err(op.precond_apply(to_dev(r)).cpu().numpy(), precond.chebyshev_apply(Ao, r, 5)) <= 1e-12
    op.set_preconditioner(hx.HX_PREC_LOR_MC, 7)
    Amc = precond.lor_matrix(om, 2.0, 0.7, "collocated")
    assert rel_err(op.precond_apply(to_dev(r)).cpu().numpy(), precond.chebyshev_apply(Amc, r, 7)) <= 1e-12
    b = S.random_vector(om.n_dof, 72)
    x, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["true_rel_residual"] <= 1.01e-10
    assert rel_err(x.cpu().numpy(), jacobi_pcg(fem.Operator(om, 2.0, 0.7), b, 1e-12)[0]) <= 1e-8


def test_lor_matrix_follows_coefficients(hx):
    from oracle import precond
    p, shape = 3, (2, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1.0, 1.0)
    op.set_preconditioner(hx.HX_PREC_LOR, 4)
    op.set_coefficients(30.0, 0.2)
    A = _dense(*op.lor_csr(), om.n_dof)
    Ao = precond.lor_operator(om, 30.0, 0.2).assembled(constrained=True)
    assert np.abs(A - Ao).max() <= 1e-13 * np.abs(Ao).max()


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_lor_precond_apply_matches_oracle(hx, k):
    from oracle import precond
    p, shape = 4, (3, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 10.0, 0.5)
    op.set_preconditioner(hx.HX_PREC_LOR, k)
    r = np.where(om.dirichlet, 0.0, S.uniform_pm1(31, om.n_dof))
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    zo = precond.chebyshev_apply(precond.lor_operator(om, 10.0, 0.5).assembled(constrained=True), r, k)
    assert rel_err(z, zo) <= 1e-12


@pytest.mark.parametrize("p", [2, 3, 5])
def test_lor_mc_matrix_matches_oracle(hx, p):
    from oracle import precond
    shape = (3, 2, 2)
    V, EV, om = case(shape, p, perturb=0.15, seed=450 + p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 40.0, 0.3)
    op.set_preconditioner(hx.HX_PREC_LOR_MC, 3)
    A = _dense(*op.lor_csr(), om.n_dof)
    Ao = precond.lor_matrix(om, 40.0, 0.3, "collocated")
    assert np.abs(A - Ao).max() <= 1e-13 * np.abs(Ao).max()
    r = np.where(om.dirichlet, 0.0, S.uniform_pm1(33, om.n_dof))
    assert rel_err(op.precond_apply(to_dev(r)).cpu().numpy(), precond.chebyshev_apply(Ao, r, 3)) <= 1e-12


@pytest.mark.parametrize("kind,alpha", [("LOR", 0.0), ("LOR_MC", 0.0), ("LOR_MC", 1000.0), ("LOR", 1000.0)])
def test_lor_pcg_matches_oracle(hx, kind, alpha):
    """Iterations: the LOR forms need well under half of Jacobi's on Poisson; with alpha = 1000 the
    collocated-mass form stays at Jacobi's count, while the Q1-mass form needs more (its mass
    is a poor match of M), which is why HX_PREC_LOR_MC exists."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    p, shape = 4, (4, 4, 4)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    nu = 1.0 if alpha == 0.0 else 1e-2
    op = hx.Operator(mesh, alpha, nu)
    b = S.random_vector(om.n_dof, 37)
    x_j, info_j = op.solve(to_dev(b), rtol=1e-10)
    op.set_preconditioner(getattr(hx, "HX_PREC_" + kind), 8)
    x_l, info_l = op.solve(to_dev(b), rtol=1e-10)
    assert info_l["status"] == 0 and info_l["true_rel_residual"] <= 1.01e-10
    xo, _, _, _ = jacobi_pcg(fem.Operator(om, alpha, nu), b, 1e-12)
    assert rel_err(x_l.cpu().numpy(), xo) <= 1e-8
    if alpha == 0.0:
        assert 2 * info_l["iterations"] < info_j["iterations"]
    elif kind == "LOR_MC":
        assert info_l["iterations"] <= info_j["iterations"] + 3


def test_lor_neumann_poisson(hx):
    from oracle import fem
    from oracle.solve import jacobi_pcg_nullspace
    p, shape = 3, (3, 3, 3)
    V, EV, om = case(shape, p, dirichlet=False)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    op.set_preconditioner(hx.HX_PREC_LOR, 6)
    b = S.random_vector(om.n_dof, 41)
    x, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    xo, _, _, _ = jacobi_pcg_nullspace(fem.Operator(om, 0.0, 1.0), b, 1e-12)
    assert rel_err(x.cpu().numpy(), xo) <= 1e-8
    m1 = fem.Operator(om, 1.0, 0.0).apply(np.ones(om.n_dof))
    xs = x.cpu().numpy()
    assert abs(m1 @ xs) <= 1e-12 * np.abs(xs).max()


def test_lor_in_a_batch(hx):
    from oracle import fem
    from oracle.solve import jacobi_pcg
    ops, bs, xs, refs = [], [], [], []
    cases = [(4, 3, hx.HX_PREC_LOR), (3, 5, hx.HX_PREC_JACOBI), (5, 2, hx.HX_PREC_LOR)]
    for k, (N, p, prec) in enumerate(cases):
        V = S.structured_vertices(N, N, N, 0.1, 500 + k)
        mesh = hx.Mesh.structured(N, N, N, p, p + 2, V)
        op = hx.Operator(mesh, 0.0, 1.0)
        op.set_preconditioner(prec, 6)
        b = to_dev(S.uniform_pm1(600 + k, mesh.n_dof))
        refs.append(op.solve(b, rtol=1e-10))
        ops.append(op)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    batch = hx.Batch(ops, bs, xs, rtol=1e-10)
    infos = batch.solve()
    for k, ((xr, ir), x, i, b) in enumerate(zip(refs, xs, infos, bs)):
        assert i["status"] == 0 and i["iterations"] == ir["iterations"]
        assert torch.equal(x, xr)
        # the preconditioner changes the iterates, not the solution: the oracle's Jacobi-PCG
        # solution of the same Poisson problem (to 1e-12) within the solution tolerance
        N, p, _ = cases[k]
        _, _, om = case((N, N, N), p, seed=500 + k)
        xo, _, _, conv = jacobi_pcg(fem.Operator(om, 0.0, 1.0), b.cpu().numpy(), 1e-12, 20000)
        assert conv and rel_err(x.cpu().numpy(), xo) <= 1e-8


def test_lor_errors(hx):
    p, shape = 2, (2, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    E, Q = om.n_elem, (p + 2) ** 3
    op = hx.Operator(mesh, 1.0, 0.0, to_dev(np.full((E, Q), 0.3)))
    with pytest.raises(hx.HxError) as ei:
        op.set_preconditioner(hx.HX_PREC_LOR, 4)
    assert ei.value.status == -7
    op2 = hx.Operator(mesh, 1.0, 1.0)
    for bad in (0, 65):
        with pytest.raises(hx.HxError) as ei:
            op2.set_preconditioner(hx.HX_PREC_LOR, bad)
        assert ei.value.status == -1
    op2.set_preconditioner(hx.HX_PREC_LOR, 4)
    with pytest.raises(hx.HxError) as ei:
        op2.solve_mixed(to_dev(S.uniform_pm1(3, om.n_dof)))
    assert ei.value.status == -7
    with pytest.raises(hx.HxError) as ei:
        op2.set_coefficients(1.0, 1.0, to_dev(np.full((E, Q), 0.3)))
    assert ei.value.status == -7


# ---------------------------------------------------------------------------
# geometric multigrid V-cycle on the LOR matrix (Sec. 5.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,p,dirichlet,alpha,deg", [(4, 2, True, 0.0, 3), (2, 4, True, 5.0, 2), (4, 2, False, 0.0, 3),
                                                     (3, 3, True, 1.0, 3), (4, 4, True, 100.0, 4), (4, 2, True, 0.0, 1),
                                                     (4, 4, False, 0.0, 1), (2, 4, True, 5.0, 1)])
def test_mg_vcycle_matches_oracle(hx, N, p, dirichlet, alpha, deg):
    from oracle import precond
    shape = (N, N, N)
    V, EV, om = case(shape, p, seed=700 + N + p, dirichlet=dirichlet)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    op = hx.Operator(mesh, alpha, 1.0)
    op.set_preconditioner(hx.HX_PREC_LOR_MG, deg)
    A = precond.lor_matrix(om, alpha, 1.0, "collocated")
    levels = precond.mg_hierarchy(A, (p * N + 1,) * 3, om.dirichlet)
    r = np.where(om.dirichlet, 0.0, S.uniform_pm1(800 + N, om.n_dof))
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    zo = precond.vcycle(levels, r, smooth_degree=deg)
    assert rel_err(z, zo) <= 1e-11, (len(levels), rel_err(z, zo))


@pytest.mark.parametrize("alpha,dirichlet", [(0.0, True), (1000.0, True), (0.0, False)])
def test_mg_pcg_matches_oracle(hx, alpha, dirichlet):
    from oracle import fem
    from oracle.solve import jacobi_pcg, jacobi_pcg_nullspace
    p, shape = 4, (4, 4, 4)
    V, EV, om = case(shape, p, dirichlet=dirichlet)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    nu = 1.0 if alpha == 0.0 else 1e-2
    op = hx.Operator(mesh, alpha, nu)
    b = S.random_vector(om.n_dof, 43)
    x_j, info_j = op.solve(to_dev(b), rtol=1e-10)
    op.set_preconditioner(hx.HX_PREC_LOR_MG, 3)
    x, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    oop = fem.Operator(om, alpha, nu)
    xo = (jacobi_pcg(oop, b, 1e-12) if dirichlet else jacobi_pcg_nullspace(oop, b, 1e-12))[0]
    assert rel_err(x.cpu().numpy(), xo) <= 1e-8
    if alpha == 0.0:
        assert 2 * info["iterations"] < info_j["iterations"], (info["iterations"], info_j["iterations"])
    else:
        assert info["iterations"] <= info_j["iterations"] + 3


def test_mg_iterations_flat_under_refinement(hx):
    its = []
    for N in (4, 8, 16):
        V = S.structured_vertices(N, N, N, 0.1, 900 + N)
        mesh = hx.Mesh.structured(N, N, N, 4, 6, V)
        op = hx.Operator(mesh, 0.0, 1.0)
        op.set_preconditioner(hx.HX_PREC_LOR_MG, 3)
        x, info = op.solve(to_dev(S.uniform_pm1(901, mesh.n_dof)), rtol=1e-10)
        assert info["status"] == 0
        its.append(info["iterations"])
    assert its[-1] <= its[0] + 10, its


def test_mg_needs_a_structured_mesh(hx):
    from oracle import fem
    p, shape = 2, (2, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.general(p, p + 2, V, EV.astype(np.int64), om.n_dof, om.restriction.astype(np.int32),
                           om.dirichlet.astype(np.uint8))
    op = hx.Operator(mesh, 1.0, 1.0)
    with pytest.raises(hx.HxError) as ei:
        op.set_preconditioner(hx.HX_PREC_LOR_MG, 3)
    assert ei.value.status == -7


@pytest.mark.parametrize("alpha,dirichlet", [(0.0, True), (0.0, False), (1000.0, True)])
def test_mixed_solve_with_multigrid(hx, alpha, dirichlet):
    """Mixed precision with the LOR multigrid: the FP32 inner CG is preconditioned by the V-cycle
    in FP32; the FP64 refinement still reaches 1e-10 and the oracle's solution."""
    from oracle import fem
    from oracle.solve import jacobi_pcg, jacobi_pcg_nullspace
    p, shape = 4, (4, 4, 4)
    V, EV, om = case(shape, p, dirichlet=dirichlet)
    mesh = hx.Mesh.box(*shape, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    nu = 1.0 if alpha == 0.0 else 1e-2
    op = hx.Operator(mesh, alpha, nu)
    op.set_preconditioner(hx.HX_PREC_LOR_MG, 2)
    b = S.random_vector(om.n_dof, 47)
    x64, info64 = op.solve(to_dev(b), rtol=1e-10)
    x, info = op.solve_mixed(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    assert info["refinements"] <= 4
    oop = fem.Operator(om, alpha, nu)
    xo = (jacobi_pcg(oop, b, 1e-12) if dirichlet else jacobi_pcg_nullspace(oop, b, 1e-12))[0]
    assert rel_err(x.cpu().numpy(), xo) <= 1e-8
    # the inner solves need about as many iterations per refinement as the FP64 solve in all
    assert info["iterations"] <= info["refinements"] * (info64["iterations"] + 5)


def _face_mask(shape, p, faces):
    gx, gy, gz = p * shape[0] + 1, p * shape[1] + 1, p * shape[2] + 1
    K, J, I = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    sel = [(1, I == 0), (2, I == gx - 1), (4, J == 0), (8, J == gy - 1), (16, K == 0), (32, K == gz - 1)]
    mask = np.zeros(gx * gy * gz, bool)
    for bit, m in sel:
        if faces & bit:
            mask |= m
    return mask


@pytest.mark.parametrize("shape,p,q,faces", [((4, 4, 2), 1, 2, 63), ((2, 2, 2), 3, 4, 3), ((4, 2, 2), 2, 4, 16 | 32),
                                             ((1, 1, 1), 8, 9, 63), ((2, 2, 2), 4, 6, 1)])
def test_mg_vcycle_more_cases(hx, shape, p, q, faces):
    """Q_1 meshes (the LOR mesh is the mesh), q = p + 1, partial Dirichlet faces, one element of Q_8."""
    from oracle import fem, precond
    V = S.structured_vertices(*shape, 0.1, 990 + p)
    om = fem.StructuredMesh(*shape, p, q, V, S.structured_elem_vert(*shape), dirichlet_boundary=False)
    om.dirichlet = _face_mask(shape, p, faces)
    mesh = hx.Mesh.box(*shape, p, q, V, dirichlet_faces=faces)
    op = hx.Operator(mesh, 3.0, 0.4)
    op.set_preconditioner(hx.HX_PREC_LOR_MG, 3)
    A = precond.lor_matrix(om, 3.0, 0.4, "collocated")
    levels = precond.mg_hierarchy(A, tuple(p * s + 1 for s in shape), om.dirichlet)
    r = np.where(om.dirichlet, 0.0, S.uniform_pm1(991, om.n_dof))
    z = op.precond_apply(to_dev(r)).cpu().numpy()
    assert rel_err(z, precond.vcycle(levels, r, smooth_degree=3)) <= 1e-11


@pytest.mark.parametrize("kind,dirichlet", [("LOR_MG", False), ("LOR_MG", True), ("LOR_MC", True)])
def test_preconditioner_symmetric_positive_at_size(hx, kind, dirichlet):
    """At 32^3, p = 5 (4.2 M DoFs): the preconditioner is a symmetric positive operator on the
    constrained space, (B x).y = x.(B y) and (B x).x > 0, as CG requires (a property that holds at
    any size; the oracle checks the same cycle element by element on small grids)."""
    N, p = 32, 5
    V = S.structured_vertices(N, N, N, 0.1, 1910)
    mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=63 if dirichlet else 0)
    op = hx.Operator(mesh, 0.0 if not dirichlet else 10.0, 1.0)
    op.set_preconditioner(getattr(hx, "HX_PREC_" + kind), 2 if kind == "LOR_MG" else 8)
    dmask = torch.zeros(mesh.n_dof, dtype=torch.bool, device="cuda")
    if dirichlet:
        xyz = mesh.node_coords()
        dmask = ((xyz <= 1e-14) | (xyz >= 1 - 1e-14)).any(dim=1)
    x = to_dev(S.uniform_pm1(71, mesh.n_dof)).masked_fill(dmask, 0.0)
    y = to_dev(S.uniform_pm1(72, mesh.n_dof)).masked_fill(dmask, 0.0)
    bx, by = op.precond_apply(x), op.precond_apply(y)
    lhs, rhs = torch.dot(bx, y).item(), torch.dot(x, by).item()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + torch.norm(bx).item() * torch.norm(y).item())
    assert torch.dot(bx, x).item() > 0
