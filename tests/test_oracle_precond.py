"""Oracle preconditioners (collocated mass, Sec. 5.1; low-order refined operator, Sec. 5.2) pinned by
closed forms and published spectral bounds."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import synthetic as S
from oracle import fem, precond
from oracle.basis import gll_nodes


def one_element(p, A=None):
    V = S.structured_vertices(1, 1, 1, 0.0, 1)
    if A is not None:
        V = S.affine_map(V, np.asarray(A, dtype=float), np.array([0.3, -0.2, 0.1]))
    return fem.StructuredMesh(1, 1, 1, p, p + 2, V, S.structured_elem_vert(1, 1, 1), dirichlet_boundary=False)


SHEAR = [[1.5, 0.3, 0.0], [0.0, 0.8, 0.2], [0.1, 0.0, 1.2]]


def test_gll_weights_closed_forms():
    assert np.allclose(precond.gll_weights(1), [1, 1], rtol=0, atol=1e-15)
    assert np.allclose(precond.gll_weights(2), [1 / 3, 4 / 3, 1 / 3], rtol=0, atol=1e-15)
    assert np.allclose(precond.gll_weights(3), [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=0, atol=1e-15)
    assert np.allclose(precond.gll_weights(4), [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_rule_exact_to_degree_2p_minus_1(p):
    x, w = gll_nodes(p), precond.gll_weights(p)
    for k in range(2 * p):
        exact = float(Fraction(2, k + 1)) if k % 2 == 0 else 0.0
        assert abs(w @ x ** k - exact) <= 1e-14
    # and not beyond: x^(2p) is integrated with an error
    assert abs(w @ x ** (2 * p) - 2.0 / (2 * p + 1)) > 1e-7


@pytest.mark.parametrize("p", [2, 3, 5])
def test_collocated_mass_sums_to_volume(p):
    """detJ of a trilinear map has degree <= 2 per variable; GLL with p >= 2 integrates it exactly."""
    shape = (3, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 7)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    d = precond.collocated_mass_diagonal(mesh, 2.5)
    assert abs(d.sum() - 2.5) <= 1e-13
    assert np.all(d > 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("A", [None, SHEAR])
def test_collocated_mass_spectral_bounds(p, A):
    """On an affine element M and Mc are tensor products of the 1D forms scaled by the constant detJ,
    and the 1D pencil has eigenvalues in [p / (2p + 1), 1], both attained (the mode P_p gives the
    lower end): so the 3D spectrum of Mc^-1 M spans [(p / (2p + 1))^3, 1]."""
    mesh = one_element(p, A)
    M = fem.Operator(mesh, 1.0, 0.0).assembled()
    d = precond.collocated_mass_diagonal(mesh)
    ev = sl.eigh(M, np.diag(d), eigvals_only=True)
    lo = (p / (2 * p + 1)) ** 3
    assert abs(ev.min() - lo) <= 1e-12 and abs(ev.max() - 1.0) <= 1e-12


def test_lor_of_p1_is_the_mesh_itself():
    """For p = 1 the refined mesh is the original mesh: A_LOR = the q = 2 operator of Q_1."""
    shape = (3, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 8)
    m1 = fem.StructuredMesh(*shape, 1, 2, V, S.structured_elem_vert(*shape))
    A = fem.Operator(m1, 2.0, 0.7).assembled()
    AL = precond.lor_operator(m1, 2.0, 0.7).assembled()
    assert np.abs(A - AL).max() <= 1e-15 * np.abs(A).max()


@pytest.mark.parametrize("p", [2, 4, 7])
def test_lor_volume_and_null_space(p):
    shape = (2, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 9)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    one = np.ones(mesh.n_dof)
    ML = precond.lor_operator(mesh, 1.0, 0.0)
    KL = precond.lor_operator(mesh, 0.0, 1.0)
    assert abs(one @ ML.apply(one) - 1.0) <= 1e-13
    assert np.abs(KL.apply(one)).max() <= 1e-13 * np.abs(KL.assembled()).max()
    # every sub-element is positively oriented: the LOR mass diagonal is positive
    assert np.all(ML.diagonal() > 0)


@pytest.mark.parametrize("p", range(2, 9))
def test_lor_stiffness_equivalence_1d(p):
    """On one box element, functions of x alone (zero at the x = const faces) reduce both stiffness
    forms to 1D times the same constant: K_LOR <= K (the piecewise-linear interpolant has the mean
    slope on every sub-interval) and K <= (pi^2 / 4) K_LOR (the FEM-SEM equivalence on Gauss-Lobatto
    points); for p = 2 the single interior mode gives exactly 4/3."""
    mesh = one_element(p, np.diag([2.0, 0.7, 1.3]))
    n = p + 1
    K = fem.Operator(mesh, 0.0, 1.0).assembled()
    KL = precond.lor_operator(mesh, 0.0, 1.0).assembled()
    V = np.zeros((n ** 3, n - 2))
    for i in range(1, n - 1):
        for k in range(n):
            for j in range(n):
                V[i + n * j + n * n * k, i - 1] = 1.0
    ev = sl.eigh(V.T @ K @ V, V.T @ KL @ V, eigvals_only=True)
    assert ev.min() >= 1.0 - 1e-12 and ev.max() <= np.pi ** 2 / 4
    if p == 2:
        assert abs(ev[0] - 4.0 / 3.0) <= 1e-12


def test_lor_condition_bounded_in_p():
    """kappa(A_LOR^-1 A) stays bounded as p grows while kappa(diag(A)^-1 A) grows (Sec. 5.2)."""
    shape = (2, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 10)
    kl, kj = [], []
    for p in (2, 4, 6):
        mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
        A = fem.Operator(mesh, 1.0, 1.0).assembled(constrained=True)
        AL = precond.lor_operator(mesh, 1.0, 1.0).assembled(constrained=True)
        ev = sl.eigh(A, AL, eigvals_only=True)
        kl.append(ev.max() / ev.min())
        d = np.diag(A)
        ej = sl.eigh(A, np.diag(d), eigvals_only=True)
        kj.append(ej.max() / ej.min())
    assert max(kl) <= 12.0
    assert kj[-1] > 5 * kl[-1] and kj[-1] > 2 * kj[0]


def _cheb_T(k, x):
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(k * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** k * np.cosh(k * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("k", [1, 2, 5, 8])
def test_chebyshev_is_the_residual_polynomial(k):
    """After k steps from z = 0 the error is R_k(D^-1 A) times the initial error, with
    R_k(l) = T_k((theta - l) / delta) / T_k(theta / delta) on [a, b] = [b / k^2, b]; so
    z = D^-1/2 f(S) D^-1/2 r, f(l) = (1 - R_k(l)) / l, S = D^-1/2 A D^-1/2 (eigendecomposition)."""
    shape, p = (2, 2, 2), 3
    V = S.structured_vertices(*shape, 0.1, 11)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    A = precond.lor_operator(mesh, 2.0, 1.0).assembled(constrained=True)
    r = S.uniform_pm1(12, mesh.n_dof)
    z = precond.chebyshev_apply(A, r, k)
    d = np.diag(A)
    Sm = A / np.sqrt(np.outer(d, d))
    lam, Vv = np.linalg.eigh(Sm)
    b = precond.gershgorin_bound(A)
    assert lam.max() <= b * (1 + 1e-12)          # the Gershgorin bound is an upper bound
    a = b / k ** 2
    theta, delta = (b + a) / 2, (b - a) / 2
    if k == 1:
        f = np.full_like(lam, 1.0 / theta)
    else:
        R = _cheb_T(k, (theta - lam) / delta) / _cheb_T(k, np.array([theta / delta]))[0]
        f = (1 - R) / lam
    z_ref = (Vv @ (f * (Vv.T @ (r / np.sqrt(d))))) / np.sqrt(d)
    assert np.abs(z - z_ref).max() <= 1e-11 * np.abs(z_ref).max()


def test_lor_collocated_mass_variant_is_the_sum_of_its_parts():
    shape, p = (2, 2, 1), 3
    V = S.structured_vertices(*shape, 0.1, 13)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    A = precond.lor_matrix(mesh, 4.0, 0.3, "collocated")
    K = precond.lor_operator(mesh, 0.0, 0.3).assembled(constrained=True)
    d = np.where(mesh.dirichlet, 0.0, precond.collocated_mass_diagonal(mesh, 4.0))
    assert np.abs(A - K - np.diag(d)).max() <= 1e-15 * np.abs(A).max()
    assert np.array_equal(precond.lor_matrix(mesh, 4.0, 0.3), precond.lor_operator(mesh, 4.0, 0.3).assembled(True))


# ---- geometric multigrid on the LOR matrix ----
def _lor_case(N, p, dirichlet=True, alpha=0.0, seed=14):
    V = S.structured_vertices(N, N, N, 0.1, seed)
    mesh = fem.StructuredMesh(N, N, N, p, p + 2, V, S.structured_elem_vert(N, N, N), dirichlet_boundary=dirichlet)
    A = precond.lor_matrix(mesh, alpha, 1.0, "collocated")
    return mesh, A, (p * N + 1,) * 3


def test_interpolation_reproduces_trilinear_functions():
    dims = (9, 5, 7)
    n = int(np.prod(dims))
    P, cd, cdir = precond.interpolation(dims, np.zeros(n, dtype=bool))
    assert cd == (5, 3, 4) and not cdir.any()
    def f(d):
        i = np.arange(int(np.prod(d)))
        x, y, z = i % d[0], (i // d[0]) % d[1], i // (d[0] * d[1])
        return x, y, z
    xf, yf, zf = f(dims)
    xc, yc, zc = f(cd)
    xf, yf, zf = xf / 2.0, yf / 2.0, zf / 2.0          # fine coordinates in coarse units
    for g in (lambda x, y, z: 1 + 0 * x, lambda x, y, z: 2 * x - y + 3 * z, lambda x, y, z: x * y * z - x * z + 0.5):
        assert np.abs(P @ g(xc, yc, zc) - g(xf, yf, zf)).max() <= 1e-13


def test_interpolation_respects_dirichlet():
    dims = (5, 5, 5)
    mesh_dir = np.zeros(125, dtype=bool)
    i = np.arange(125)
    x, y, z = i % 5, (i // 5) % 5, i // 25
    mesh_dir[(x == 0) | (x == 4) | (y == 0) | (y == 4) | (z == 0) | (z == 4)] = True
    P, cd, cdir = precond.interpolation(dims, mesh_dir)
    assert cd == (3, 3, 3) and cdir.sum() == 26
    assert np.all(np.asarray(P[mesh_dir].todense()) == 0)
    assert np.all(np.asarray(P[:, cdir].todense()) == 0)


def test_galerkin_coarse_operators_keep_symmetry_and_null_space():
    mesh, A, dims = _lor_case(4, 2, dirichlet=False)
    levels = precond.mg_hierarchy(A, dims, mesh.dirichlet)
    assert len(levels) == 3                          # 9^3 -> 5^3 -> 3^3
    for Al, _ in levels:
        assert np.abs(Al - Al.T).max() <= 1e-14 * np.abs(Al).max()
        assert np.abs(Al @ np.ones(Al.shape[0])).max() <= 1e-13 * np.abs(Al).max()


def test_vcycle_is_symmetric_positive_definite():
    mesh, A, dims = _lor_case(2, 4, alpha=3.0)
    levels = precond.mg_hierarchy(A, dims, mesh.dirichlet)
    n = A.shape[0]
    B = np.stack([precond.vcycle(levels, e) for e in np.eye(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_single_level_vcycle_is_the_coarse_chebyshev():
    mesh, A, dims = _lor_case(1, 2)                # 3^3 grid: below the coarsening size
    levels = precond.mg_hierarchy(A, dims, mesh.dirichlet)
    assert len(levels) == 1
    r = S.uniform_pm1(15, A.shape[0])
    z = precond.vcycle(levels, r)
    k = precond.MG_COARSE_DEGREE
    assert np.array_equal(z, precond.chebyshev_ratio_apply(A, r, k, float(k * k)))
    assert np.allclose(precond.chebyshev_ratio_apply(A, r, 5, 25.0), precond.chebyshev_apply(A, r, 5), rtol=0, atol=0)


def test_mg_pcg_iterations_bounded_under_refinement():
    """MG-preconditioned CG on the LOR Poisson matrix: iteration counts stay nearly flat as h halves,
    while Jacobi's double."""
    its_mg, its_j = [], []
    for N in (2, 4, 8):
        mesh, A, dims = _lor_case(N, 2)
        levels = precond.mg_hierarchy(A, dims, mesh.dirichlet)
        b = np.where(mesh.dirichlet, 0.0, S.uniform_pm1(16, A.shape[0]))
        for prec, its in ((lambda r: precond.vcycle(levels, r), its_mg), (lambda r: r / np.diag(A), its_j)):
            x = np.zeros_like(b); r = b.copy(); z = prec(r); pp = z.copy(); rz = r @ z
            for it in range(2000):
                Ap = A @ pp; a = rz / (pp @ Ap); x += a * pp; r -= a * Ap
                if np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b):
                    break
                z = prec(r); rz2 = r @ z; pp = z + (rz2 / rz) * pp; rz = rz2
            its.append(it + 1)
    assert its_mg[-1] <= its_mg[0] + 6 and its_mg[-1] <= 20, its_mg
    assert its_j[-1] >= 2 * its_j[1] - 5 and its_j[-1] > 3 * its_mg[-1], its_j


@pytest.mark.parametrize("p", [2, 3])
def test_lor_on_unstructured_star_prism(p):
    """The LOR matrix on a mesh whose central edge has valence 5: 1^T M_LOR 1 = the volume (the
    sub-elements of a multilinear map tile it exactly), K_LOR 1 = 0, and the rows of the central
    edge's interior DoFs couple to 2 x 5 + 1 = 11 nodes in each of 3 layers (33 entries)."""
    from tests.unstructured import star_prism, star_prism_volume
    V, EV, om = star_prism(p, dirichlet_bottom=False)
    one = np.ones(om.n_dof)
    M = precond.lor_matrix(om, 1.0, 0.0, constrained=False)
    assert abs(one @ M @ one - star_prism_volume()) < 1e-13
    K = precond.lor_matrix(om, 0.0, 1.0, constrained=False)
    assert np.abs(K @ one).max() < 1e-13
    X = om.node_coords()
    axis = (np.hypot(X[:, 0], X[:, 1]) < 1e-12) & (X[:, 2] > 1e-12) & (X[:, 2] < 1 - 1e-12)
    assert axis.sum() == 3 * p - 1
    assert np.all((K[axis] != 0).sum(axis=1) == 33)
    assert (K != 0).sum(axis=1).max() == 33


@pytest.mark.parametrize("dirichlet,alpha,nu", [(False, 0.0, 1.0), (True, 1000.0, 1e-2)])
def test_lor_rows_from_element_patches(dirichlet, alpha, nu):
    """The reference the full-size LOR tests use: a row of alpha Mc + nu K_LOR assembled from
    only the elements holding its DoF equals that row of the whole mesh's assembly, for every
    row of a small mesh (interior, face, edge and corner DoFs; with and without Dirichlet)."""
    from tests.gpu_common import case, lor_row_oracle
    V, EV, om = case((3, 3, 2), 3, dirichlet=dirichlet)
    A = precond.lor_matrix(om, alpha, nu, "collocated")
    for g in range(om.n_dof):
        cols, vals = lor_row_oracle(om, g, alpha, nu)
        nz = np.nonzero(A[g])[0]
        assert np.array_equal(cols, nz), g
        assert np.abs(vals - A[g, nz]).max() <= 1e-15 * np.abs(A[g]).max(), g
