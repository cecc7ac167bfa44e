"""Oracle operator alpha M + nu K (Sec. 3.1) pinned to exact integrals, invariants and brute force."""
import numpy as np
import pytest

import synthetic as S
from oracle import fem
from tests.oracle_pins import box_element_error, energy_error, volume_error


def small_mesh(n=(2, 1, 1), p=2, q=None, perturb=0.1, seed=5, dirichlet=False):
    q = p + 2 if q is None else q
    V = S.structured_vertices(*n, perturb, seed)
    return fem.StructuredMesh(*n, p, q, V, S.structured_elem_vert(*n), dirichlet_boundary=dirichlet)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_box_element_is_kronecker_of_exact_1d(p):
    assert box_element_error(p, p + 2) < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4])
def test_energy_exact_on_sheared_affine_mesh(p):
    eK, eM = energy_error(p, p + 2)
    assert eK < 1e-12 and eM < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_mass_integrates_volume_on_perturbed_cube(p):
    assert volume_error(p, p + 2) < 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_stiffness_annihilates_constants_and_has_nullity_one(p):
    mesh = small_mesh((2, 1, 1), p)
    K = fem.Operator(mesh, 0.0, 1.0)
    one = np.ones(mesh.n_dof)
    Kd = K.assembled()
    assert np.max(np.abs(K.apply(one))) < 1e-14 * np.max(np.abs(Kd))
    ev = np.linalg.eigvalsh(Kd)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 1


@pytest.mark.parametrize("shape,p", [((1, 1, 1), 2), ((1, 1, 1), 3), ((2, 1, 1), 2), ((1, 2, 1), 3)])
def test_spsd_by_brute_force(shape, p):
    mesh = small_mesh(shape, p)
    for alpha, nu, definite in [(0.0, 1.0, False), (1.3, 0.0, True), (2.0, 0.7, True)]:
        op = fem.Operator(mesh, alpha, nu)
        # columns of the global matrix from applies to unit vectors
        A = np.stack([op.apply(e) for e in np.eye(mesh.n_dof)], axis=1)
        assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
        ev = np.linalg.eigvalsh(A)
        assert ev.min() >= -1e-12 * ev.max()
        if definite:
            assert ev.min() > 1e-10 * ev.max()


def test_constrained_operator_and_diagonal_brute_force():
    mesh = small_mesh((2, 2, 1), 2, dirichlet=True)
    op = fem.Operator(mesh, 1.5, 0.8)
    Ac = np.stack([op.apply(e, constrained=True) for e in np.eye(mesh.n_dof)], axis=1)
    d = mesh.dirichlet
    assert np.all(Ac[np.ix_(d, d)] == np.eye(d.sum()))
    assert np.all(Ac[np.ix_(d, ~d)] == 0) and np.all(Ac[np.ix_(~d, d)] == 0)
    A = np.stack([op.apply(e) for e in np.eye(mesh.n_dof)], axis=1)
    np.testing.assert_array_equal(Ac[np.ix_(~d, ~d)], A[np.ix_(~d, ~d)])
    np.testing.assert_allclose(op.diagonal(), np.diag(A), rtol=1e-15, atol=0)
    np.testing.assert_allclose(op.diagonal(constrained=True), np.diag(Ac), rtol=1e-15, atol=0)
    assert np.all(np.linalg.eigvalsh(Ac) > 0)


def test_apply_rows_matches_apply():
    mesh = small_mesh((3, 2, 2), 3, dirichlet=True)
    op = fem.Operator(mesh, 1.0, 0.3)
    x = S.random_vector(mesh.n_dof, 9)
    dofs = np.array([0, 1, 5, 17, mesh.n_dof // 2, mesh.n_dof - 1, 123])
    for constrained in (False, True):
        y = op.apply(x, constrained)
        np.testing.assert_allclose(op.apply_rows(x, dofs, constrained), y[dofs], rtol=1e-13, atol=1e-15)


def test_structured_numbering_is_continuous():
    """Every element maps its local nodes to the same physical point as every other element sharing them."""
    mesh = small_mesh((3, 2, 2), 3)
    X = mesh.node_coords()
    XE = mesh.element_node_coords()
    np.testing.assert_allclose(XE, X[mesh.restriction], atol=1e-15)
    # DoF count and multiplicities of a structured grid
    assert mesh.n_dof == (3 * 3 + 1) * (3 * 2 + 1) * (3 * 2 + 1)
    assert len(np.unique(mesh.restriction)) == mesh.n_dof
    for g in [0, 10, 57, mesh.n_dof - 1]:
        pairs = mesh.elements_of_dof(g)
        assert all(mesh.restriction[e, l] == g for e, l in pairs)
        assert len(pairs) == np.sum(mesh.restriction == g)


def test_load_vector_equals_mass_times_interpolant_for_linear_f():
    mesh = small_mesh((2, 2, 2), 3, perturb=0.1, seed=11)
    f = lambda X: 0.3 + 1.2 * X[..., 0] - 0.7 * X[..., 1] + 2.1 * X[..., 2]
    b = fem.load_vector(mesh, f(mesh.qpoint_coords()))
    fL = f(mesh.node_coords())
    np.testing.assert_allclose(b, fem.Operator(mesh, 1.0, 0.0).apply(fL), rtol=0, atol=1e-14)


def test_nu_field_linearity():
    mesh = small_mesh((2, 1, 1), 2)
    Q = mesh.ref.Q
    x = S.random_vector(mesh.n_dof, 4)
    a = fem.Operator(mesh, 0.5, 0.25).apply(x)
    b = fem.Operator(mesh, 0.5, np.full((mesh.n_elem, Q), 0.25)).apply(x)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-15)
    nu1 = 1.0 + S.uniform_pm1(3, mesh.n_elem * Q).reshape(mesh.n_elem, Q) ** 2
    nu2 = 0.5 + S.uniform_pm1(4, mesh.n_elem * Q).reshape(mesh.n_elem, Q) ** 2
    K1 = fem.Operator(mesh, 0.0, nu1).apply(x)
    K2 = fem.Operator(mesh, 0.0, nu2).apply(x)
    K12 = fem.Operator(mesh, 0.0, nu1 + 2 * nu2).apply(x)
    np.testing.assert_allclose(K12, K1 + 2 * K2, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_unstructured_star_prism(p):
    """A mesh whose central edge has valence 5 (numbering from node positions): 1^T M 1 is the
    prism's closed-form volume (bilinear quads, linear in z: the quadrature is exact), K 1 = 0,
    and the assembled matrix is symmetric with a one-dimensional null space of K."""
    from tests.unstructured import star_prism, star_prism_volume
    V, EV, om = star_prism(p, dirichlet_bottom=False)
    one = np.ones(om.n_dof)
    assert abs(one @ fem.Operator(om, 1.0, 0.0).apply(one) - star_prism_volume()) < 1e-13
    K = fem.Operator(om, 0.0, 1.0)
    assert np.abs(K.apply(one)).max() < 1e-13
    assert np.bincount(om.restriction.ravel()).max() == 10     # the central edge: 5 sectors x 2 layers
    if p <= 2:
        A = K.assembled()
        assert np.abs(A - A.T).max() < 1e-13
        ev = np.linalg.eigvalsh(A)
        assert abs(ev[0]) < 1e-11 and ev[1] > 1e-6
