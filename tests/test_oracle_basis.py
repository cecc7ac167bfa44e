"""Oracle 1D tables (Sec. 3.1, Eqs. (B1D), (D1D)) pinned to closed forms and exact integrals."""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle.basis import gauss_rule, gll_nodes, lagrange_derivatives, lagrange_values
from tests.oracle_pins import exact_1d_matrices, oracle_1d_matrices, read_rows


def _eval(tok):
    return float(eval(tok, {"sqrt": np.sqrt}))


def test_closed_form_nodes_and_weights():
    for kind, order, what, *vals in read_rows("gll_gauss_closed_forms.txt"):
        order = int(order)
        ref = np.array([_eval(v) for v in vals])
        if kind == "gll":
            got = gll_nodes(order)
        else:
            x, w = gauss_rule(order)
            got = x if what == "nodes" else w
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 13))
def test_gll_are_roots_of_legendre_derivative(p):
    x = gll_nodes(p)
    assert x[0] == -1.0 and x[-1] == 1.0 and np.all(np.diff(x) > 0)
    dP = L.Legendre.basis(p).deriv()
    if p > 1:
        assert np.max(np.abs(dP(x[1:-1]))) < 1e-12 * max(1.0, np.max(np.abs(dP.coef)))
    # GLL quadrature weights 2/(p(p+1) P_p(x)^2) integrate degree 2p-1 exactly (independent check)
    w = 2.0 / (p * (p + 1) * L.Legendre.basis(p)(x) ** 2)
    for k in range(2 * p):
        assert abs(w @ x ** k - (2.0 / (k + 1) if k % 2 == 0 else 0.0)) < 1e-13


@pytest.mark.parametrize("q", range(1, 14))
def test_gauss_rule_matches_library_and_exactness(q):
    x, w = gauss_rule(q)
    xl, wl = L.leggauss(q)
    np.testing.assert_allclose(x, xl, atol=1e-14)
    np.testing.assert_allclose(w, wl, atol=1e-14)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * q):
        assert abs(w @ x ** k - (2.0 / (k + 1) if k % 2 == 0 else 0.0)) < 1e-13
    # not exact at degree 2q
    assert abs(w @ x ** (2 * q) - 2.0 / (2 * q + 1)) > 1e-8


@pytest.mark.parametrize("p", range(1, 9))
def test_B_D_reproduce_polynomials(p):
    q = p + 2
    nodes = gll_nodes(p)
    xq, _ = gauss_rule(q)
    B = lagrange_values(nodes, xq)
    D = lagrange_derivatives(nodes, xq)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-12)
    for k in range(p + 1):
        np.testing.assert_allclose(B @ nodes ** k, xq ** k, atol=1e-13)
        dk = k * xq ** (k - 1) if k > 0 else 0 * xq
        np.testing.assert_allclose(D @ nodes ** k, dk, atol=1e-11)
    # Lagrange property at the nodes themselves
    np.testing.assert_allclose(lagrange_values(nodes, nodes), np.eye(p + 1), atol=1e-14)


def test_p2_textbook_element_matrices():
    rows = np.array(read_rows("p2_element_matrices_1d.txt"), dtype=float)
    M_ref, K_ref = rows[:3] / 15.0, rows[3:] / 6.0
    M, K = oracle_1d_matrices(2, 4)
    np.testing.assert_allclose(M, M_ref, atol=1e-15)
    np.testing.assert_allclose(K, K_ref, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_1d_matrices_equal_exact_integrals(p):
    Me, Ke = exact_1d_matrices(p)
    M, K = oracle_1d_matrices(p, p + 2)
    np.testing.assert_allclose(M, Me, atol=1e-13 * np.abs(Me).max())
    np.testing.assert_allclose(K, Ke, atol=1e-12 * np.abs(Ke).max())
