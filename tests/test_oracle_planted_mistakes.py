"""Planted mistakes in the oracle (on the CPU) must each be caught by a pin.

Each case monkeypatches one plausible error into the oracle and checks that
the corresponding pin computation then reports a large error.
"""
import numpy as np
import pytest

from oracle import basis, fem
from tests import oracle_pins as pins


def test_transposed_jacobian_convention_is_caught(monkeypatch):
    # the literal J^-T |J| J^-1 of Eq. (localStiffnessMapped) read with J_ij = dx_i/dxi_j
    orig = fem.Operator.geometry

    def transposed(self, es):
        detJ, Jinv = orig(self, es)
        return detJ, np.swapaxes(Jinv, -1, -2)

    monkeypatch.setattr(fem.Operator, "geometry", transposed)
    eK, _ = pins.energy_error(2, 4)
    assert eK > 1e-3


def test_dropped_mass_term_is_caught(monkeypatch):
    orig = fem.Operator.__init__

    def no_mass(self, mesh, alpha, nu, *a, **k):
        orig(self, mesh, 0.0, nu, *a, **k)

    monkeypatch.setattr(fem.Operator, "__init__", no_mass)
    assert pins.volume_error(2, 4) > 0.5


def test_wrong_derivative_sign_is_caught(monkeypatch):
    # flip the sign of one basis function's derivative column (a plausible sign slip in D)
    orig = basis.lagrange_derivatives
    flip = lambda nodes, x: orig(nodes, x) * np.where(np.arange(len(nodes)) == 0, -1.0, 1.0)
    monkeypatch.setattr(fem, "lagrange_derivatives", flip)
    assert pins.box_element_error(2, 4) > 1e-3


def test_wrong_gauss_weight_is_caught(monkeypatch):
    orig = basis.gauss_rule

    def bad(q):
        x, w = orig(q)
        w = w.copy()
        w[0] *= 1.001
        return x, w

    monkeypatch.setattr(fem, "gauss_rule", bad)
    assert pins.volume_error(2, 4) > 1e-5


def test_too_few_quadrature_points_is_caught():
    # q = p (under-integration) no longer reproduces the exact energy
    eK, eM = pins.energy_error(3, 3)
    assert max(eK, eM) > 1e-8


def test_swapped_restriction_is_caught(monkeypatch):
    orig = fem.structured_restriction

    def swapped(nx, ny, nz, p):
        R = orig(nx, ny, nz, p).copy()
        R[:, [1, p + 1]] = R[:, [p + 1, 1]]   # swap local nodes (1,0,0) and (0,1,0)
        return R

    monkeypatch.setattr(fem, "structured_restriction", swapped)
    eK, eM = pins.energy_error(2, 4)
    assert max(eK, eM) > 1e-3


# ---- preconditioner and adjoint parts of the oracle ----
def test_wrong_gll_endpoint_weight_is_caught(monkeypatch):
    """An endpoint weight off by a factor (e.g. 2/(p(p+1)) read as 1/(p(p+1))) breaks the
    collocated mass's sum = alpha x volume."""
    import synthetic as S
    from oracle import precond
    orig = precond.gll_weights

    def bad(p):
        w = orig(p).copy()
        w[0] *= 0.5
        return w

    monkeypatch.setattr(precond, "gll_weights", bad)
    shape = (3, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 7)
    mesh = fem.StructuredMesh(*shape, 3, 5, V, S.structured_elem_vert(*shape))
    assert abs(precond.collocated_mass_diagonal(mesh, 2.5).sum() - 2.5) > 1e-2


def test_twisted_lor_sub_element_is_caught(monkeypatch):
    """Sub-element corners 2 and 3 exchanged (a lexicographic-vs-cyclic corner order mix-up):
    the sub-element map folds over, which the LOR volume pin (or the detJ > 0 check) rejects."""
    import synthetic as S
    from oracle import precond
    orig = precond.lor_mesh

    def twisted(mesh):
        m = orig(mesh)
        ev = m.elem_vert.copy()
        ev[:, [2, 3]] = ev[:, [3, 2]]
        return fem.Mesh(1, 2, m.vertices, ev, ev, m.n_dof, m.dirichlet)

    monkeypatch.setattr(precond, "lor_mesh", twisted)
    shape = (2, 2, 2)
    V = S.structured_vertices(*shape, 0.1, 9)
    mesh = fem.StructuredMesh(*shape, 2, 4, V, S.structured_elem_vert(*shape))
    one = np.ones(mesh.n_dof)
    try:
        vol = one @ precond.lor_operator(mesh, 1.0, 0.0).apply(one)
    except ValueError:                  # a folded sub-element: detJ <= 0 at a quadrature point
        return
    assert abs(vol - 1.0) > 1e-3        # otherwise the volume pin must see it


def test_signed_gershgorin_sum_is_caught(monkeypatch):
    """Row sums without absolute values give a 'bound' below the spectrum of D^-1 A, which the
    Chebyshev pin checks (lambda_max <= b) before using it."""
    import synthetic as S
    from oracle import precond

    def signed(A):
        A = np.asarray(A, dtype=np.float64)
        return float(np.max(A.sum(axis=1) / np.diag(A)))

    monkeypatch.setattr(precond, "gershgorin_bound", signed)
    shape, p = (2, 2, 2), 3
    V = S.structured_vertices(*shape, 0.1, 11)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    A = precond.lor_operator(mesh, 2.0, 1.0).assembled(constrained=True)
    d = np.diag(A)
    lam = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d)))
    assert lam.max() > precond.gershgorin_bound(A) * (1 + 1e-12)


def test_swapped_interpolation_axes_are_caught(monkeypatch):
    """Grid axes read in the wrong order (y fastest): trilinear functions are no longer
    reproduced on a non-cubic grid."""
    from oracle import precond
    orig = precond.interpolation
    monkeypatch.setattr(precond, "interpolation", lambda dims, d: orig((dims[1], dims[0], dims[2]), d))
    dims = (9, 5, 7)
    n = int(np.prod(dims))
    P, cd, _ = precond.interpolation(dims, np.zeros(n, dtype=bool))
    i = np.arange(n)
    xf = (i % dims[0]) / 2.0
    ic = np.arange(int(np.prod(cd)))
    xc = ic % 5                       # coarse x index of the correct (5, 3, 4) grid
    assert cd != (5, 3, 4) or np.abs(P @ (2.0 * xc) - 2.0 * xf).max() > 1e-3


def test_dropped_gradient_sign_is_caught(monkeypatch):
    """dL/dnu with the sign of the adjoint identity dropped fails the central differences."""
    import synthetic as S
    from oracle import adjoint
    orig = adjoint.point_gradients
    monkeypatch.setattr(adjoint, "point_gradients", lambda mesh, u, lam, elems=None:
                        tuple(s * g for s, g in zip((-1.0, 1.0), orig(mesh, u, lam, elems))))
    shape, p = (2, 2, 1), 2
    V = S.structured_vertices(*shape, 0.1, 3)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    E, Q = mesh.n_elem, mesh.ref.Q
    nu = np.exp(np.log(1e-2) + 0.5 * S.uniform_pm1(4, E * Q)).reshape(E, Q)
    f = S.uniform_pm1(5, E * Q).reshape(E, Q)
    ut = np.where(mesh.dirichlet, 0.0, S.uniform_pm1(6, mesh.n_dof))
    L, dnu, df, u, lam = adjoint.gradients(mesh, 3.0, nu, f, ut)
    dn = S.uniform_pm1(50, nu.size).reshape(nu.shape) * nu
    h = 1e-6
    fd = (adjoint.loss(mesh, 3.0, nu + h * dn, f, ut)[0] - adjoint.loss(mesh, 3.0, nu - h * dn, f, ut)[0]) / (2 * h)
    assert abs(fd - np.sum(dnu * dn)) > 1e-3 * abs(fd)
