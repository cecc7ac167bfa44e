"""Oracle adjoint gradients pinned by central finite differences of the loss."""
import numpy as np
import pytest

import synthetic as S
from oracle import adjoint, fem


def _problem(seed=3):
    shape, p = (2, 2, 1), 2
    V = S.structured_vertices(*shape, 0.1, seed)
    mesh = fem.StructuredMesh(*shape, p, p + 2, V, S.structured_elem_vert(*shape))
    E, Q = mesh.n_elem, mesh.ref.Q
    nu = np.exp(np.log(1e-2) + 0.5 * S.uniform_pm1(seed + 1, E * Q)).reshape(E, Q)
    f = S.uniform_pm1(seed + 2, E * Q).reshape(E, Q)
    ut = np.where(mesh.dirichlet, 0.0, S.uniform_pm1(seed + 3, mesh.n_dof))
    return mesh, 3.0, nu, f, ut


def test_gradients_match_central_differences():
    mesh, alpha, nu, f, ut = _problem()
    L, dnu, df, u, lam = adjoint.gradients(mesh, alpha, nu, f, ut)
    L0, _ = adjoint.loss(mesh, alpha, nu, f, ut)
    assert abs(L - L0) <= 1e-14 * abs(L0)
    for k in range(4):
        dn = S.uniform_pm1(50 + k, nu.size).reshape(nu.shape) * nu     # relative perturbation
        dfv = S.uniform_pm1(60 + k, f.size).reshape(f.shape)
        h = 1e-6
        Lp, _ = adjoint.loss(mesh, alpha, nu + h * dn, f + h * dfv, ut)
        Lm, _ = adjoint.loss(mesh, alpha, nu - h * dn, f - h * dfv, ut)
        fd = (Lp - Lm) / (2 * h)
        an = np.sum(dnu * dn) + np.sum(df * dfv)
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-12), (fd, an)


def test_gradient_of_f_is_interpolated_adjoint():
    """dL/df vanishes where the adjoint does (Dirichlet-only support) and is linear in lam."""
    mesh, alpha, nu, f, ut = _problem(5)
    L, dnu, df, u, lam = adjoint.gradients(mesh, alpha, nu, f, ut)
    assert np.all(lam[mesh.dirichlet] == 0)
    # df contracted with f gives lam . b (b linear in f)
    b = np.where(mesh.dirichlet, 0.0, fem.load_vector(mesh, f))
    assert abs(np.sum(df * f) - lam @ b) <= 1e-12 * abs(lam @ b)
