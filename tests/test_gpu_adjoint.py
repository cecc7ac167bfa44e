"""Adjoint gradients (dL/dnu_q, dL/df_q of a loss of the solved field) through the C ABI and the
torch.autograd binding, vs the CPU oracle and central finite differences."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


def lognormal_nu(E, Q, seed, mu=np.log(1e-2), sigma=0.5):
    return np.exp(mu + sigma * S.uniform_pm1(seed, E * Q)).reshape(E, Q)


@pytest.mark.parametrize("p,dq", [(1, 2), (2, 1), (2, 2), (3, 2), (4, 1), (4, 2), (5, 2), (6, 2), (7, 1), (8, 2)])
def test_gradient_kernel_matches_oracle(hx, p, dq):
    """The contraction alone, on arbitrary u and lam (zero on the Dirichlet boundary)."""
    from oracle.adjoint import point_gradients
    shape = (3, 2, 2) if p <= 5 else (2, 2, 1)
    V, EV, om = case(shape, p, p + dq, perturb=0.15, seed=77 + p)
    mesh = hx.Mesh.structured(*shape, p, p + dq, V)
    op = hx.Operator(mesh, 1.0, 0.5)
    u = np.where(om.dirichlet, 0.0, S.uniform_pm1(5 + p, om.n_dof))
    lam = np.where(om.dirichlet, 0.0, S.uniform_pm1(6 + p, om.n_dof))
    dnu, df = op.gradient(to_dev(u), to_dev(lam))
    dnu_o, df_o = point_gradients(om, u, lam)
    assert rel_err(dnu.cpu().numpy(), dnu_o) <= 1e-12
    assert rel_err(df.cpu().numpy(), df_o) <= 1e-12


def test_gradient_ignores_dirichlet_entries(hx):
    """Entries of u and lam at Dirichlet DoFs do not enter (they are zero for solutions of A_c)."""
    p, shape = 3, (2, 2, 2)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1.0, 1.0)
    u = S.uniform_pm1(11, om.n_dof)
    lam = S.uniform_pm1(12, om.n_dof)
    a = op.gradient(to_dev(u), to_dev(lam))
    b = op.gradient(to_dev(np.where(om.dirichlet, 0.0, u)), to_dev(np.where(om.dirichlet, 0.0, lam)))
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def _problem(hx, shape=(4, 4, 4), p=4, alpha=10.0, seed=21, mu=np.log(1e-2)):
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    E, Q = om.n_elem, om.ref.Q
    nu = lognormal_nu(E, Q, seed, mu)
    f = S.uniform_pm1(seed + 1, E * Q).reshape(E, Q)
    ut = np.where(om.dirichlet, 0.0, S.uniform_pm1(seed + 2, om.n_dof))
    return om, mesh, alpha, nu, f, ut


def _loss(hx, ag, op, mass, alpha, nu, f, ut, rtol=1e-13):
    u = ag.solve(op, alpha, nu, f, rtol=rtol)
    d = u - ut
    return 0.5 * torch.dot(d, ag.apply(mass, d))


def test_autograd_matches_oracle(hx):
    from oracle import adjoint
    import paper_1910_03032_b300.autograd as ag
    om, mesh, alpha, nu, f, ut = _problem(hx)
    L_o, dnu_o, df_o, u_o, lam_o = adjoint.gradients(om, alpha, nu, f, ut)
    op = hx.Operator(mesh, alpha, 0.0, to_dev(nu))
    mass = hx.Operator(mesh, 1.0, 0.0)
    nu_t = to_dev(nu).requires_grad_(True)
    f_t = to_dev(f).requires_grad_(True)
    L = _loss(hx, ag, op, mass, alpha, nu_t, f_t, to_dev(ut))
    L.backward()
    assert abs(L.item() - L_o) <= 1e-10 * abs(L_o)
    assert rel_err(nu_t.grad.cpu().numpy(), dnu_o) <= 1e-9
    assert rel_err(f_t.grad.cpu().numpy(), df_o) <= 1e-9


def test_autograd_matches_central_differences(hx):
    """20 random directions, 10 in nu (h = 1e-6 relative to nu) and 10 in f, on the GPU solve itself."""
    import paper_1910_03032_b300.autograd as ag
    om, mesh, alpha, nu, f, ut = _problem(hx, shape=(4, 4, 3), p=3, alpha=1.0, seed=31, mu=np.log(0.1))
    op = hx.Operator(mesh, alpha, 0.0, to_dev(nu))
    mass = hx.Operator(mesh, 1.0, 0.0)
    nu_t, f_t, ut_t = to_dev(nu).requires_grad_(True), to_dev(f).requires_grad_(True), to_dev(ut)
    L = _loss(hx, ag, op, mass, alpha, nu_t, f_t, ut_t, 1e-14)
    L.backward()
    gnu, gf = nu_t.grad.clone(), f_t.grad.clone()
    h = 1e-6
    # directions with a non-zero mean, so that the directional derivative is not a sum of
    # cancelling terms far below the rounding of L (eps |L| / h)
    with torch.no_grad():
        for k in range(20):
            dn = to_dev((0.5 + 0.5 * S.uniform_pm1(100 + k, nu.size)).reshape(nu.shape) * nu * (k < 10))
            dfv = to_dev((0.5 + S.uniform_pm1(200 + k, f.size)).reshape(f.shape) * (k >= 10))
            Lp = _loss(hx, ag, op, mass, alpha, to_dev(nu) + h * dn, to_dev(f) + h * dfv, ut_t, 1e-14).item()
            Lm = _loss(hx, ag, op, mass, alpha, to_dev(nu) - h * dn, to_dev(f) - h * dfv, ut_t, 1e-14).item()
            fd = (Lp - Lm) / (2 * h)
            an = (torch.sum(gnu * dn) + torch.sum(gf * dfv)).item()
            floor = 64 * np.finfo(float).eps * abs(L.item()) / h
            assert abs(fd - an) <= 1e-5 * abs(an) + floor, (k, fd, an, floor)


def test_backward_after_operator_changed(hx):
    """The backward solve re-sets the forward coefficients when the operator was changed in between."""
    import paper_1910_03032_b300.autograd as ag
    om, mesh, alpha, nu, f, ut = _problem(hx, shape=(3, 3, 2), p=3, seed=41)
    op = hx.Operator(mesh, alpha, 0.0, to_dev(nu))
    mass = hx.Operator(mesh, 1.0, 0.0)
    grads = []
    for change in (False, True):
        nu_t = to_dev(nu).requires_grad_(True)
        L = _loss(hx, ag, op, mass, alpha, nu_t, to_dev(f), to_dev(ut))
        if change:
            op.set_coefficients(alpha, 0.0, to_dev(2.0 * nu))
        L.backward()
        grads.append(nu_t.grad.cpu().numpy())
    assert rel_err(grads[1], grads[0]) <= 1e-12


def test_gradient_identities_full_size(hx):
    """At 32^3, p = 4: sum(dnu * nu) = -lam^T K(nu) u and sum(df * f) = lam^T P b(f), plus sampled
    elements of the contraction against the oracle, for the GPU's own u and lam."""
    from oracle.adjoint import point_gradients
    shape, p = (32, 32, 32), 4
    V, EV, om = case(shape, p, lazy=True)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    E, Q = om.n_elem, (p + 2) ** 3
    nu = to_dev(lognormal_nu(E, Q, 51))
    f = to_dev(S.uniform_pm1(52, E * Q).reshape(E, Q))
    op = hx.Operator(mesh, 1000.0, 0.0, nu)
    b = op.load_vector(f)
    u, info = op.solve(b, rtol=1e-11)
    rhs = to_dev(S.uniform_pm1(53, om.n_dof))
    lam, _ = op.solve(rhs, rtol=1e-11)
    dnu, df = op.gradient(u, lam)
    Kop = hx.Operator(mesh, 0.0, 0.0, nu)
    lKu = torch.dot(lam, Kop.apply(u)).item()
    assert abs(torch.sum(dnu * nu).item() + lKu) <= 1e-11 * abs(lKu)
    bm = torch.where(to_dev(om.dirichlet.astype(np.float64)) > 0, torch.zeros_like(b), b)
    lb = torch.dot(lam, bm).item()
    assert abs(torch.sum(df * f).item() - lb) <= 1e-11 * abs(lb)
    els = np.unique(S.permutation(E, 54)[:6].tolist() + [0, E - 1])
    un, ln = u.cpu().numpy(), lam.cpu().numpy()
    dnu_o, df_o = point_gradients(om, un, ln, els)
    assert rel_err(dnu.cpu().numpy()[els], dnu_o) <= 1e-12
    assert rel_err(df.cpu().numpy()[els], df_o) <= 1e-12
