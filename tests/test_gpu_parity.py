"""CUDA path (through the C ABI) vs the CPU FP64 oracle, element by element.

Tolerance for the FP64 operator: relative 1e-12 in the 2-norm and per entry
1e-12 of the largest entry (the sum-factorized, even-odd folded kernels round
in a different order from the oracle's explicit element matrices; the
difference is a few ulps times the number of terms, ~1e-15 relative).
"""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, mms_exact, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-12

# (p, mesh shape): several thread blocks and a ragged last block for each order
# (elements per block: p=1: 64, 2: 32, 3: 16, 4: 8, 5: 6, 6: 4, 7: 3, 8: 2)
CASES = [(1, (5, 5, 3)), (2, (5, 5, 3)), (3, (5, 5, 3)), (4, (5, 3, 3)), (5, (4, 3, 2)), (6, (3, 3, 1)),
         (7, (2, 2, 2)), (8, (3, 3, 1))]


def _assert_close(y, ref, tol=TOL):
    y, ref = np.asarray(y), np.asarray(ref)
    assert rel_err(y, ref) <= tol, rel_err(y, ref)
    np.testing.assert_allclose(y, ref, rtol=0, atol=tol * np.abs(ref).max())


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


@pytest.mark.parametrize("p,shape", CASES)
@pytest.mark.parametrize("dq", [1, 2])
@pytest.mark.parametrize("geom", [0, 1])
def test_apply_matches_oracle(hx, p, shape, dq, geom):
    from oracle import fem
    q = p + dq
    V, EV, om = case(shape, p, q)
    alpha, nu = 1.7, 0.45
    oop = fem.Operator(om, alpha, nu)
    mesh = hx.Mesh.structured(*shape, p, q, V)
    op = hx.Operator(mesh, alpha, nu, geom_mode=geom)
    x = S.random_vector(om.n_dof, 3032)
    xd = to_dev(x)
    for constrained in (False, True):
        y = op.apply(xd, constrained=constrained).cpu().numpy()
        _assert_close(y, oop.apply(x, constrained=constrained))


@pytest.mark.parametrize("geom", [0, 1])
def test_apply_nu_field(hx, geom):
    from oracle import fem
    p, shape = 3, (4, 3, 3)
    V, EV, om = case(shape, p)
    Q = om.ref.Q
    nu_q = np.exp(np.log(1e-2) + 0.5 * S.uniform_pm1(99, om.n_elem * Q)).reshape(om.n_elem, Q)
    oop = fem.Operator(om, 2.0, nu_q)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 2.0, 0.0, nu_q=to_dev(nu_q), geom_mode=geom)
    x = S.random_vector(om.n_dof, 5)
    _assert_close(op.apply(to_dev(x)).cpu().numpy(), oop.apply(x))


@pytest.mark.parametrize("p,shape", [(1, (5, 5, 3)), (2, (5, 5, 3)), (4, (5, 3, 3)), (6, (3, 3, 1)), (8, (3, 1, 1))])
@pytest.mark.parametrize("geom", [0, 1])
def test_diagonal_matches_oracle(hx, p, shape, geom):
    from oracle import fem
    V, EV, om = case(shape, p)
    oop = fem.Operator(om, 3.0, 0.2)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 3.0, 0.2, geom_mode=geom)
    for constrained in (False, True):
        _assert_close(op.diagonal(constrained).cpu().numpy(), oop.diagonal(constrained))


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_coordinates_and_load_vector(hx, p):
    from oracle import fem
    shape = (3, 2, 2) if p < 8 else (2, 1, 1)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    xq = mesh.qpoint_coords().cpu().numpy()
    np.testing.assert_allclose(xq, om.qpoint_coords(), rtol=0, atol=1e-15)
    np.testing.assert_allclose(mesh.node_coords().cpu().numpy(), om.node_coords(), rtol=0, atol=1e-15)
    op = hx.Operator(mesh, 1.0, 1.0)
    f = (1 + 3 * np.pi ** 2) * mms_exact(xq)
    _assert_close(op.load_vector(to_dev(f)).cpu().numpy(), fem.load_vector(om, f))


def test_apply_is_bitwise_reproducible(hx):
    p, shape = 4, (5, 4, 3)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    x = to_dev(S.random_vector(om.n_dof, 17))
    y1 = op.apply(x, constrained=True)
    y2 = op.apply(x, constrained=True)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("p,q,shape", [(1, 3, (3, 2, 2)), (2, 4, (4, 3, 5)), (3, 4, (3, 3, 2)), (4, 6, (5, 4, 3)),
                                       (5, 7, (2, 3, 2)), (8, 10, (2, 2, 3)), (3, 5, (1, 1, 1)), (2, 3, (7, 1, 1))])
def test_box_mesh_assembly_equals_transpose_map(hx, p, q, shape):
    """A box mesh assembles by index arithmetic (one x-run of nodes per thread, E-vectors in the
    line layout), a general mesh through its transpose map: the same mesh built both ways gives
    bit-identical FP64 and FP32 applies (the arithmetic visits a DoF's element entries in the
    map's order).  The solves agree to rounding: the CG inner products are summed run by run on
    the box mesh and DoF by DoF on the general one."""
    V, EV, om = case(shape, p, q=q)
    box = hx.Mesh.structured(*shape, p, q, V)
    gen = hx.Mesh.general(p, q, V, EV, om.n_dof, om.restriction, om.dirichlet.astype(np.uint8))
    ops = [hx.Operator(m, 1.3, 0.7) for m in (box, gen)]
    x = to_dev(S.random_vector(om.n_dof, 9))
    for constrained in (False, True):
        a, b = (o.apply(x, constrained=constrained) for o in ops)
        assert torch.equal(a, b)
    a, b = (o.apply_f32(x.float()) for o in ops)
    assert torch.equal(a, b)
    for constrained in (False, True):
        a, b = (o.diagonal(constrained) for o in ops)
        assert torch.equal(a, b)
    (xa, ia), (xb, ib) = (o.solve(x, rtol=1e-10) for o in ops)
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    assert float((xa - xb).norm() / xb.norm()) < 1e-8


def test_general_mesh_with_permuted_numbering(hx):
    """hx_mesh_create with shuffled elements and DoF ids gives the permuted result."""
    from oracle import fem
    p, shape = 3, (4, 3, 2)
    V, EV, om = case(shape, p)
    eperm = S.permutation(om.n_elem, 41)
    dperm = S.permutation(om.n_dof, 42)          # new id of old DoF g is dperm[g]
    R = dperm[om.restriction[eperm]]
    dirichlet = np.zeros(om.n_dof, np.uint8)
    dirichlet[dperm[om.dirichlet]] = 1
    mesh = hx.Mesh.general(p, p + 2, V, EV[eperm], om.n_dof, R, dirichlet)
    op = hx.Operator(mesh, 1.3, 0.7)
    oop = fem.Operator(om, 1.3, 0.7)
    x = S.random_vector(om.n_dof, 7)
    xn = np.empty_like(x)
    xn[dperm] = x
    for constrained in (False, True):
        y = op.apply(to_dev(xn), constrained=constrained).cpu().numpy()
        _assert_close(y[dperm], oop.apply(x, constrained=constrained))


def test_solve_config1_manufactured_solution(hx):
    """4^3 perturbed mesh, Q_3, 5^3 Gauss points, alpha = nu = 1, Jacobi-PCG to 1e-10."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    p, shape = 3, (4, 4, 4)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1.0, 1.0)
    x = S.random_vector(om.n_dof, 3032)
    oop = fem.Operator(om, 1.0, 1.0)
    _assert_close(op.apply(to_dev(x)).cpu().numpy(), oop.apply(x))
    # manufactured right-hand side, assembled by each side from its own quadrature points
    xq = mesh.qpoint_coords()
    f = (1.0 + 3 * np.pi ** 2) * mms_exact(xq.cpu().numpy())
    b = op.load_vector(to_dev(f))
    bo = fem.load_vector(om, (1.0 + 3 * np.pi ** 2) * mms_exact(om.qpoint_coords()))
    _assert_close(b.cpu().numpy(), bo)
    u, info = op.solve(b, rtol=1e-10)
    uo, its, rel, conv = jacobi_pcg(oop, bo, 1e-10)
    assert info["status"] == 0 and conv
    assert abs(info["iterations"] - its) <= 2, (info, its)
    assert info["rel_residual"] <= 1e-10 and info["true_rel_residual"] <= 1.01e-10
    assert rel_err(u.cpu().numpy(), uo) <= 1e-8
    # the discrete solution converges to the manufactured one
    assert fem.l2_error(om, u.cpu().numpy(), mms_exact) < 2e-4


@pytest.mark.parametrize("geom", [0, 1])
def test_solve_matches_dense_and_host_api(hx, geom):
    from oracle import fem
    p, shape = 2, (3, 3, 2)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1000.0, 1e-2, geom_mode=geom)
    oop = fem.Operator(om, 1000.0, 1e-2)
    b = S.random_vector(om.n_dof, 8)
    Ac = oop.assembled(constrained=True)
    xd = np.linalg.solve(Ac, np.where(om.dirichlet, 0.0, b))
    x, info = op.solve(to_dev(b), rtol=1e-12)
    assert info["status"] == 0
    assert rel_err(x.cpu().numpy(), xd) <= 1e-10
    xh = np.zeros(om.n_dof)
    info_h = hx.hx_solve_pcg_host(op.handle, np.ascontiguousarray(b), xh, 1e-12, 10000, False)
    assert info_h["iterations"] == info["iterations"]
    np.testing.assert_array_equal(xh, x.cpu().numpy())
    # warm start from the solution converges at once
    x2, info2 = op.solve(to_dev(b), x=x.clone(), rtol=1e-8)
    assert info2["iterations"] <= 1
    # new coefficients enqueued on the caller's stream, then a host-buffer solve:
    # the solve must see the updated factors and diagonal
    op.set_coefficients(10.0, 0.5)
    hx.hx_solve_pcg_host(op.handle, np.ascontiguousarray(b), xh, 1e-12, 10000, False)
    A2 = fem.Operator(om, 10.0, 0.5).assembled(constrained=True)
    assert rel_err(xh, np.linalg.solve(A2, np.where(om.dirichlet, 0.0, b))) <= 1e-10


def test_solver_status_codes(hx):
    p, shape = 2, (3, 3, 3)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    b = to_dev(S.random_vector(om.n_dof, 2))
    x, info = op.solve(b, rtol=1e-14, max_it=3, raise_on_fail=False)
    assert info["status"] == hx.HX_ERR_NOT_CONVERGED and info["iterations"] == 3
    with pytest.raises(hx.HxError) as ei:
        op.solve(b, rtol=1e-14, max_it=3)
    assert ei.value.status == hx.HX_ERR_NOT_CONVERGED
    bn = b.clone()
    bn[om.n_dof // 2] = float("nan")
    x, info = op.solve(bn, raise_on_fail=False)
    assert info["status"] == hx.HX_ERR_BREAKDOWN
    # zero right-hand side: converged at once with x = 0
    x, info = op.solve(torch.zeros_like(b))
    assert info["iterations"] == 0 and not x.any()


def test_inverted_element_is_rejected(hx):
    shape = (2, 2, 2)
    V = S.structured_vertices(*shape, 0.0)
    V[13] = [0.9, 0.9, 0.9]  # centre vertex pushed past a corner: detJ < 0 somewhere
    mesh = hx.Mesh.structured(*shape, 2, 4, V)
    for geom in (0, 1):
        with pytest.raises(hx.HxError) as ei:
            hx.Operator(mesh, 1.0, 1.0, geom_mode=geom)
        assert ei.value.status == hx.HX_ERR_INVALID_MESH


def test_argument_errors(hx):
    V = S.structured_vertices(1, 1, 1, 0.0)
    with pytest.raises(hx.HxError) as ei:
        hx.Mesh.structured(1, 1, 1, 2, 7, V)
    assert ei.value.status == hx.HX_ERR_UNSUPPORTED
    with pytest.raises(hx.HxError) as ei:
        hx.Mesh.general(2, 4, V, S.structured_elem_vert(1, 1, 1), 27, np.full((1, 27), 99, np.int64))
    assert ei.value.status == hx.HX_ERR_ARG


def test_destroy_mesh_before_operator(hx):
    """Freeing the mesh first and the operator afterwards touches no freed memory."""
    V = S.structured_vertices(2, 2, 2, 0.1, 3)
    m = hx.hx_mesh_create_structured(2, 2, 2, 2, 4, V)
    op = hx.hx_op_create(m, 1.0, 1.0)
    hx.hx_mesh_destroy(m)
    hx.hx_op_destroy(op)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_unstructured_mesh(hx, p):
    """A mesh whose central edge has valence 5 (10 elements share its DoFs), numbering from node
    positions: both geometry modes vs the oracle, constrained and not, and a Jacobi-PCG solve."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    from tests.unstructured import star_prism
    V, EV, om = star_prism(p)
    mesh = hx.Mesh.general(p, p + 2, V, EV, om.n_dof, om.restriction.astype(np.int32),
                           om.dirichlet.astype(np.uint8))
    oop = fem.Operator(om, 1.3, 0.7)
    x = S.random_vector(om.n_dof, 81)
    for gm in (hx.HX_GEOM_STORED, hx.HX_GEOM_ONTHEFLY):
        op = hx.Operator(mesh, 1.3, 0.7, geom_mode=gm)
        for constrained in (False, True):
            _assert_close(op.apply(to_dev(x), constrained=constrained).cpu().numpy(),
                          oop.apply(x, constrained=constrained))
    b = S.random_vector(om.n_dof, 82)
    u, info = op.solve(to_dev(b), rtol=1e-10)
    assert info["status"] == 0 and info["true_rel_residual"] <= 1.01e-10
    assert rel_err(u.cpu().numpy(), jacobi_pcg(oop, b, 1e-12)[0]) <= 1e-8


@pytest.mark.parametrize("p", [2, 5])
def test_coefficient_updates_rescale_and_recompute(hx, p):
    """New constant coefficients (both nonzero) rescale the stored factors in place and combine
    the diagonal from its mass and stiffness parts; a zero coefficient, a nu field or more than
    64 updates in a row recompute them.  Every state matches the oracle of its coefficients."""
    from oracle import fem
    shape = (3, 2, 4)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 3.0, 0.25)
    x = S.random_vector(om.n_dof, 77)
    for step, (alpha, nu) in enumerate([(7.0, 0.5), (0.0, 2.0), (5.0, 2.0), (5.0, 0.125)] + [(1.5, 0.75)] * 66):
        op.set_coefficients(alpha, nu)
        if step < 4 or step in (66, 67, 69):  # before, at and after the recomputation cap
            oop = fem.Operator(om, alpha, nu)
            for constrained in (False, True):
                _assert_close(op.apply(to_dev(x), constrained=constrained).cpu().numpy(),
                              oop.apply(x, constrained=constrained))
                _assert_close(op.diagonal(constrained).cpu().numpy(), oop.diagonal(constrained))
    # a nu field replaces the constant, and a constant afterwards recomputes the factors
    mesh = op.mesh
    nu_q = torch.full((mesh.n_elem, (p + 2) ** 3), 0.3, dtype=torch.float64, device="cuda")
    op.set_coefficients(2.0, 0.0, nu_q=nu_q)
    _assert_close(op.apply(to_dev(x)).cpu().numpy(), fem.Operator(om, 2.0, 0.3).apply(x))
    op.set_coefficients(4.0, 0.6)
    _assert_close(op.diagonal(True).cpu().numpy(), fem.Operator(om, 4.0, 0.6).diagonal(True))
