"""Mixed precision (FP64 iterative refinement around an FP32 Jacobi-PCG) vs the FP64 oracle.

Tolerances.  FP32 operator apply: relative 2e-5 in the 2-norm (FP32 unit
roundoff 6e-8 times the ~10^2 terms of each sum-factorized output, on inputs
rounded to FP32 before the oracle sees them).  Mixed solve: the FP64
residual it reports is recomputed in FP64, so the 1e-10 target is checked
exactly as for the FP64 solver; its solution must agree with the oracle's
FP64 solution to 1e-8 (both solved to 1e-10).
"""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, mms_exact, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    return require_gpu()


@pytest.mark.parametrize("p,shape", [(1, (5, 5, 3)), (2, (5, 5, 3)), (3, (5, 5, 3)), (4, (5, 3, 3)), (5, (4, 3, 2)),
                                     (6, (3, 3, 1)), (7, (2, 2, 2)), (8, (3, 3, 1))])
@pytest.mark.parametrize("geom,kind", [(0, -1), (0, 0), (0, 1), (0, 2), (1, -1), (1, 0), (1, 2)])
def test_fp32_apply_matches_oracle(hx, p, shape, geom, kind):
    """Every FP32 element kernel (collocated, B/D-direct with staged or loaded factors, and the
    autotuner's pick) on meshes spanning several blocks with a ragged last block."""
    from oracle import fem
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.7, 0.45, geom_mode=geom)
    op.set_f32_kernel(kind)
    x32 = S.random_vector(om.n_dof, 3032).astype(np.float32)
    y = op.apply_f32(torch.as_tensor(x32, device="cuda")).double().cpu().numpy()
    ref = fem.Operator(om, 1.7, 0.45).apply(x32.astype(np.float64), constrained=True)
    assert rel_err(y, ref) <= 2e-5, rel_err(y, ref)
    used, ne, ms = op.f32_kernel()
    assert used == kind if kind >= 0 else used in ((0, 1, 2) if geom == 0 else (0, 2))
    assert (ne in (1, 2, 4, 8)) if used in (1, 2) else ne == -1
    if kind < 0 and used >= 0 and ms[used] >= 0:  # tuned here (not taken from the process cache)
        assert ms[used] == min(m for m in ms if m >= 0)


@pytest.mark.parametrize("p,q,shape", [(1, 3, (5, 5, 3)), (2, 4, (5, 5, 3)), (3, 5, (5, 5, 3)), (4, 6, (5, 3, 3)),
                                       (4, 5, (3, 3, 3)), (5, 7, (4, 3, 2)), (6, 8, (3, 3, 1)), (8, 10, (3, 3, 1))])
@pytest.mark.parametrize("kind", [1, 2])
def test_fp32_direct_tiles_match_oracle(hx, p, q, shape, kind):
    """Every tile variant the autotuner may pick (half, default and twice the elements per block
    of the B/D-direct kernels), forced one by one, on meshes with a ragged last block; a variant
    the order does not have is refused."""
    from oracle import fem
    V, EV, om = case(shape, p, q=q)
    op = hx.Operator(hx.Mesh.structured(*shape, p, q, V), 1.7, 0.45)
    ref_op = fem.Operator(om, 1.7, 0.45)
    x32 = S.random_vector(om.n_dof, 3033).astype(np.float32)
    ref = ref_op.apply(x32.astype(np.float64), constrained=True)
    seen = []
    for tile in (-1, 0, 1):
        op.set_f32_kernel(kind)
        op.set_f32_tile(tile)
        default = 8 if 8 * q * q <= 256 else 4 if 4 * q * q <= 256 else 2
        ne = default // 2 if tile < 0 else default * 2 if tile > 0 else default
        if ne < 1 or ne > 8 or ((ne * q * q + 31) // 32) * 32 > 1024:
            with pytest.raises(hx.HxError) as ei:
                op.apply_f32(torch.as_tensor(x32, device="cuda"))
            assert ei.value.status == hx.HX_ERR_UNSUPPORTED
            continue
        try:
            y = op.apply_f32(torch.as_tensor(x32, device="cuda")).double().cpu().numpy()
        except hx.HxError as e:  # a variant whose shared memory exceeds a block's limit
            assert kind == 1 and tile > 0, e
            continue
        assert rel_err(y, ref) <= 2e-5, (tile, rel_err(y, ref))
        used, got_ne, _ = op.f32_kernel()
        assert used == kind and got_ne == ne
        seen.append(ne)
    assert default in seen
    with pytest.raises(hx.HxError):
        op.set_f32_tile(2)


@pytest.mark.parametrize("p,shape", [(1, (5, 5, 3)), (2, (5, 5, 3)), (3, (5, 5, 3)), (4, (5, 3, 3)), (5, (4, 3, 2)),
                                     (6, (3, 3, 1)), (7, (2, 2, 2)), (8, (3, 3, 1))])
@pytest.mark.parametrize("kind,tol", [(3, 3e-2), (4, 1e-4)])
def test_fp32_tensor_core_apply_matches_oracle(hx, p, shape, kind, tol):
    """The tensor-core kernels: BF16 operands (unit roundoff 2^-9 ~ 2e-3, six contraction stages
    with both operands rounded: 3e-2) and the hi/lo BF16 split (dropped lo*lo terms ~ 2^-18
    each, plus the tensor cores' FP32 accumulation: 1e-4)."""
    from oracle import fem
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.7, 0.45)
    op.set_f32_kernel(kind)
    x32 = S.random_vector(om.n_dof, 3032).astype(np.float32)
    y = op.apply_f32(torch.as_tensor(x32, device="cuda")).double().cpu().numpy()
    ref = fem.Operator(om, 1.7, 0.45).apply(x32.astype(np.float64), constrained=True)
    err = rel_err(y, ref)
    assert err <= tol, err
    assert op.f32_kernel()[0] == kind


@pytest.mark.parametrize("p", [2, 4, 8])
def test_mixed_solve_tensor_core_bf16x3(hx, p):
    """The mixed solve with the hi/lo BF16 tensor-core operator still reaches the FP64 1e-10."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    shape = (4, 4, 4) if p <= 4 else (3, 3, 3)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    op.set_f32_kernel(hx.HX_F32_MMA_BF16X3)
    b = to_dev(S.random_vector(om.n_dof, 5))
    x, info = op.solve_mixed(b, rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    uo, _, _, conv = jacobi_pcg(fem.Operator(om, 1.0, 1.0), b.cpu().numpy(), 1e-12)
    assert conv and rel_err(x.cpu().numpy(), uo) <= 1e-8


def test_fp32_kernel_selection_errors(hx):
    V = S.structured_vertices(2, 2, 2, 0.1, 5)
    mesh = hx.Mesh.structured(2, 2, 2, 3, 5, V)
    op = hx.Operator(mesh, 1.0, 1.0, geom_mode=hx.HX_GEOM_ONTHEFLY)
    with pytest.raises(hx.HxError) as ei:
        op.set_f32_kernel(hx.HX_F32_DIRECT_STAGED)
    assert ei.value.status == hx.HX_ERR_UNSUPPORTED
    for kind in (hx.HX_F32_MMA_BF16, hx.HX_F32_MMA_BF16X3):
        with pytest.raises(hx.HxError) as ei:
            op.set_f32_kernel(kind)
        assert ei.value.status == hx.HX_ERR_UNSUPPORTED
    with pytest.raises(hx.HxError) as ei:
        op.set_f32_kernel(7)
    assert ei.value.status == hx.HX_ERR_ARG
    assert op.f32_kernel()[0] == -1  # nothing chosen before the first FP32 set-up


@pytest.mark.parametrize("p", [3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("geom", [0, 1])
@pytest.mark.parametrize("kind", [-1, 0, 2])
def test_mixed_solve_reaches_fp64_tolerance(hx, p, geom, kind):
    """4^3 perturbed mesh, alpha = nu = 1, manufactured right-hand side (the small config at p = 4..8)."""
    from oracle import fem
    from oracle.solve import jacobi_pcg
    shape = (4, 4, 4) if p <= 5 else (3, 3, 3)
    V, EV, om = case(shape, p)
    mesh = hx.Mesh.structured(*shape, p, p + 2, V)
    op = hx.Operator(mesh, 1.0, 1.0, geom_mode=geom)
    op.set_f32_kernel(kind if (kind != 2 or geom == 1) else 1)  # stored: the staged direct kernel
    f = (1.0 + 3 * np.pi ** 2) * mms_exact(mesh.qpoint_coords().cpu().numpy())
    b = op.load_vector(to_dev(f))
    x, info = op.solve_mixed(b, rtol=1e-10, inner_rtol=1e-5)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    assert 1 <= info["refinements"] <= 6
    # the residual it reports is the FP64 one: recompute it independently
    r = torch.where(torch.as_tensor(om.dirichlet, device="cuda"), torch.zeros_like(b), b) - op.apply(x, constrained=True)
    bn = torch.linalg.norm(torch.where(torch.as_tensor(om.dirichlet, device="cuda"), torch.zeros_like(b), b))
    assert float(torch.linalg.norm(r) / bn) <= 1.01e-10
    uo, its, rel, conv = jacobi_pcg(fem.Operator(om, 1.0, 1.0), b.cpu().numpy(), 1e-10)
    assert rel_err(x.cpu().numpy(), uo) <= 1e-8


@pytest.mark.parametrize("geom", [0, 1])
def test_mixed_solve_helmholtz_time_step(hx, geom):
    """alpha = 1/dt = 1000, nu = 1e-2 (the sweep's coefficients) on an 8^3 Q_4 mesh, random RHS."""
    p, shape = 4, (8, 8, 8)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1000.0, 1e-2, geom_mode=geom)
    b = to_dev(S.random_vector(om.n_dof, 77))
    x64, i64 = op.solve(b, rtol=1e-10)
    x, info = op.solve_mixed(b, rtol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    assert rel_err(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-8
    # a second solve after new coefficients refreshes the FP32 factors
    op.set_coefficients(10.0, 0.5)
    x2, info2 = op.solve_mixed(b, rtol=1e-10)
    x2_64, _ = op.solve(b, rtol=1e-10)
    assert info2["status"] == 0 and rel_err(x2.cpu().numpy(), x2_64.cpu().numpy()) <= 1e-8


def test_mixed_solve_status(hx):
    p, shape = 2, (3, 3, 3)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    b = to_dev(S.random_vector(om.n_dof, 2))
    x, info = op.solve_mixed(b, rtol=1e-10, max_it=2, raise_on_fail=False)
    assert info["status"] == hx.HX_ERR_NOT_CONVERGED
    x, info = op.solve_mixed(torch.zeros_like(b))
    assert info["status"] == 0 and info["refinements"] == 0 and not x.any()
