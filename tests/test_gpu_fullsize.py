"""Full-size meshes of the FP64 scaling sweep (the launch configuration the benchmark times):
sampled entries vs the oracle computed row by row, plus a size-independent property."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, require_gpu, to_dev, torch

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
