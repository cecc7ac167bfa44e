"""Batched solves: independent instances of different order, size and coefficients (and a
pure-Neumann Poisson instance) in one graph launch.  Each instance must match the oracle's
Jacobi-PCG solution of the same mesh (its null-space variant for the pure-Neumann Poisson,
Sec. 5.3) and equal, bit for bit, its own one-by-one FP64 solve."""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

SPECS = [  # (N, p, alpha, nu, dirichlet faces: 63 = all six, 0 = none)
    (3, 2, 1000.0, 1e-2, 63), (2, 5, 0.0, 1.0, 63), (4, 3, 50.0, 3e-3, 63),
    (2, 8, 1.0, 0.5, 63), (3, 4, 0.0, 1.0, 0), (5, 2, 1e4, 1e-4, 63),
]


def oracle_solution(N, p, alpha, nu, faces, seed, b):
    """The oracle's PCG solution of one instance, to a tighter 1e-12 so that its own
    stopping error stays far below the 1e-8 solution tolerance."""
    from oracle import fem
    from oracle.solve import jacobi_pcg, jacobi_pcg_nullspace
    _, _, om = case((N, N, N), p, seed=seed, dirichlet=faces == 63)
    op = fem.Operator(om, alpha, nu)
    if faces == 0:
        x, _, _, conv = jacobi_pcg_nullspace(op, b, 1e-12, 20000)
    else:
        x, _, _, conv = jacobi_pcg(op, b, 1e-12, 20000)
    assert conv
    return x


def test_batch_matches_oracle_and_individual_solves():
    hx = require_gpu()
    ops, bs, xs, refs, oracle = [], [], [], [], []
    for k, (N, p, a, nu, faces) in enumerate(SPECS):
        V = S.structured_vertices(N, N, N, 0.1, 100 + k)
        mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=faces)
        op = hx.Operator(mesh, a, nu)
        bh = S.random_vector(mesh.n_dof, 200 + k)
        b = to_dev(bh)
        x_ref, info = op.solve(b, rtol=1e-10)
        assert info["status"] == 0
        ops.append(op)
        bs.append(b)
        xs.append(torch.full_like(b, float("nan")))
        refs.append((x_ref, info))
        oracle.append(oracle_solution(N, p, a, nu, faces, 100 + k, bh))
    # all concurrent, one chain, chains of several solves, and autotuned (-1: timed at the
    # first solve over 1, 2, 4 and 6 lanes; the results cannot depend on the choice)
    for lanes in (0, 1, 2, 4, -1):
        batch = hx.Batch(ops, bs, xs, rtol=1e-10, lanes=lanes)
        assert batch.lanes == (len(ops) if lanes <= 0 else lanes)
        for rep in range(2):  # the bound graph is reusable
            for x in xs:
                x.fill_(float("nan"))
            infos = batch.solve()
            for (x_ref, info), x, bi, xo in zip(refs, xs, infos, oracle):
                assert bi["status"] == 0 and bi["iterations"] == info["iterations"]
                assert bi["true_rel_residual"] <= 1.01e-10
                xb = x.cpu().numpy()
                assert np.array_equal(xb, x_ref.cpu().numpy())
                assert rel_err(xb, xo) <= 1e-8
            if lanes < 0:
                assert batch.lanes in (1, 2, 4, len(ops))
        del batch


def test_batch_reports_failures():
    hx = require_gpu()
    V = S.structured_vertices(3, 3, 3, 0.1, 9)
    op = hx.Operator(hx.Mesh.structured(3, 3, 3, 2, 4, V), 1.0, 1.0)
    b = to_dev(S.random_vector(op.n_dof, 1))
    x = torch.zeros_like(b)
    batch = hx.Batch([op], [b], [x], rtol=1e-14, max_it=2)
    infos = batch.solve(raise_on_fail=False)
    assert infos[0]["status"] == hx.HX_ERR_NOT_CONVERGED and infos[0]["iterations"] == 2
