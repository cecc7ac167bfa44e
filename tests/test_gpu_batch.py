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
    # all concurrent, one chain, chains of several solves, lock-step iterations (-2) and
    # autotuned (-1: timed at the first solve over 1, 2, 4 and 6 lanes and the lock-step mode;
    # the results cannot depend on the choice)
    for lanes in (0, 1, 2, 4, hx.HX_BATCH_FUSED, hx.HX_BATCH_AUTO):
        batch = hx.Batch(ops, bs, xs, rtol=1e-10, lanes=lanes)
        assert batch.lanes == (lanes if lanes == hx.HX_BATCH_FUSED else len(ops) if lanes <= 0 else lanes)
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
            if lanes == hx.HX_BATCH_AUTO:
                assert batch.lanes in (1, 2, 4, len(ops), hx.HX_BATCH_FUSED)
        del batch


def test_fused_batch_with_mixed_preconditioners_and_failures():
    """Lock-step mode beside LOR-preconditioned branches; an instance that fails its cap stops
    alone while the others finish; the loop ends when every instance is done."""
    hx = require_gpu()
    specs = [(3, 2, 1.0, 1.0, hx.HX_PREC_JACOBI, 10000), (2, 4, 0.0, 1.0, hx.HX_PREC_LOR_MG, 10000),
             (4, 3, 5.0, 0.1, hx.HX_PREC_COLLOCATED_MASS, 10000), (2, 6, 1.0, 1.0, hx.HX_PREC_JACOBI, 10000)]
    ops, bs, xs, refs = [], [], [], []
    for k, (N, p, a, nu, prec, _) in enumerate(specs):
        V = S.structured_vertices(N, N, N, 0.1, 300 + k)
        op = hx.Operator(hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=63), a, nu)
        op.set_preconditioner(prec, 1)
        b = to_dev(S.random_vector(op.n_dof, 400 + k))
        refs.append(op.solve(b, rtol=1e-10))
        ops.append(op)
        bs.append(b)
        xs.append(torch.full_like(b, float("nan")))
    batch = hx.Batch(ops, bs, xs, rtol=1e-10, lanes=hx.HX_BATCH_FUSED)
    infos = batch.solve()
    for (xr, ir), x, i in zip(refs, xs, infos):
        assert i["status"] == 0 and i["iterations"] == ir["iterations"]
        assert torch.equal(x, xr)
    # a cap of 3 iterations: every instance stops with NOT_CONVERGED after 3 iterations
    capped = hx.Batch(ops, bs, xs, rtol=1e-10, max_it=3, lanes=hx.HX_BATCH_FUSED)
    infos = capped.solve(raise_on_fail=False)
    assert all(i["status"] == hx.HX_ERR_NOT_CONVERGED and i["iterations"] == 3 for i in infos)


def test_batch_reports_failures():
    hx = require_gpu()
    V = S.structured_vertices(3, 3, 3, 0.1, 9)
    op = hx.Operator(hx.Mesh.structured(3, 3, 3, 2, 4, V), 1.0, 1.0)
    b = to_dev(S.random_vector(op.n_dof, 1))
    x = torch.zeros_like(b)
    batch = hx.Batch([op], [b], [x], rtol=1e-14, max_it=2)
    infos = batch.solve(raise_on_fail=False)
    assert infos[0]["status"] == hx.HX_ERR_NOT_CONVERGED and infos[0]["iterations"] == 2
