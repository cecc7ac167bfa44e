"""Failure detection without a GPU fault.

For p <= 4 with stored factors the collocated FP32 operator kernel stages each block's
factors into shared memory with one bulk (TMA) copy, and the B/D-direct kernel with staged
factors copies each block's restriction and factors that way; both wait for the copies with
a bounded number of mbarrier try_wait attempts.  Here that bound is set to 0 (hx_op_set_wait_limit), so
every block's first wait gives up at once while the copies themselves complete
normally: each block raises the operator's error flag, skips its remaining stages,
and waits for its copy (with the far larger exit bound) before it exits.  The mixed
solve must report HX_ERR_CUDA; with the default bound restored, the next solves on
the same operator and device must run normally and match the oracle.
"""
import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import case, rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

DEFAULT_WAIT_LIMIT = 1 << 16


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("kind", [0, 1])  # collocated (staged for p <= 4), B/D-direct staged
def test_bounded_wait_gives_up_as_a_status(p, kind):
    from oracle import fem
    from oracle.solve import jacobi_pcg
    hx = require_gpu()
    shape = (4, 4, 3)
    V, EV, om = case(shape, p)
    op = hx.Operator(hx.Mesh.structured(*shape, p, p + 2, V), 1.0, 1.0)
    op.set_f32_kernel(kind)
    b = S.random_vector(om.n_dof, 21)
    bd = to_dev(b)
    x0, info0 = op.solve_mixed(bd, rtol=1e-10)
    assert info0["status"] == 0

    op.set_wait_limit(0)
    with pytest.raises(hx.HxError) as ei:
        op.solve_mixed(bd, rtol=1e-10, max_it=40)
    assert ei.value.status == hx.HX_ERR_CUDA and "timed out" in str(ei.value)

    op.set_wait_limit(DEFAULT_WAIT_LIMIT)
    x1, info1 = op.solve_mixed(bd, rtol=1e-10)
    assert info1["status"] == 0 and info1["rel_residual"] <= 1e-10
    assert torch.equal(x1, x0)  # the same arithmetic as before the failure
    xo, _, _, conv = jacobi_pcg(fem.Operator(om, 1.0, 1.0), b, 1e-12)
    assert conv and rel_err(x1.cpu().numpy(), xo) <= 1e-8
    # the FP64 path on the same device is unaffected
    x2, info2 = op.solve(bd, rtol=1e-10)
    assert info2["status"] == 0 and rel_err(x2.cpu().numpy(), xo) <= 1e-8


def test_wait_limit_rejects_negative():
    hx = require_gpu()
    V = S.structured_vertices(2, 2, 2, 0.1, 3)
    op = hx.Operator(hx.Mesh.structured(2, 2, 2, 3, 5, V), 1.0, 1.0)
    with pytest.raises(hx.HxError) as ei:
        op.set_wait_limit(-1)
    assert ei.value.status == hx.HX_ERR_ARG
