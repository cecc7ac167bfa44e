"""hx_apply_noalloc: the operator apply for callers that cannot allocate device memory.

Such callers (code inside a framework whose pool allocator owns all device
memory, services with a device memory budget fixed at start-up, latency-bound
loops that cannot pay for the synchronization of cudaMalloc / cudaFree) pass
every array in; the library uses a fixed scratch array in static device
memory.  The entry point must give the same result as the allocating path,
hx_op_apply on an on-the-fly operator, call after call: the scratch keeps the
previous call's contents, so two calls in a row with different inputs are
checked, and the device's free memory must not change across a call.

This file is named to be collected last: a failure here leaves every other
test already run.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from tests.gpu_common import rel_err, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 operator tolerance of the parity tests


def _inputs(shape, p):
    """Caller-side arrays: corner coordinates, restriction and its transpose (built on the host)."""
    nx, ny, nz = shape
    n = p + 1
    V = S.structured_vertices(nx, ny, nz, 0.1, 1910)
    EV = S.structured_elem_vert(nx, ny, nz)
    gx, gy = p * nx + 1, p * ny + 1
    e = np.arange(nx * ny * nz)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    l = np.arange(n ** 3)
    i, j, k = l % n, (l // n) % n, l // (n * n)
    R = (p * ex[:, None] + i) + gx * ((p * ey[:, None] + j) + gy * (p * ez[:, None] + k))
    n_dof = gx * gy * (p * nz + 1)
    order = np.argsort(R.ravel(), kind="stable")           # positions, increasing within each DoF
    off = np.concatenate([[0], np.cumsum(np.bincount(R.ravel(), minlength=n_dof))])
    X8 = V[EV].reshape(-1, 24)
    dev_i = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device="cuda")
    return V, n_dof, to_dev(X8), dev_i(R), dev_i(off), dev_i(order)


@pytest.mark.parametrize("p,dq,shape", [(3, 2, (5, 4, 3)), (4, 1, (3, 3, 2)), (8, 2, (2, 2, 1))])
def test_noalloc_apply_matches_allocating_apply_twice(p, dq, shape):
    hx = require_gpu()
    q = p + dq
    V, n_dof, X8, R, off, idx = _inputs(shape, p)
    alpha, nu = 2.5, 0.3
    op = hx.Operator(hx.Mesh.structured(*shape, p, q, V), alpha, nu, geom_mode=hx.HX_GEOM_ONTHEFLY)
    # one call first: the first use of the library's kernels in a process loads their code and
    # the static scratch array onto the device (module loading, not an allocation by the call)
    hx.hx_apply_noalloc(p, q, X8, R, off, idx, alpha, nu, to_dev(S.random_vector(n_dof, 10)),
                        torch.empty(n_dof, dtype=torch.float64, device="cuda"))
    for seed in (11, 12):  # two calls in a row, the second over the first call's scratch contents
        x = to_dev(S.random_vector(n_dof, seed))
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        hx.hx_apply_noalloc(p, q, X8, R, off, idx, alpha, nu, x, y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0  # nothing allocated on the device
        ref = op.apply(x, constrained=False)
        torch.cuda.synchronize()
        yn, rn = y.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(yn).all()
        assert rel_err(yn, rn) <= TOL
        np.testing.assert_allclose(yn, rn, rtol=0, atol=TOL * np.abs(rn).max())


def test_noalloc_rejects_sizes_beyond_the_scratch():
    hx = require_gpu()
    p = 4
    n_elem = hx.HX_NOALLOC_MAX_EVEC // (p + 1) ** 3 + 1
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = hx._lib.hx_apply_noalloc(p, p + 2, n_elem, 1000, dummy, dummy, dummy, dummy, 1.0, 1.0, dummy,
                                  ctypes.c_void_p(32), None)
    assert st == hx.HX_ERR_UNSUPPORTED
    assert "exceeds the static scratch" in hx.hx_last_error()
