"""Shared set-up for the GPU parity tests: the same seeded mesh for the CUDA path and the oracle."""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    import paper_1910_03032_b300 as hx  # raises ImportError when libhx.so is missing
    return hx


def mms_exact(X):
    return np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])


def case(shape, p, q=None, perturb=0.1, seed=1910, lazy=False, dirichlet=True):
    """(vertices, elem_vert, oracle StructuredMesh) for an nx x ny x nz perturbed grid."""
    from oracle import fem
    q = p + 2 if q is None else q
    V = S.structured_vertices(*shape, perturb, seed)
    EV = S.structured_elem_vert(*shape)
    om = fem.StructuredMesh(*shape, p, q, V, EV, dirichlet_boundary=dirichlet, lazy=lazy)
    return V, EV, om


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
