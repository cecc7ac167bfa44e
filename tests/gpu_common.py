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


def lor_row_oracle(om, g, alpha, nu):
    """Row g of the oracle's alpha Mc + nu K_LOR (constrained): only the elements holding DoF g
    contribute to it (its sub-elements and its collocated mass), so the oracle assembles that
    patch of elements alone. Returns (global columns, values) of the row's non-zeros."""
    from oracle import fem, precond
    els = sorted({e for e, _ in om.elements_of_dof(int(g))})
    R = np.stack([om.element_dofs(e) for e in els])
    ids, Rl = np.unique(R, return_inverse=True)
    sub = fem.Mesh(om.p, om.q, om.vertices, om.elem_vert[els], Rl.reshape(R.shape), len(ids), om.dirichlet[ids])
    row = precond.lor_matrix(sub, alpha, nu, "collocated")[np.searchsorted(ids, g)]
    nz = row != 0
    return ids[nz], row[nz]
