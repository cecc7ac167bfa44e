"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds only input generation: a counter-based random number
generator, structured hexahedral meshes of the unit cube with randomly
perturbed interior vertices, and random vectors.  It contains none of the
finite element arithmetic (no basis, no quadrature, no operator, no DoF
numbering); those live separately in ``oracle/`` (CPU reference) and in the
CUDA library.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter form: output ``i`` of stream
``seed`` is ``mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)``.  A double in
[-1, 1) is ``((x >> 11) * 2**-53) * 2 - 1``.

Mesh recipe (the paper's 3D benchmarks use Cartesian hexahedral meshes; the
trilinear, perturbed variant exercises non-affine geometry):
  * vertices of an ``nx x ny x nz`` grid on [0,1]^3, ordered lexicographically
    with x fastest, components (x, y, z);
  * every interior vertex coordinate is moved by ``frac * h_d * U[-1,1)``,
    drawn from stream ``seed`` at counter ``3 * vertex_index + component``;
  * elements are ordered lexicographically (x fastest); the 8 corners of an
    element are ordered lexicographically too: corner ``c = cx + 2*cy + 4*cz``.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_MESH_SEED = 1910
DEFAULT_VECTOR_SEED = 3032


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles uniform in [-1, 1) from SplitMix64 stream ``seed``."""
    x = splitmix64(seed, count, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def random_vector(n: int, seed: int = DEFAULT_VECTOR_SEED) -> np.ndarray:
    """A length-``n`` vector of U[-1,1) doubles."""
    return uniform_pm1(seed, n)


def structured_vertices(nx: int, ny: int, nz: int, perturb_frac: float = 0.1,
                        seed: int = DEFAULT_MESH_SEED) -> np.ndarray:
    """Vertex coordinates ``((nx+1)(ny+1)(nz+1), 3)`` of a perturbed grid on [0,1]^3.

    Boundary vertices stay on the faces of the cube, so the domain is the unit
    cube exactly; interior vertices move by up to ``perturb_frac`` of the local
    spacing in each coordinate independently.
    """
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    zs = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    v = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if perturb_frac != 0.0:
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        r = uniform_pm1(seed, v.shape[0] * 3).reshape(-1, 3)
        kz, ky, kx = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        interior = ((kx > 0) & (kx < nx) & (ky > 0) & (ky < ny) & (kz > 0) & (kz < nz)).ravel()
        v[interior] += perturb_frac * h[None, :] * r[interior]
    return v


def structured_elem_vert(nx: int, ny: int, nz: int) -> np.ndarray:
    """Element-to-vertex table ``(nx*ny*nz, 8)`` (int64) for the grid of ``structured_vertices``."""
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ex, ey, ez = ex.transpose(2, 1, 0).ravel(), ey.transpose(2, 1, 0).ravel(), ez.transpose(2, 1, 0).ravel()
    sx, sy = nx + 1, (nx + 1) * (ny + 1)
    out = np.empty((ex.size, 8), dtype=np.int64)
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        out[:, c] = (ex + cx) + (ey + cy) * sx + (ez + cz) * sy
    return out


def affine_map(vertices: np.ndarray, A: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """Apply ``x -> A x + b`` to every vertex (builds sheared / stretched affine meshes)."""
    out = vertices @ np.asarray(A, dtype=np.float64).T
    if b is not None:
        out = out + np.asarray(b, dtype=np.float64)[None, :]
    return out


def permutation(n: int, seed: int) -> np.ndarray:
    """A seeded random permutation of ``0..n-1`` (argsort of SplitMix64 outputs)."""
    return np.argsort(splitmix64(seed, n), kind="stable")
