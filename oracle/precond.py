"""Oracle for the preconditioners of Sec. 5.1 and Sec. 5.2 (test infrastructure only).

Collocated mass (Sec. 5.1): integrating the mass form with the Gauss-Lobatto rule
at the nodes of the nodal basis makes it diagonal,
    Mc_ii = sum over elements K and local nodes l of K with global id i of
            w_a w_b w_c detJ_K(xi_l),   l = (a, b, c),
where w are the Gauss-Lobatto weights w_j = 2 / (p (p+1) P_p(x_j)^2).

Low-order refined operator (Sec. 5.2): A_LOR = c M_LOR + nu K_LOR is the
standard Q1 discretization on the mesh obtained by cutting every element along
the Cartesian product of its Gauss-Lobatto points.  The DoFs are shared with the
high-order space (the identity maps one to the other).  Each sub-element is the
image of a box of the reference cube under the element's trilinear map.  That
image is itself trilinear in the sub-element's local coordinates, with the
mapped Gauss-Lobatto nodes as corners.  So the LOR mesh is a p = 1 mesh on the
mapped nodes, and its operator is the ``fem.Operator`` of that mesh.  For
"standard" quadrature we read 2 Gauss points per direction, which integrates
the Q1 mass exactly on affine sub-elements.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import gll_nodes, legendre
from .fem import Mesh, Operator, trilinear_map


def gll_weights(p: int) -> np.ndarray:
    """Gauss-Lobatto weights of the p+1 nodes: 2 / (p (p+1) P_p(x_j)^2)."""
    x = gll_nodes(p)
    P, _ = legendre(p, x)
    return 2.0 / (p * (p + 1) * P * P)


def collocated_mass_element(mesh: Mesh, elems=None) -> np.ndarray:
    """(e, (p+1)^3) element diagonals w_a w_b w_c detJ at the local nodes (node index a + n b + n^2 c)."""
    p, n = mesh.p, mesh.p + 1
    w = gll_weights(p)
    es = np.arange(mesh.n_elem) if elems is None else np.asarray(elems)
    _, J = trilinear_map(mesh.vertices[mesh.elem_vert[es]], mesh.ref.node_xi)
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    w3 = (w[a] * w[b] * w[c]).ravel()
    return w3[None, :] * np.linalg.det(J)


def collocated_mass_diagonal(mesh: Mesh, alpha: float = 1.0) -> np.ndarray:
    """alpha Mc as an n_dof vector (unconstrained: Dirichlet rows keep their value)."""
    d = np.zeros(mesh.n_dof)
    np.add.at(d, mesh.restriction, alpha * collocated_mass_element(mesh))
    return d


def lor_mesh(mesh: Mesh) -> Mesh:
    """The p = 1, q = 2 mesh of the Gauss-Lobatto refined sub-elements (same DoFs and Dirichlet mask).

    Sub-element (s, t, u) of element K has corners at local nodes (s + dx, t + dy, u + dz),
    corner index dx + 2 dy + 4 dz; sub-elements are numbered K p^3 + s + p t + p^2 u.
    """
    p, n = mesh.p, mesh.p + 1
    R = mesh.restriction                                        # (E, n^3)
    u, t, s = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    s, t, u = s.ravel(), t.ravel(), u.ravel()                   # sub-element order s fastest
    corners = []
    for c in range(8):
        dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        corners.append((s + dx) + n * (t + dy) + n * n * (u + dz))
    L = np.stack(corners, axis=1)                               # (p^3, 8) local node ids
    sub = R[:, L].reshape(-1, 8)                                # (E p^3, 8) global ids
    X = mesh.node_coords()
    return Mesh(1, 2, X, sub, sub, mesh.n_dof, mesh.dirichlet)


def lor_operator(mesh: Mesh, alpha: float, nu: float) -> Operator:
    """A_LOR = alpha M_LOR + nu K_LOR (Sec. 5.2) as the oracle operator of the refined p = 1 mesh."""
    return Operator(lor_mesh(mesh), alpha, nu)


def lor_matrix(mesh: Mesh, alpha: float, nu: float, mass: str = "consistent", constrained: bool = True):
    """Dense A_LOR.  mass = "consistent": alpha M_LOR + nu K_LOR (Sec. 5.2 as written);
    mass = "collocated": alpha Mc + nu K_LOR, the LOR stiffness with the collocated
    Gauss-Lobatto mass of Sec. 5.1 (diagonal) in place of the Q1 mass."""
    if mass == "consistent":
        return lor_operator(mesh, alpha, nu).assembled(constrained=constrained)
    if mass != "collocated":
        raise ValueError(mass)
    A = lor_operator(mesh, 0.0, nu).assembled(constrained=False)
    A[np.diag_indices_from(A)] += collocated_mass_diagonal(mesh, alpha)
    if constrained:
        d = mesh.dirichlet
        A[d, :] = 0.0
        A[:, d] = 0.0
        A[d, d] = 1.0
    return A


def gershgorin_bound(A) -> float:
    """max_i sum_j |a_ij| / a_ii: an upper bound of the spectrum of D^-1 A (D = diag A)."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.max(np.abs(A).sum(axis=1) / np.diag(A)))


def chebyshev_apply(A, r, degree: int) -> np.ndarray:
    """z after `degree` steps of the Chebyshev iteration for A z = r with Jacobi scaling, z_0 = 0.

    The iteration follows Saad, Iterative Methods for Sparse Linear Systems (2nd ed.), Sec. 12.3
    (Algorithm 12.1) on the system D^-1 A z = D^-1 r over the interval [b / k^2, b], b the
    Gershgorin bound of D^-1 A and k the degree:
      theta = (b + a) / 2, delta = (b - a) / 2, sigma = theta / delta, rho_0 = 1 / sigma,
      res_0 = D^-1 r, d_0 = res_0 / theta, z_1 = d_0, and for j = 1 .. k-1:
      res_j = res_{j-1} - D^-1 A d_{j-1},  rho_j = 1 / (2 sigma - rho_{j-1}),
      d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) res_j,  z_{j+1} = z_j + d_j.
    """
    A = np.asarray(A, dtype=np.float64)
    dinv = 1.0 / np.diag(A)
    b = gershgorin_bound(A)
    a = b / degree ** 2
    theta, delta = (b + a) / 2, (b - a) / 2
    res = dinv * r
    d = res / theta
    z = d.copy()
    if degree < 2:
        return z
    sigma = theta / delta
    rho = 1.0 / sigma
    for _ in range(1, degree):
        res = res - dinv * (A @ d)
        rn = 1.0 / (2 * sigma - rho)
        d = rn * rho * d + (2 * rn / delta) * res
        z = z + d
        rho = rn
    return z


# --------------------------------------------------------------------------
# geometric multigrid V-cycle on the LOR matrix of a structured mesh (the paper solves
# A_LOR with a structured geometric multigrid V-cycle, Sec. 5.2; here the smoother is a
# Chebyshev-Jacobi polynomial instead of ordered ILU, and the coarse operators are Galerkin
# products of the logical-grid trilinear interpolation)
# --------------------------------------------------------------------------
MG_SMOOTH_DEGREE = 3      # Chebyshev steps of each pre- and post-smoothing
MG_SMOOTH_RATIO = 10.0    # smoothing interval [b / 10, b]
MG_COARSE_DEGREE = 16     # Chebyshev steps on the coarsest grid, interval [b / 16^2, b]
MG_MIN_DIM = 5            # a grid is coarsened while every dimension is odd and >= 5
MG_MAX_LEVELS = 16


def chebyshev_ratio_apply(A, r, degree: int, ratio: float) -> np.ndarray:
    """`degree` Chebyshev-Jacobi steps for A z = r from z = 0 on [b / ratio, b] (b the Gershgorin
    bound); the recurrence of ``chebyshev_apply``."""
    A = np.asarray(A, dtype=np.float64)
    dinv = 1.0 / np.diag(A)
    b = gershgorin_bound(A)
    a = b / ratio
    theta, delta = (b + a) / 2, (b - a) / 2
    res = dinv * r
    d = res / theta
    z = d.copy()
    if degree < 2:
        return z
    sigma = theta / delta
    rho = 1.0 / sigma
    for _ in range(1, degree):
        res = res - dinv * (A @ d)
        rn = 1.0 / (2 * sigma - rho)
        d = rn * rho * d + (2 * rn / delta) * res
        z = z + d
        rho = rn
    return z


def interpolation(dims, dirichlet):
    """Trilinear interpolation P (n_fine x n_coarse) from the vertex-centred coarse grid (every other
    node, dims (m + 1) / 2) of a logical grid with odd dims, lexicographic order (x fastest).
    Rows of Dirichlet fine nodes and columns of Dirichlet coarse nodes are zero.
    Returns (P, coarse dims, coarse Dirichlet mask)."""
    mx, my, mz = dims
    cx, cy, cz = (mx + 1) // 2, (my + 1) // 2, (mz + 1) // 2
    nf = mx * my * mz
    gi = np.arange(nf)
    ix, iy, iz = gi % mx, (gi // mx) % my, gi // (mx * my)
    cdir = dirichlet.reshape(mz, my, mx)[::2, ::2, ::2].ravel()
    rows, cols, vals = [], [], []
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                # coarse index along each axis: i / 2 for even i (once), (i -+ 1) / 2 for odd i
                Jx = np.where(ix % 2 == 0, ix // 2, (ix - 1) // 2 + ox)
                Jy = np.where(iy % 2 == 0, iy // 2, (iy - 1) // 2 + oy)
                Jz = np.where(iz % 2 == 0, iz // 2, (iz - 1) // 2 + oz)
                w = (np.where(ix % 2 == 0, 1.0 - ox, 0.5) * np.where(iy % 2 == 0, 1.0 - oy, 0.5) *
                     np.where(iz % 2 == 0, 1.0 - oz, 0.5))
                J = Jx + cx * (Jy + cy * Jz)
                keep = (w > 0) & ~dirichlet
                keep[keep] &= ~cdir[J[keep]]
                rows.append(gi[keep])
                cols.append(J[keep])
                vals.append(w[keep])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nf, cx * cy * cz))
    return P, (cx, cy, cz), cdir


def mg_hierarchy(A, dims, dirichlet):
    """[(A_l, P_l)] from the fine matrix down: A_{l+1} = P_l^T A_l P_l with identity rows at the
    Dirichlet coarse nodes; the last entry has P = None (the coarsest grid)."""
    levels = []
    A = np.asarray(A, dtype=np.float64)
    dims = tuple(int(d) for d in dims)
    dirichlet = np.asarray(dirichlet, dtype=bool)
    while (len(levels) < MG_MAX_LEVELS - 1 and all(d % 2 == 1 and d >= MG_MIN_DIM for d in dims)):
        P, cdims, cdir = interpolation(dims, dirichlet)
        Ac = np.asarray((P.T @ sp.csr_matrix(A) @ P).todense())
        Ac[cdir, :] = 0.0
        Ac[:, cdir] = 0.0
        Ac[cdir, cdir] = 1.0
        levels.append((A, P))
        A, dims, dirichlet = Ac, cdims, cdir
    levels.append((A, None))
    return levels


def vcycle(levels, b, level=0, smooth_degree=MG_SMOOTH_DEGREE):
    """One symmetric V-cycle for A_0 x = b from x = 0: Chebyshev pre-smoothing, residual,
    restriction P^T, the V-cycle of the next grid, prolongation P, residual and Chebyshev
    post-smoothing (the same polynomial, so the cycle is a symmetric linear operator);
    Chebyshev with MG_COARSE_DEGREE steps on the coarsest grid."""
    A, P = levels[level]
    if P is None:
        return chebyshev_ratio_apply(A, b, MG_COARSE_DEGREE, float(MG_COARSE_DEGREE ** 2))
    x = chebyshev_ratio_apply(A, b, smooth_degree, MG_SMOOTH_RATIO)
    x = x + P @ vcycle(levels, P.T @ (b - A @ x), level + 1, smooth_degree)
    return x + chebyshev_ratio_apply(A, b - A @ x, smooth_degree, MG_SMOOTH_RATIO)
