"""Oracle finite element operator: explicit element matrices, element-sum assembly.

Everything here follows the definitions of the paper's Section 3 written out
directly (no sum factorization, no blocking):

  * basis phi_ijk(xi) = phi_i(xi_1) phi_j(xi_2) phi_k(xi_3) on the Gauss-Lobatto
    points, 0 <= i,j,k <= p, built as full 3D products (Sec. 3.1);
  * tensor Gauss quadrature with n_q^3 points and weights w_a w_b w_c (Sec. 3.1);
  * element map T^K: [-1,1]^3 -> K trilinear in the 8 vertices, J_ij = dx_i/dxi_j;
  * element matrix (Eqs. (vectorMass), (localStiffnessQuadrature), with the
    Helmholtz combination A = c M + L of Sec. 5.2):
        A^K = sum_q w_q detJ_q [ alpha Phi_q Phi_q^T + nu_q (J^-T dPhi_q)^T (J^-T dPhi_q) ];
  * global action y = sum_K R_K^T A^K R_K x: the element-by-element sum of the
    operator action described in Sec. 3.1.

Local node order is lexicographic, i (the xi_1 index) fastest; quadrature
points likewise.  Global DoF order for structured meshes: lexicographic over
the (p nx + 1) x (p ny + 1) x (p nz + 1) grid of nodes, x fastest.
"""
from __future__ import annotations

import numpy as np

from .basis import gauss_rule, gll_nodes, lagrange_derivatives, lagrange_values


# --------------------------------------------------------------------------
# reference element
# --------------------------------------------------------------------------
class ReferenceElement:
    """1D and 3D basis tables of Q_p on [-1,1]^3 with an n_q-point Gauss rule per direction."""

    def __init__(self, p: int, q: int):
        self.p, self.q = p, q
        self.n = n = p + 1
        self.nodes = gll_nodes(p)
        self.xq, self.wq = gauss_rule(q)
        # Eq. (B1D): B[a, j] = phi_j(xi_a);  Eq. (D1D): D[a, j] = phi_j'(xi_a)
        self.B = lagrange_values(self.nodes, self.xq)
        self.D = lagrange_derivatives(self.nodes, self.xq)
        Q, N = q ** 3, n ** 3
        self.Q, self.N = Q, N
        # 3D quadrature points xi (Q, 3) and weights (Q,), index a + q b + q^2 c
        c, b, a = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
        a, b, c = a.ravel(), b.ravel(), c.ravel()
        self.xi = np.stack([self.xq[a], self.xq[b], self.xq[c]], axis=1)
        self.w = self.wq[a] * self.wq[b] * self.wq[c]
        # 3D basis as full products, node index i + n j + n^2 k
        kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
        Bx, By, Bz = self.B[a][:, i], self.B[b][:, j], self.B[c][:, k]
        Dx, Dy, Dz = self.D[a][:, i], self.D[b][:, j], self.D[c][:, k]
        self.Phi = Bx * By * Bz                                   # (Q, N)
        self.dPhi = np.stack([Dx * By * Bz, Bx * Dy * Bz, Bx * By * Dz], axis=2)  # (Q, N, 3)
        # reference coordinates of the local nodes (N, 3)
        self.node_xi = np.stack([self.nodes[i], self.nodes[j], self.nodes[k]], axis=1)


def trilinear_map(X8: np.ndarray, xi: np.ndarray):
    """Physical points x(xi) and Jacobians J[..., i, j] = dx_i/dxi_j of trilinear maps.

    X8 is (..., 8, 3): corner c = cx + 2 cy + 4 cz sits at reference corner
    (2cx-1, 2cy-1, 2cz-1), and its shape function is prod_d (1 + s_cd xi_d) / 2.
    xi is (P, 3).  Returns x (..., P, 3) and J (..., P, 3, 3).
    """
    X8 = np.asarray(X8, dtype=np.float64)
    lead = X8.shape[:-2]
    P = xi.shape[0]
    x = np.zeros(lead + (P, 3))
    J = np.zeros(lead + (P, 3, 3))
    for c in range(8):
        s = np.array([2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1], dtype=np.float64)
        f = (1.0 + s[None, :] * xi) / 2.0            # (P, 3) 1D factors
        N = f[:, 0] * f[:, 1] * f[:, 2]               # (P,)
        dN = np.stack([s[0] / 2 * f[:, 1] * f[:, 2],
                       s[1] / 2 * f[:, 0] * f[:, 2],
                       s[2] / 2 * f[:, 0] * f[:, 1]], axis=1)   # (P, 3): dN/dxi_j
        Xc = X8[..., c, :]                            # (..., 3)
        x += N[:, None] * Xc[..., None, :]
        J += Xc[..., None, :, None] * dN[:, None, :]
    return x, J


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
class Mesh:
    """A Q_p hexahedral mesh with trilinear elements.

    vertices (V, 3); elem_vert (E, 8); restriction (E, (p+1)^3) global DoF ids;
    dirichlet (n_dof,) bool mask of eliminated DoFs.
    """

    def __init__(self, p, q, vertices, elem_vert, restriction, n_dof, dirichlet=None):
        self.p, self.q = int(p), int(q)
        self.ref = ReferenceElement(self.p, self.q)
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.elem_vert = np.asarray(elem_vert, dtype=np.int64)
        self.restriction = np.asarray(restriction, dtype=np.int64)
        self.n_elem = self.elem_vert.shape[0]
        self.n_dof = int(n_dof)
        self.dirichlet = np.zeros(self.n_dof, dtype=bool) if dirichlet is None else np.asarray(dirichlet, dtype=bool)

    def element_dofs(self, e):
        return self.restriction[e]

    def qpoint_coords(self):
        """Physical coordinates of every quadrature point, (E, Q, 3)."""
        x, _ = trilinear_map(self.vertices[self.elem_vert], self.ref.xi)
        return x

    def element_node_coords(self):
        """Physical coordinates of every element's local nodes, (E, N, 3)."""
        x, _ = trilinear_map(self.vertices[self.elem_vert], self.ref.node_xi)
        return x

    def node_coords(self):
        """Physical coordinates of every global DoF (n_dof, 3), set from the element maps."""
        out = np.zeros((self.n_dof, 3))
        out[self.restriction] = self.element_node_coords()
        return out


def structured_restriction(nx, ny, nz, p, elems=None):
    """Global ids (len(elems), (p+1)^3) of the local nodes of elements of an nx x ny x nz grid.

    Element e = ex + nx (ey + ny ez) has local node (i, j, k) at global grid
    node (p ex + i, p ey + j, p ez + k), numbered x fastest.
    """
    n = p + 1
    gx, gy = p * nx + 1, p * ny + 1
    e = np.arange(nx * ny * nz, dtype=np.int64) if elems is None else np.asarray(elems, dtype=np.int64)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    l = np.arange(n ** 3, dtype=np.int64)
    i, j, k = l % n, (l // n) % n, l // (n * n)
    return (p * ex[:, None] + i[None, :]) + gx * ((p * ey[:, None] + j[None, :]) + gy * (p * ez[:, None] + k[None, :]))


def structured_boundary(nx, ny, nz, p):
    """Mask of global DoFs on the boundary of the box (homogeneous Dirichlet set)."""
    gx, gy, gz = p * nx + 1, p * ny + 1, p * nz + 1
    I, J, K = np.meshgrid(np.arange(gx), np.arange(gy), np.arange(gz), indexing="ij")
    on = (I == 0) | (I == gx - 1) | (J == 0) | (J == gy - 1) | (K == 0) | (K == gz - 1)
    return on.transpose(2, 1, 0).ravel()


class StructuredMesh(Mesh):
    """Mesh of an nx x ny x nz grid of hexahedra (vertex layout of ``synthetic``).

    lazy=True skips building the full restriction (large meshes): element
    DoFs are then computed per element by ``element_dofs``.
    """

    def __init__(self, nx, ny, nz, p, q, vertices, elem_vert, dirichlet_boundary=True, lazy=False):
        R = None if lazy else structured_restriction(nx, ny, nz, p)
        n_dof = (p * nx + 1) * (p * ny + 1) * (p * nz + 1)
        dmask = structured_boundary(nx, ny, nz, p) if dirichlet_boundary else None
        self.shape = (nx, ny, nz)
        if lazy:
            Mesh.__init__(self, p, q, vertices, elem_vert, np.zeros((0, (p + 1) ** 3), np.int64), n_dof, dmask)
            self.restriction = None
        else:
            super().__init__(p, q, vertices, elem_vert, R, n_dof, dmask)

    def element_dofs(self, e):
        if self.restriction is not None:
            return self.restriction[e]
        return structured_restriction(*self.shape, self.p, [e])[0]

    def elements_of_dof(self, g):
        """(element, local index) pairs containing global DoF g."""
        nx, ny, nz = self.shape
        p, n = self.p, self.p + 1
        gx, gy = p * nx + 1, p * ny + 1
        I, J, K = g % gx, (g // gx) % gy, g // (gx * gy)
        out = []
        for ez in {(K - 1) // p, K // p}:
            for ey in {(J - 1) // p, J // p}:
                for ex in {(I - 1) // p, I // p}:
                    if 0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz:
                        i, j, k = I - p * ex, J - p * ey, K - p * ez
                        if 0 <= i <= p and 0 <= j <= p and 0 <= k <= p:
                            out.append((ex + nx * (ey + ny * ez), i + n * (j + n * k)))
        return sorted(out)


# --------------------------------------------------------------------------
# operator alpha M + nu K
# --------------------------------------------------------------------------
class Operator:
    """A = alpha M + K(nu) on a Mesh, by explicit element matrices.

    nu is a scalar or an (E, Q) array of per-quadrature-point values.  All
    element matrices are built at construction when ``cache=True`` (small
    meshes); otherwise rows are built on demand (``apply_rows``).
    """

    def __init__(self, mesh: Mesh, alpha: float, nu, cache: bool = True, chunk: int = 256):
        self.mesh, self.alpha = mesh, float(alpha)
        self.nu = np.asarray(nu, dtype=np.float64) if np.ndim(nu) else float(nu)
        self._A = None
        if cache:
            E = mesh.n_elem
            self._A = np.empty((E, mesh.ref.N, mesh.ref.N))
            for e0 in range(0, E, chunk):
                es = np.arange(e0, min(E, e0 + chunk))
                self._A[es] = self.element_matrices(es)

    def _nu(self, es):
        Q = self.mesh.ref.Q
        if np.ndim(self.nu):
            return self.nu.reshape(self.mesh.n_elem, Q)[es]
        return np.full((len(es), Q), self.nu)

    def geometry(self, es):
        """(detJ (n,Q), Jinv (n,Q,3,3)) at the quadrature points of elements ``es``."""
        _, J = trilinear_map(self.mesh.vertices[self.mesh.elem_vert[es]], self.mesh.ref.xi)
        return np.linalg.det(J), np.linalg.inv(J)

    def element_matrices(self, es, rows=None):
        """A^K[rows, :] for every element K in ``es`` (Eq. (localStiffnessQuadrature) plus mass).

        A^K_ij = sum_q w_q detJ_q ( alpha phi_i phi_j + nu_q (J^-T dphi_i) . (J^-T dphi_j) ).
        """
        ref = self.mesh.ref
        es = np.atleast_1d(np.asarray(es))
        detJ, Jinv = self.geometry(es)
        if np.any(detJ <= 0):
            raise ValueError("non-positive Jacobian determinant")
        # physical gradients grad phi = J^-T dphi, stored as row vectors dphi^T J^-1
        gphys = np.einsum("qnd,eqdk->eqnk", ref.dPhi, Jinv)       # (n, Q, N, 3)
        cm = self.alpha * ref.w[None, :] * detJ                    # (n, Q) mass coefficient
        ck = self._nu(es) * ref.w[None, :] * detJ                  # (n, Q) stiffness coefficient
        r = slice(None) if rows is None else np.asarray(rows)
        Phi_r = ref.Phi[:, r]                                      # (Q, Nr)
        A = np.einsum("qi,eq,qj->eij", Phi_r, cm, ref.Phi, optimize=True)
        for d in range(3):
            A += np.einsum("eqi,eq,eqj->eij", gphys[:, :, r, d], ck, gphys[:, :, :, d], optimize=True)
        return A

    def element_matrix(self, e):
        return self._A[e] if self._A is not None else self.element_matrices([e])[0]

    def apply(self, x, constrained=False):
        """y = sum_K R_K^T A^K R_K x; constrained: y = P A P x + (I - P) x."""
        mesh = self.mesh
        x = np.asarray(x, dtype=np.float64)
        xin = np.where(mesh.dirichlet, 0.0, x) if constrained else x
        yE = np.matmul(self._A, xin[mesh.restriction][:, :, None])[:, :, 0]
        y = np.zeros(mesh.n_dof)
        np.add.at(y, mesh.restriction, yE)
        if constrained:
            y = np.where(mesh.dirichlet, x, y)
        return y

    def apply_rows(self, x, dofs, constrained=False):
        """Entries ``dofs`` of the action, each summed over the elements holding the DoF."""
        mesh = self.mesh
        x = np.asarray(x, dtype=np.float64)
        xin = np.where(mesh.dirichlet, 0.0, x) if constrained else x
        out = np.zeros(len(dofs))
        for t, g in enumerate(dofs):
            if constrained and mesh.dirichlet[g]:
                out[t] = x[g]
                continue
            for e, l in mesh.elements_of_dof(int(g)):
                row = self.element_matrices([e], [l])[0, 0]
                out[t] += row @ xin[mesh.element_dofs(e)]
        return out

    def diagonal(self, constrained=False):
        """diag(A) = sum_K R_K^T diag(A^K); Dirichlet rows are 1 when constrained."""
        mesh = self.mesh
        d = np.zeros(mesh.n_dof)
        np.add.at(d, mesh.restriction, np.einsum("eii->ei", self._A))
        if constrained:
            d = np.where(mesh.dirichlet, 1.0, d)
        return d

    def assembled(self, constrained=False):
        """Dense global matrix summed from the element matrices (small meshes only)."""
        mesh = self.mesh
        A = np.zeros((mesh.n_dof, mesh.n_dof))
        for e in range(mesh.n_elem):
            R = mesh.restriction[e]
            A[np.ix_(R, R)] += self._A[e]
        if constrained:
            P = ~mesh.dirichlet
            A = A * P[:, None] * P[None, :]
            A[mesh.dirichlet, mesh.dirichlet] = 1.0
        return A


def load_vector(mesh: Mesh, f_q):
    """b_i = sum_K sum_q w_q detJ_q f(x_q) phi_i(xi_q): the weak right-hand side (f, phi_i)."""
    ref = mesh.ref
    f_q = np.asarray(f_q, dtype=np.float64).reshape(mesh.n_elem, ref.Q)
    _, J = trilinear_map(mesh.vertices[mesh.elem_vert], ref.xi)
    detJ = np.linalg.det(J)
    bE = (ref.w[None, :] * detJ * f_q) @ ref.Phi                  # (E, N)
    b = np.zeros(mesh.n_dof)
    np.add.at(b, mesh.restriction, bE)
    return b


def l2_error(mesh: Mesh, u_dofs, u_exact, extra_points: int = 2):
    """||u_h - u||_L2 integrated with (q + extra_points) Gauss points per direction."""
    ref = ReferenceElement(mesh.p, mesh.q + extra_points)
    x, J = trilinear_map(mesh.vertices[mesh.elem_vert], ref.xi)
    detJ = np.linalg.det(J)
    uh = np.asarray(u_dofs)[mesh.restriction] @ ref.Phi.T        # (E, Q)
    return float(np.sqrt(np.sum(ref.w[None, :] * detJ * (uh - u_exact(x)) ** 2)))
