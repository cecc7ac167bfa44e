"""Pin computations shared by the oracle tests and the planted-mistake tests.

Each function returns an error measure that must be ~0 for a correct oracle;
the planted-mistake tests monkeypatch the oracle and check that the same
function then reports a large error.
"""
import os

from fractions import Fraction

import numpy as np
import sympy as sp

import synthetic as S
from oracle import fem
from oracle.basis import gauss_rule, gll_nodes, lagrange_derivatives, lagrange_values

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            out[i + j] += ai * bj
    return out


def _pder(a):
    return [k * a[k] for k in range(1, len(a))] or [Fraction(0)]


def _pint11(a):
    """Exact integral over [-1, 1] of the polynomial with coefficients a (ascending)."""
    return sum((c * 2 / (k + 1) for k, c in enumerate(a) if k % 2 == 0), Fraction(0))


def exact_1d_matrices(p):
    """Exact 1D mass and stiffness of the Lagrange basis on the GLL nodes.

    Exact rational arithmetic (Python Fractions) on the double-precision nodes:
    the Lagrange polynomials are expanded into monomials and integrated
    exactly, so nothing is shared with the oracle's quadrature or its product
    formulas.
    """
    nodes = [Fraction(float(v)) for v in gll_nodes(p)]
    n = p + 1
    phis = []
    for j in range(n):
        poly = [Fraction(1)]
        for m in range(n):
            if m != j:
                d = nodes[j] - nodes[m]
                poly = _pmul(poly, [-nodes[m] / d, 1 / d])
        phis.append(poly)
    dphis = [_pder(f) for f in phis]
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            M[i, j] = float(_pint11(_pmul(phis[i], phis[j])))
            K[i, j] = float(_pint11(_pmul(dphis[i], dphis[j])))
    return M, K


def oracle_1d_matrices(p, q):
    """1D mass and stiffness from the oracle's B, D and Gauss weights: B^T W B, D^T W D."""
    ref = fem.ReferenceElement(p, q)
    W = np.diag(ref.wq)
    return ref.B.T @ W @ ref.B, ref.D.T @ W @ ref.D


def box_element_error(p, q, a=0.7, b=1.3, c=0.4, alpha=1.7, nu=0.6):
    """Axis-aligned box element: oracle A^K vs the Kronecker form of exact 1D matrices."""
    M1, K1 = exact_1d_matrices(p)
    V = S.structured_vertices(1, 1, 1, 0.0)
    V = S.affine_map(V, np.diag([a, b, c]), [0.2, -0.1, 0.3])
    mesh = fem.StructuredMesh(1, 1, 1, p, q, V, S.structured_elem_vert(1, 1, 1), dirichlet_boundary=False)
    A = fem.Operator(mesh, alpha, nu).element_matrix(0)
    vol = a * b * c / 8.0
    kr = lambda Z, Y, X: np.kron(Z, np.kron(Y, X))  # node index i + n j + n^2 k
    ref = alpha * vol * kr(M1, M1, M1) + nu * vol * (
        (2 / a) ** 2 * kr(M1, M1, K1) + (2 / b) ** 2 * kr(M1, K1, M1) + (2 / c) ** 2 * kr(K1, M1, M1))
    return np.max(np.abs(A - ref)) / np.max(np.abs(ref))


SHEAR = np.array([[1.0, 0.35, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.05, 1.2]])
SHIFT = np.array([0.1, -0.2, 0.05])


def _poly(p):
    x, y, z = sp.symbols("x y z")
    terms = [1, x, -2 * y, z / 3, x * y, -z * z / 2, x * z, y * y]
    if p >= 3:
        terms += [x * y * z / 4, -x ** 3 / 3, y * z * z]
    if p >= 4:
        terms += [x * x * y * y / 2, -z ** 4 / 5, x * y * z * z]
    return (x, y, z), sum(sp.Rational(1, 1) * sp.sympify(tm) for tm in terms)


def energy_error(p, q, nx=2, ny=2, nz=1):
    """Sheared affine mesh: u^T K u = int |grad u|^2 and u^T M u = int u^2, exactly (degree <= p u)."""
    (x, y, z), u = _poly(p)
    A = sp.Matrix(SHEAR.tolist()).applyfunc(lambda v: sp.nsimplify(v))
    bvec = sp.Matrix(SHIFT.tolist()).applyfunc(lambda v: sp.nsimplify(v))
    s1, s2, s3 = sp.symbols("s1 s2 s3")
    X = A * sp.Matrix([s1, s2, s3]) + bvec
    sub = {x: X[0], y: X[1], z: X[2]}
    grad2 = sum(sp.diff(u, v) ** 2 for v in (x, y, z))
    detA = abs(A.det())
    intK = float(detA * sp.integrate(sp.expand(grad2.subs(sub)), (s1, 0, 1), (s2, 0, 1), (s3, 0, 1)))
    intM = float(detA * sp.integrate(sp.expand((u * u).subs(sub)), (s1, 0, 1), (s2, 0, 1), (s3, 0, 1)))
    V = S.affine_map(S.structured_vertices(nx, ny, nz, 0.0), SHEAR, SHIFT)
    mesh = fem.StructuredMesh(nx, ny, nz, p, q, V, S.structured_elem_vert(nx, ny, nz), dirichlet_boundary=False)
    ufun = sp.lambdify((x, y, z), u, "numpy")
    Xn = mesh.node_coords()
    uL = ufun(Xn[:, 0], Xn[:, 1], Xn[:, 2]) * np.ones(mesh.n_dof)
    K = fem.Operator(mesh, 0.0, 1.0)
    M = fem.Operator(mesh, 1.0, 0.0)
    eK = abs(uL @ K.apply(uL) - intK) / abs(intK)
    eM = abs(uL @ M.apply(uL) - intM) / abs(intM)
    return eK, eM


def volume_error(p, q, n=3):
    """1^T M 1 equals the volume (= 1) of the perturbed unit cube."""
    V = S.structured_vertices(n, n, n, 0.1, 77)
    mesh = fem.StructuredMesh(n, n, n, p, q, V, S.structured_elem_vert(n, n, n), dirichlet_boundary=False)
    one = np.ones(mesh.n_dof)
    return abs(one @ fem.Operator(mesh, 1.0, 0.0).apply(one) - 1.0)


def mms_errors(p, Ns, perturb, alpha=1.0, nu=1.0):
    """L2 errors of the Jacobi-PCG solution of the manufactured problem u = sin(pi x) sin(pi y) sin(pi z)."""
    from oracle.solve import jacobi_pcg
    q = p + 2
    uex = lambda X: np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    errs = []
    for N in Ns:
        V = S.structured_vertices(N, N, N, perturb, 1910)
        mesh = fem.StructuredMesh(N, N, N, p, q, V, S.structured_elem_vert(N, N, N))
        op = fem.Operator(mesh, alpha, nu)
        f = (alpha + 3 * np.pi ** 2 * nu) * uex(mesh.qpoint_coords())
        b = fem.load_vector(mesh, f)
        x, its, rel, conv = jacobi_pcg(op, b, 1e-12, 5000)
        assert conv
        errs.append(fem.l2_error(mesh, x, uex))
    return np.array(errs)
