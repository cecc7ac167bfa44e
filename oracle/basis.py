"""1D nodes, quadrature and Lagrange polynomials for the oracle (Sec. 3.1).

Gauss-Lobatto points: -1, +1 and the roots of P_p'(x) (P_p the Legendre
polynomial of degree p).  Gauss points: the roots of P_q(x), with weights
w = 2 / ((1 - x^2) P_q'(x)^2).  Both found by Newton's method on the
three-term Legendre recurrence.  Lagrange basis functions and their
derivatives are evaluated with the direct product formulas.
"""
from __future__ import annotations

import math

import numpy as np


def legendre(n: int, x):
    """Return (P_n(x), P_n'(x)) by the three-term recurrence (n >= 0)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n); valid off the endpoints
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    # endpoints: P_n'(+-1) = (+-1)^(n-1) n (n+1) / 2
    end = np.abs(np.abs(x) - 1.0) == 0.0
    if np.any(end):
        dp = np.where(end, np.sign(x) ** (n - 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gauss_rule(q: int):
    """Nodes and weights of the q-point Gauss-Legendre rule on [-1, 1], ascending."""
    if q < 1:
        raise ValueError("q >= 1")
    x = np.array([-math.cos(math.pi * (i + 0.75) / (q + 0.5)) for i in range(q)])
    for _ in range(100):
        pq, dq = legendre(q, x)
        dx = pq / dq
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dq = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dq * dq)
    return x, w


def gll_nodes(p: int):
    """The p+1 Gauss-Lobatto-Legendre points on [-1, 1], ascending (p >= 1)."""
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([-1.0, 1.0])
    # interior points: roots of P_p'; Newton on f = P_p' with
    # f' = P_p'' = (2x P_p' - p(p+1) P_p) / (1 - x^2)  (Legendre's equation)
    x = np.array([-math.cos(math.pi * i / p) for i in range(1, p)])
    for _ in range(100):
        P, dP = legendre(p, x)
        d2P = (2.0 * x * dP - p * (p + 1) * P) / (1.0 - x * x)
        dx = dP / d2P
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    return np.concatenate([[-1.0], x, [1.0]])


def lagrange_values(nodes, x):
    """V[a, j] = phi_j(x_a), phi_j the Lagrange polynomial of ``nodes`` with phi_j(nodes[k]) = delta_jk."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    V = np.ones((x.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                V[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return V


def lagrange_derivatives(nodes, x):
    """G[a, j] = phi_j'(x_a) by the product rule applied to the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    G = np.zeros((x.size, n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(x.size, 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            G[:, j] += term
    return G
