"""An unstructured hexahedral test mesh: a star-shaped prism whose central edge has valence k.

k convex quads share the centre vertex of the plane: quad j has corners (centre, spoke j,
tip j, spoke j + 1), spokes at radius r1 and angle 2 pi j / k, tips at radius r2 halfway
between. Each quad is split m x m (bilinearly) and the plane is extruded into nz layers of
height h / nz. The Q_p numbering comes from matching the physical coordinates of every
element's local nodes (shared nodes coincide up to rounding), so it holds for any conforming
mesh. With k = 5 the DoFs on the central edge couple to 2k + 1 = 11 nodes per layer in the
low-order refined matrix: 33 entries in a row instead of the 27 of a structured grid.

Test infrastructure: the node positions use the oracle's reference element.
"""
import math

import numpy as np


def star_prism(p, q=None, k=5, m=2, nz=3, r1=1.0, r2=1.3, h=1.0, dirichlet_bottom=True):
    """(vertices, elem_vert, oracle Mesh); Dirichlet DoFs on the bottom face z = 0 if asked."""
    from oracle import fem
    q = p + 2 if q is None else q
    # plane vertices, merged by position
    keys, plane = {}, []

    def vid(x, y):
        key = (round(x, 12), round(y, 12))
        if key not in keys:
            keys[key] = len(plane)
            plane.append((x, y))
        return keys[key]

    quads = []
    for j in range(k):
        a0, a1 = 2 * math.pi * j / k, 2 * math.pi * (j + 1) / k
        c = np.zeros(2)
        s0 = r1 * np.array([math.cos(a0), math.sin(a0)])
        s1 = r1 * np.array([math.cos(a1), math.sin(a1)])
        t = r2 * np.array([math.cos((a0 + a1) / 2), math.sin((a0 + a1) / 2)])
        # local corners: (0,0) centre, (1,0) spoke j, (1,1) tip j, (0,1) spoke j + 1
        ids = np.empty((m + 1, m + 1), np.int64)
        for b in range(m + 1):
            for a in range(m + 1):
                u, v = a / m, b / m
                x = (1 - u) * (1 - v) * c + u * (1 - v) * s0 + u * v * t + (1 - u) * v * s1
                ids[b, a] = vid(x[0], x[1])
        for b in range(m):
            for a in range(m):
                quads.append((ids[b, a], ids[b, a + 1], ids[b + 1, a], ids[b + 1, a + 1]))
    P = np.array(plane)
    n2 = len(plane)
    V = np.concatenate([np.column_stack([P, np.full(n2, h * l / nz)]) for l in range(nz + 1)])
    EV = np.array([[l * n2 + v for v in qd] + [(l + 1) * n2 + v for v in qd]
                   for l in range(nz) for qd in quads], dtype=np.int64)
    # Q_p numbering by node position
    n3 = (p + 1) ** 3
    probe = fem.Mesh(p, q, V, EV, np.zeros((len(EV), n3), np.int64), 1)
    X = probe.element_node_coords().reshape(-1, 3)
    _, first, inv = np.unique(np.round(X, 9), axis=0, return_index=True, return_inverse=True)
    # ids in order of first appearance (element by element), so the numbering is not sorted by position
    order = np.argsort(first)
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    R = rank[inv.ravel()].reshape(len(EV), n3)
    n_dof = len(first)
    dirichlet = np.zeros(n_dof, bool)
    if dirichlet_bottom:
        dirichlet[R.ravel()[np.abs(X[:, 2]) < 1e-12]] = True
    om = fem.Mesh(p, q, V, EV, R, n_dof, dirichlet)
    return V, EV, om


def star_prism_volume(k=5, r1=1.0, r2=1.3, h=1.0):
    """Closed-form volume: k quads, each two triangles of area r1 r2 sin(pi / k) / 2, times h."""
    return k * r1 * r2 * math.sin(math.pi / k) * h
