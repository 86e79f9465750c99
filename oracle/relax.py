"""Mesh optimisation: the jello model and flip refinement (oracle).

Test infrastructure only.  Section 3 ("Mesh generation"): nodes joined by springs along the
triangle edges and along the heights relax towards a mesh of near-perfect triangles.  The
damping is strong enough to drop the second time derivative, so the motion is first order and
an Euler step does.  The nodes that seed the input geometry stay put, and the node cloud is
remeshed now and then, because deformed triangles stop the relaxation around them.

Readings (where the paper gives the idea but not the formulas):
* rest length of edge ab: L0 = (h_a + h_b) / 2 from a size per node; without sizes, the edge of
  an equilateral triangle of the mean area: h = sqrt(4 A / (sqrt(3) n_t)), A the total area;
* a height spring joins each vertex v to the midpoint m of its opposite edge (for an
  equilateral triangle, along the height) with rest length H0 = sqrt(3)/2 times the mean rest
  length of the triangle's edges;
* all springs have unit stiffness, so the forces are -grad E for
  E = sum_edges (|ab| - L0)^2 / 2 + sum_heights (|v - m| - H0)^2 / 2;
* one step: x += tau F, each node's displacement clamped to 0.1 of its shortest rest edge and
  to 0.15 of the smallest height h among its triangles (2 area / longest edge L, at the current
  positions): moves of at most d per vertex change twice a triangle's area by at most
  3 d L + 4 d^2 <= 0.54 h L, less than the 2 area = h L it has, so no triangle turns over;
  nodes on the boundary (on an edge of one triangle) do not move;
* remesh: Lawson flips of the interior edges that are not locally Delaunay (the vertex
  opposite in one triangle inside the other's circumcircle, beyond a relative 1e-10 margin),
  until none is left; boundary edges are never flipped, so holes keep their contours;
* anchoring: the seeding nodes of the input geometry stay put.  Boundary nodes are anchored
  always; nodes of interior geometry (an object's contour meshed on both sides, a path) are
  named by the caller, and so are the geometry edges between them, which the remesh keeps.

Parity: pinned by tests/test_oracle_relax.py (forces against central differences of E, the
equilateral lattice as a fixed point, E non-increasing along the flow, Lawson flips of a
scrambled triangulation of random points giving Qhull's Delaunay triangulation, Lawson flips
with kept edges giving the constrained Delaunay triangulation that flip refinement builds
independently, and anchored contour nodes and kept contour edges surviving the relaxation).
"""
from __future__ import annotations

import math

import numpy as np


def orient_ccw(xy: np.ndarray, tris: np.ndarray) -> np.ndarray:
    t = np.array(tris, np.int64)
    a, b, c = xy[t[:, 0]], xy[t[:, 1]], xy[t[:, 2]]
    neg = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]) < 0
    t[neg, 1], t[neg, 2] = t[neg, 2].copy(), t[neg, 1].copy()
    return t


def edges_of(tris: np.ndarray):
    """(unique edges (low, high), number of triangles of each edge)."""
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    u, cnt = np.unique(e, axis=0, return_counts=True)
    return u, cnt


def boundary_nodes(n_nodes: int, tris: np.ndarray) -> np.ndarray:
    u, cnt = edges_of(tris)
    bnd = np.zeros(n_nodes, bool)
    bnd[u[cnt == 1].ravel()] = True
    return bnd


def uniform_size(xy: np.ndarray, tris: np.ndarray) -> float:
    t = orient_ccw(xy, tris)
    a, b, c = xy[t[:, 0]], xy[t[:, 1]], xy[t[:, 2]]
    area = 0.5 * np.sum((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    return math.sqrt(4.0 * area / (math.sqrt(3.0) * t.shape[0]))


def rest_lengths(tris: np.ndarray, h_nodes: np.ndarray):
    """(edges, L0 per edge, H0 per triangle)."""
    edges, _ = edges_of(tris)
    L0 = 0.5 * (h_nodes[edges[:, 0]] + h_nodes[edges[:, 1]])
    he = [0.5 * (h_nodes[tris[:, q]] + h_nodes[tris[:, (q + 1) % 3]]) for q in range(3)]
    H0 = math.sqrt(3.0) / 2.0 * (he[0] + he[1] + he[2]) / 3.0
    return edges, L0, H0


def energy(xy, tris, edges, L0, H0) -> float:
    d = np.linalg.norm(xy[edges[:, 1]] - xy[edges[:, 0]], axis=1)
    E = 0.5 * np.sum((d - L0) ** 2)
    for q in range(3):
        v, p, r = tris[:, q], tris[:, (q + 1) % 3], tris[:, (q + 2) % 3]
        hm = np.linalg.norm(xy[v] - 0.5 * (xy[p] + xy[r]), axis=1)
        E += 0.5 * np.sum((hm - H0) ** 2)
    return float(E)


def forces(xy, tris, edges, L0, H0, bnd) -> np.ndarray:
    """-grad E, zero on the boundary nodes."""
    F = np.zeros_like(xy)
    a, b = edges[:, 0], edges[:, 1]
    dv = xy[b] - xy[a]
    L = np.linalg.norm(dv, axis=1)
    f = ((L - L0) / L)[:, None] * dv            # pulls a towards b when stretched
    np.add.at(F, a, f)
    np.add.at(F, b, -f)
    for q in range(3):
        v, p, r = tris[:, q], tris[:, (q + 1) % 3], tris[:, (q + 2) % 3]
        w = xy[v] - 0.5 * (xy[p] + xy[r])
        hm = np.linalg.norm(w, axis=1)
        g = ((hm - H0) / hm)[:, None] * w       # grad of (|w| - H0)^2 / 2 with respect to v
        np.add.at(F, v, -g)
        np.add.at(F, p, 0.5 * g)
        np.add.at(F, r, 0.5 * g)
    F[bnd] = 0.0
    return F


def relax(xy, tris, iters: int, tau: float = 0.05, h_nodes=None, flip_every: int = 0, anchors=(),
          keep=()):
    """(new positions, new triangles (CCW), number of flips) after `iters` Euler steps, with
    Lawson flips after every `flip_every` steps (0: never).  `anchors`: node ids that stay put
    besides the boundary nodes (the seeding nodes of interior geometry); `keep`: node-id pairs,
    edges of the geometry that are never flipped."""
    xy = np.array(xy, np.float64)
    t = orient_ccw(xy, tris)
    if h_nodes is None:
        h_nodes = np.full(xy.shape[0], uniform_size(xy, t))
    bnd = boundary_nodes(xy.shape[0], t)
    bnd[np.asarray(anchors, np.int64).reshape(-1)] = True
    n_flips = 0
    edges, L0, H0 = rest_lengths(t, h_nodes)
    for it in range(iters):
        # the cap of a node: 0.1 of its shortest rest edge, 0.15 of its triangles' smallest height
        cap = np.full(xy.shape[0], np.inf)
        np.minimum.at(cap, edges[:, 0], 0.1 * L0)
        np.minimum.at(cap, edges[:, 1], 0.1 * L0)
        a, b, c = xy[t[:, 0]], xy[t[:, 1]], xy[t[:, 2]]
        area2 = np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
        lmax = np.maximum(np.maximum(np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1)),
                          np.linalg.norm(a - c, axis=1))
        hmin = area2 / lmax
        for q in range(3):
            np.minimum.at(cap, t[:, q], 0.15 * hmin)
        dx = tau * forces(xy, t, edges, L0, H0, bnd)
        n = np.linalg.norm(dx, axis=1)
        scale = np.where(n > cap, cap / np.where(n > 0, n, 1.0), 1.0)
        xy = xy + dx * scale[:, None]
        if flip_every > 0 and (it + 1) % flip_every == 0:
            t, k = lawson_flips(xy, t, keep)
            n_flips += k
            edges, L0, H0 = rest_lengths(t, h_nodes)
    return xy, t, n_flips


def _in_circle(xy, a, b, c, d) -> bool:
    """d strictly inside the circumcircle of the CCW triangle abc, beyond a relative margin."""
    ax, ay = xy[a] - xy[d]
    bx, by = xy[b] - xy[d]
    cx, cy = xy[c] - xy[d]
    det = ((ax * ax + ay * ay) * (bx * cy - by * cx) - (bx * bx + by * by) * (ax * cy - ay * cx)
           + (cx * cx + cy * cy) * (ax * by - ay * bx))
    s = max(ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy)
    return det > 1e-10 * s * s


def _ccw(xy, a, b, c) -> float:
    return (xy[b][0] - xy[a][0]) * (xy[c][1] - xy[a][1]) - (xy[b][1] - xy[a][1]) * (xy[c][0] - xy[a][0])


def lawson_flips(xy, tris, keep=()):
    """Flip interior edges, except the node-id pairs in `keep`, until every one is locally
    Delaunay; (triangles, flips)."""
    fixed = {frozenset((int(u), int(v))) for u, v in np.asarray(keep, np.int64).reshape(-1, 2)}
    t = [list(r) for r in orient_ccw(xy, tris)]
    owner = {}          # directed edge (u, v) -> triangle holding it in CCW order
    for i, (a, b, c) in enumerate(t):
        for u, v in ((a, b), (b, c), (c, a)):
            owner[(u, v)] = i
    stack = [e for e in owner if (e[1], e[0]) in owner and e[0] < e[1]]
    flips = 0
    while stack:
        a, b = stack.pop()
        if (a, b) not in owner or (b, a) not in owner or frozenset((a, b)) in fixed:
            continue
        i, j = owner[(a, b)], owner[(b, a)]
        c = [x for x in t[i] if x != a and x != b][0]      # (a, b, c) CCW
        d = [x for x in t[j] if x != a and x != b][0]      # (b, a, d) CCW
        if not _in_circle(xy, a, b, c, d):
            continue
        if _ccw(xy, a, d, c) <= 0 or _ccw(xy, d, b, c) <= 0:   # quad not convex: keep
            continue
        for u, v in ((a, b), (b, c), (c, a), (b, a), (a, d), (d, b)):
            owner.pop((u, v), None)
        t[i] = [a, d, c]
        t[j] = [d, b, c]
        for k, (u, v, w) in ((i, t[i]), (j, t[j])):
            for e in ((u, v), (v, w), (w, u)):
                owner[e] = k
        flips += 1
        for u, v in ((a, d), (d, b), (b, c), (c, a)):
            stack.append((min(u, v), max(u, v)))
    return np.asarray(t, np.int64), flips
