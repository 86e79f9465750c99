"""Mesh symbols of Fig. 2 in the caller's numbering (oracle; test infrastructure only).

Field placement (Fig. 1): E and the current j on edges, B on triangles, the density n on nodes.
Fig. 2 names, per edge i, a "right" and a "left" triangle R(i), L(i), and per triangle j its
three edges A(j, q).  The paper leaves the direction of e_i free; this oracle fixes:

* every triangle is made counter-clockwise (sign of the FP64 orientation determinant);
* edge i is directed from its lower to its higher caller node id; edges are numbered by sorting
  the (low, high) pairs lexicographically (the caller edge numbering);
* A(j, q) for q = 0, 1, 2 is the edge from vertex q to vertex q+1 (mod 3) of the CCW triangle;
* s(j, q) = +1 if that edge's direction agrees with the CCW walk around triangle j, else -1;
* R(i) is the triangle with s = +1 (the edge runs counter-clockwise around it), L(i) the one
  with s = -1.  This is the only assignment for which the two sums of eq. 10 cancel, i.e. for
  which the discrete energy is conserved;
* an edge with a single triangle is a boundary edge: the ideal-resonator condition of eq. 10
  (E = 0 on the outer edges) removes it from the unknowns.

Parity: pinned by tests/test_oracle_mesh.py (hand-worked two-triangle and strip meshes,
orientation handling, error cases) and by the exact invariants in tests/test_oracle_invariants.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# error codes shared in meaning (not in code) with the C-ABI
ERR_ARG = -1
ERR_NONMANIFOLD = -2
ERR_DEGENERATE = -3


class MeshError(ValueError):
    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


@dataclasses.dataclass
class Mesh:
    xy: np.ndarray          # f64 [n_n, 2]
    tris: np.ndarray        # i64 [n_t, 3], counter-clockwise
    edges: np.ndarray       # i64 [n_e, 2], (low, high) caller node ids, lexicographic order
    tri_edge: np.ndarray    # i64 [n_t, 3], A(j, q)
    tri_sign: np.ndarray    # i64 [n_t, 3], s(j, q) in {+1, -1}
    R: np.ndarray           # i64 [n_e], -1 if none
    L: np.ndarray           # i64 [n_e], -1 if none
    interior: np.ndarray    # bool [n_e]

    @property
    def n_nodes(self):
        return self.xy.shape[0]

    @property
    def n_tris(self):
        return self.tris.shape[0]

    @property
    def n_edges(self):
        return self.edges.shape[0]

    @property
    def interior_ids(self):
        return np.nonzero(self.interior)[0]


def orient2d(xy: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Twice the signed area of each triangle, (p1 - p0) x (p2 - p0), in FP64."""
    p0 = xy[tris[:, 0]]
    p1 = xy[tris[:, 1]]
    p2 = xy[tris[:, 2]]
    return (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])


def canonicalize(xy, tris) -> Mesh:
    """Build the Fig. 2 symbols from caller arrays; raise MeshError on invalid input."""
    xy = np.asarray(xy, dtype=np.float64)
    tris = np.asarray(tris)
    if xy.ndim != 2 or xy.shape[1] != 2 or tris.ndim != 2 or tris.shape[1] != 3 or tris.shape[0] == 0:
        raise MeshError(ERR_ARG, "xy must be [n,2] and tris [m,3] with m > 0")
    if not np.all(np.isfinite(xy)):
        raise MeshError(ERR_ARG, "non-finite node coordinate")
    tris = tris.astype(np.int64)
    n = xy.shape[0]
    if tris.min() < 0 or tris.max() >= n:
        raise MeshError(ERR_ARG, "triangle vertex index out of range")
    if np.any((tris[:, 0] == tris[:, 1]) | (tris[:, 1] == tris[:, 2]) | (tris[:, 0] == tris[:, 2])):
        raise MeshError(ERR_DEGENERATE, "triangle with a repeated vertex")
    det = orient2d(xy, tris)
    if np.any(det == 0):
        raise MeshError(ERR_DEGENERATE, "degenerate triangle (zero orientation determinant)")
    tris = tris.copy()
    cw = det < 0
    tris[cw] = tris[cw][:, [0, 2, 1]]
    # half-edge (j, q): tris[j, q] -> tris[j, q+1]
    a = tris[:, [0, 1, 2]]
    b = tris[:, [1, 2, 0]]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = (lo * n + hi).reshape(-1)
    uniq, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    if np.any(cnt > 2):
        raise MeshError(ERR_NONMANIFOLD, "edge shared by more than two triangles")
    edges = np.stack([uniq // n, uniq % n], axis=1)
    tri_edge = inv.reshape(-1, 3)
    tri_sign = np.where(a < b, 1, -1).astype(np.int64)
    n_e = edges.shape[0]
    R = np.full(n_e, -1, np.int64)
    L = np.full(n_e, -1, np.int64)
    owner = np.repeat(np.arange(tris.shape[0]), 3)
    s = tri_sign.reshape(-1)
    e = tri_edge.reshape(-1)
    pos = s > 0
    # an edge walked twice in the same direction means overlapping / folded triangles
    if np.bincount(e[pos], minlength=n_e).max(initial=0) > 1 or \
            np.bincount(e[~pos], minlength=n_e).max(initial=0) > 1:
        raise MeshError(ERR_NONMANIFOLD, "edge walked twice in the same direction (folded or overlapping triangles)")
    R[e[pos]] = owner[pos]
    L[e[~pos]] = owner[~pos]
    interior = cnt == 2
    return Mesh(xy, tris, edges, tri_edge, tri_sign, R, L, interior)
