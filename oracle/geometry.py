"""FP64 geometry of eqs. 3, 4, 7 and 8 (oracle; test infrastructure only).

* O_j: circumcentre of triangle j, where B_j lives (Fig. 2).
* C_i: midpoint of edge i, where E_i and j_i live.
* |e_i|: edge length; S_j: triangle area.
* d_i: the distance |O_R(i) O_L(i)| of eq. 3, taken signed: d_i = (O_R - O_L) . n_i where n_i is
  the unit normal pointing from the edge into R(i) (to the left of e_i).  For a Delaunay mesh
  d_i >= 0 and it equals |O_R O_L|, which is also O_R C_i + O_L C_i of eq. 8.
* the literal sign factor of eq. 4, sgn(y0 . (O_j C_A(j,q) x e_A(j,q))), kept for comparison
  with the integer orientation sign used by the scheme (they agree whenever the angle opposite
  the edge is acute; they can differ when O_j falls outside the triangle).

Parity: pinned by tests/test_oracle_geometry.py (closed forms for equilateral and right
triangles, an independent cotangent formula for d_i, total area, the acute-angle agreement of
the literal sign).
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh


def circumcentres(xy: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Circumcentre of each triangle, computed relative to its first vertex."""
    p0 = xy[tris[:, 0]]
    b = xy[tris[:, 1]] - p0
    c = xy[tris[:, 2]] - p0
    D = 2.0 * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0])
    b2 = b[:, 0] ** 2 + b[:, 1] ** 2
    c2 = c[:, 0] ** 2 + c[:, 1] ** 2
    ux = (c[:, 1] * b2 - b[:, 1] * c2) / D
    uy = (b[:, 0] * c2 - c[:, 0] * b2) / D
    return p0 + np.stack([ux, uy], axis=1)


def areas(xy: np.ndarray, tris: np.ndarray) -> np.ndarray:
    p0 = xy[tris[:, 0]]
    p1 = xy[tris[:, 1]]
    p2 = xy[tris[:, 2]]
    return 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0]))


def edge_vectors(mesh: Mesh) -> np.ndarray:
    return mesh.xy[mesh.edges[:, 1]] - mesh.xy[mesh.edges[:, 0]]


def edge_lengths(mesh: Mesh) -> np.ndarray:
    v = edge_vectors(mesh)
    return np.hypot(v[:, 0], v[:, 1])


def midpoints(mesh: Mesh) -> np.ndarray:
    return 0.5 * (mesh.xy[mesh.edges[:, 0]] + mesh.xy[mesh.edges[:, 1]])


def dual_lengths(mesh: Mesh, O: np.ndarray) -> np.ndarray:
    """Signed |O_R O_L| for every edge (NaN on boundary edges)."""
    v = edge_vectors(mesh)
    ln = np.hypot(v[:, 0], v[:, 1])
    nx = -v[:, 1] / ln
    ny = v[:, 0] / ln
    d = np.full(mesh.n_edges, np.nan)
    ii = mesh.interior
    dO = O[mesh.R[ii]] - O[mesh.L[ii]]
    d[ii] = dO[:, 0] * nx[ii] + dO[:, 1] * ny[ii]
    return d


def literal_signs(mesh: Mesh, O: np.ndarray) -> np.ndarray:
    """sgn(y0 . (O_j C_q x e_q)) for every (triangle, q); 0 where the cross product is 0."""
    C = midpoints(mesh)
    v = edge_vectors(mesh)
    e = mesh.tri_edge
    oc = C[e] - O[:, None, :]
    ev = v[e]
    cr = oc[..., 0] * ev[..., 1] - oc[..., 1] * ev[..., 0]
    return np.sign(cr).astype(np.int64)


class Geometry:
    """All per-mesh FP64 quantities the scheme needs."""

    def __init__(self, mesh: Mesh):
        self.O = circumcentres(mesh.xy, mesh.tris)
        self.S = areas(mesh.xy, mesh.tris)
        self.elen = edge_lengths(mesh)
        self.C = midpoints(mesh)
        self.d = dual_lengths(mesh, self.O)
