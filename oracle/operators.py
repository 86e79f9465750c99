"""The discrete curl operators L_B (eq. 3) and L_E (eq. 4) and the metric of eq. 7.

Oracle; test infrastructure only.  Unknowns are the interior edges (ideal resonator, eq. 10:
E = 0 on boundary edges) in increasing caller edge id, and all triangles in caller order.

* (L_B B)_i = (B_R(i) - B_L(i)) / d_i                                    eq. 3
* (L_E E)_j = -(1/S_j) sum_q s(j,q) |e_A(j,q)| E_A(j,q)                   eq. 4
  with s(j,q) the orientation sign of the mesh module standing for the literal
  sgn(y0 . (O_j C x e)) factor of eq. 4.
* metric (eq. 7): w_E,i = d_i |e_i| on edges, w_B,j = S_j on triangles.

A merged variant (``merged_operators``) treats every interior edge with d_i <= tol * |e_i|
(cocircular neighbours, O_R = O_L, where eq. 3 would divide by zero) by fusing its two
triangles into one cell (B at the common circumcentre, area S_R + S_L) and dropping the edge.
On a square lattice cut by diagonals this yields exactly the Yee scheme.

Parity: pinned by tests/test_oracle_invariants.py (discrete gradient in the kernel of L_E,
adjointness W_E L_B = -(W_B L_E)^T, div E flux) and test_oracle_spectral.py (Yee closed form on
the merged right-split lattice).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import Geometry
from .mesh import Mesh


class Operators:
    def __init__(self, mesh: Mesh, geom: Geometry | None = None):
        geom = geom if geom is not None else Geometry(mesh)
        self.mesh = mesh
        self.geom = geom
        ie = mesh.interior_ids
        self.ie = ie                               # caller ids of the unknown edges
        self.n_ei = ie.size
        self.n_t = mesh.n_tris
        d = geom.d[ie]
        if np.any(~(d > 0)):
            raise ValueError("non-positive dual length |O_R O_L| (mesh is not Delaunay)")
        self.d = d
        self.elen = geom.elen[ie]
        self.S = geom.S
        self.w_E = d * self.elen
        self.w_B = geom.S.copy()
        k = np.arange(self.n_ei)
        R = mesh.R[ie]
        L = mesh.L[ie]
        self.L_B = sp.csr_matrix(
            (np.concatenate([1.0 / d, -1.0 / d]), (np.concatenate([k, k]), np.concatenate([R, L]))),
            shape=(self.n_ei, self.n_t))
        # L_E: only interior edges carry unknowns
        col_of_edge = np.full(mesh.n_edges, -1, np.int64)
        col_of_edge[ie] = k
        rows = np.repeat(np.arange(self.n_t), 3)
        cols = col_of_edge[mesh.tri_edge.reshape(-1)]
        vals = (-mesh.tri_sign * geom.elen[mesh.tri_edge] / geom.S[:, None]).reshape(-1)
        keep = cols >= 0
        self.L_E = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(self.n_t, self.n_ei))
        self.col_of_edge = col_of_edge

    # caller-numbered (all edges) <-> unknowns
    def restrict(self, E_all: np.ndarray) -> np.ndarray:
        return np.asarray(E_all, np.float64)[self.ie]

    def extend(self, E_int: np.ndarray) -> np.ndarray:
        out = np.zeros(self.mesh.n_edges)
        out[self.ie] = E_int
        return out


class MergedOperators:
    """L_B, L_E over cells after fusing triangles across zero-dual edges."""

    def __init__(self, mesh: Mesh, geom: Geometry | None = None, tol: float = 1e-12):
        geom = geom if geom is not None else Geometry(mesh)
        ie_all = mesh.interior_ids
        zero = np.abs(geom.d[ie_all]) <= tol * geom.elen[ie_all]
        # union-find over triangles joined by zero-dual edges
        parent = np.arange(mesh.n_tris)

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        for i in ie_all[zero]:
            a, b = find(mesh.R[i]), find(mesh.L[i])
            if a != b:
                parent[max(a, b)] = min(a, b)
        roots = np.array([find(j) for j in range(mesh.n_tris)])
        cell_ids, cell_of_tri = np.unique(roots, return_inverse=True)
        self.n_c = cell_ids.size
        self.cell_of_tri = cell_of_tri
        self.S = np.bincount(cell_of_tri, weights=geom.S, minlength=self.n_c)
        ie = ie_all[~zero]
        d = geom.d[ie]
        if np.any(~(d > 0)):
            raise ValueError("negative dual length")
        self.ie = ie
        self.n_ei = ie.size
        self.d = d
        self.elen = geom.elen[ie]
        self.w_E = d * self.elen
        self.w_B = self.S
        k = np.arange(self.n_ei)
        R = cell_of_tri[mesh.R[ie]]
        L = cell_of_tri[mesh.L[ie]]
        self.L_B = sp.csr_matrix(
            (np.concatenate([1.0 / d, -1.0 / d]), (np.concatenate([k, k]), np.concatenate([R, L]))),
            shape=(self.n_ei, self.n_c))
        col_of_edge = np.full(mesh.n_edges, -1, np.int64)
        col_of_edge[ie] = k
        rows = cell_of_tri[np.repeat(np.arange(mesh.n_tris), 3)]
        cols = col_of_edge[mesh.tri_edge.reshape(-1)]
        vals = (-mesh.tri_sign * geom.elen[mesh.tri_edge] / self.S[cell_of_tri][:, None]).reshape(-1)
        keep = cols >= 0
        self.L_E = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(self.n_c, self.n_ei))
