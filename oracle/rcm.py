"""Locality reordering and the device connectivity tables (oracle; test infrastructure only).

The paper's "Divide and conqueror" section motivates keeping neighbouring triangles together in
memory (KD parts, shared-boundary length).  Within one mesh the library orders triangles by
reverse Cuthill-McKee on the dual graph (triangles joined by interior edges).  The paper gives
no tie-break rules; the ones used here (and, independently, by the library) are:

* components in increasing order of their smallest caller triangle id;
* the start of a component is its triangle of minimum (degree, caller id), degree = number of
  interior edges;
* breadth-first: each dequeued triangle appends its unvisited neighbours sorted by
  (degree, caller id);
* the concatenated order is reversed at the end.

For the temporally blocked variant the triangles are further grouped into KD parts
(``kd_order``) or greedy parts (``greedy_order``), keeping the RCM order inside each part.

From an order the tables follow (same definitions in the library, separate code):

* ``perm_tri[new] = caller triangle id``;
* each triangle's CCW vertex triple is rotated so that its smallest caller node id comes first;
  its edges A(j, q) are then (v_q, v_q+1);
* interior edges are numbered by (min, max) of their two new triangle ids;
  ``edge_caller[k]`` = caller edge id, ``edge_tri[k] = (R, L)`` in new triangle ids;
* ``tri_code[j, q] = 2 k + (s(j,q) < 0)`` for an interior edge k, ``2 n_ei`` for a boundary edge
  (a slot whose value stays 0).

Parity: pinned by tests/test_oracle_mesh.py (valid permutation, contiguous components, a strip
whose RCM order is known in closed form, bandwidth not above the caller order's on lattices; for
the greedy partition: on a strip the parts are consecutive segments of known sizes with the short
last one joined, parts are connected and capped with no hanging triangle left where its
neighbour has room, and at nearly KD's part count the shared boundary is close to KD's, Fig. 6).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .mesh import Mesh


def dual_adjacency(mesh: Mesh):
    nbr = [[] for _ in range(mesh.n_tris)]
    for i in mesh.interior_ids:
        r, l = int(mesh.R[i]), int(mesh.L[i])
        nbr[r].append(l)
        nbr[l].append(r)
    return nbr


def rcm_order(mesh: Mesh) -> np.ndarray:
    nbr = dual_adjacency(mesh)
    deg = [len(a) for a in nbr]
    n = mesh.n_tris
    seen = [False] * n
    order = []
    for root in range(n):
        if seen[root]:
            continue
        # collect the component to find its start vertex
        comp = [root]
        seen[root] = True
        k = 0
        while k < len(comp):
            for w in nbr[comp[k]]:
                if not seen[w]:
                    seen[w] = True
                    comp.append(w)
            k += 1
        for v in comp:
            seen[v] = False
        start = min(comp, key=lambda v: (deg[v], v))
        q = deque([start])
        seen[start] = True
        while q:
            v = q.popleft()
            order.append(v)
            for w in sorted((w for w in nbr[v] if not seen[w]), key=lambda w: (deg[w], w)):
                seen[w] = True
                q.append(w)
    return np.asarray(order[::-1], np.int64)


def kd_order(mesh: Mesh, rcm: np.ndarray, tile_tris: int):
    """KD partition of the "Divide and conqueror" section: split a part at the median of its
    triangle centroids along the longer side of their bounding box (ties by RCM position)
    until it has at most tile_tris triangles.  Parts in depth-first order (left first), RCM
    order inside a part.  Returns (order, tile offsets)."""
    t = mesh.tris
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    cx = (x[t[:, 0]] + x[t[:, 1]] + x[t[:, 2]]) / 3.0
    cy = (y[t[:, 0]] + y[t[:, 1]] + y[t[:, 2]]) / 3.0
    pos = np.empty(mesh.n_tris, np.int64)
    pos[rcm] = np.arange(mesh.n_tris)
    order, offs = [], [0]

    def part(ids):
        if ids.size <= tile_tris:
            order.extend(ids[np.argsort(pos[ids], kind="stable")].tolist())
            offs.append(len(order))
            return
        ex = cx[ids].max() - cx[ids].min()
        ey = cy[ids].max() - cy[ids].min()
        key = cx if ex >= ey else cy
        srt = ids[np.lexsort((pos[ids], key[ids]))]
        mid = ids.size // 2
        part(srt[:mid])
        part(srt[mid:])

    part(np.asarray(rcm, np.int64))
    return np.asarray(order, np.int64), np.asarray(offs, np.int64)


def greedy_order(mesh: Mesh, rcm: np.ndarray, tile_tris: int):
    """Greedy partition of the "Divide and conqueror" section, with its two refinements.
    Returns (order, tile offsets); no part holds more than tile_tris triangles.

    Readings (the paper states the ideas, not the rules):
    * a part is grown from its root, breadth first, each triangle taken from the front adding
      its unassigned neighbours in RCM order, up to tile_tris - tile_tris // 8 triangles (room
      left for the refinements) or until the front is empty;
    * the next root is the "sharpest" triangle on the boundary of what is assigned (or of the
      mesh): the unassigned triangle with the fewest unassigned neighbours, counting only those
      with fewer than three, ties by RCM position;
    * a part of fewer than theta = tile_tris // 8 triangles joins its smallest neighbouring part
      of at least theta triangles that has room for it (ties by part index); parts are visited in
      creation order;
    * a "hanging" triangle (one edge on its own part, its two other edges on one other part Q)
      moves to Q when Q has room; sweeps over the triangles in RCM order, moving as found, repeat
      until one moves nothing;
    * parts are laid out in creation order, RCM order inside each."""
    n = mesh.n_tris
    nbr = dual_adjacency(mesh)
    pos = np.empty(n, np.int64)
    pos[rcm] = np.arange(n)
    nbr = [sorted(a, key=lambda w: pos[w]) for a in nbr]
    theta = tile_tris // 8
    target = tile_tris - theta

    part = np.full(n, -1, np.int64)
    n_free = np.array([len(a) for a in nbr], np.int64)
    parts = []
    while (part < 0).any():
        cand = np.flatnonzero((part < 0) & (n_free < 3))
        if cand.size:
            root = int(cand[np.lexsort((pos[cand], n_free[cand]))[0]])
        else:
            free = np.flatnonzero(part < 0)
            root = int(free[np.argmin(pos[free])])
        pid = len(parts)
        grown = []

        def eat(u):
            part[u] = pid
            grown.append(u)
            for w in nbr[u]:
                n_free[w] -= 1

        eat(root)
        front = deque([root])
        while front and len(grown) < target:
            u = front.popleft()
            for w in nbr[u]:
                if len(grown) >= target:
                    break
                if part[w] < 0:
                    eat(w)
                    front.append(w)
        parts.append(grown)

    size = [len(g) for g in parts]
    for pid, grown in enumerate(parts):
        if size[pid] == 0 or size[pid] >= theta:
            continue
        touching = {int(part[w]) for u in grown for w in nbr[u]} - {pid}
        ok = [q for q in touching if size[q] >= theta and size[q] + size[pid] <= tile_tris]
        if not ok:
            continue
        q = min(ok, key=lambda r: (size[r], r))
        part[grown] = q
        size[q] += size[pid]
        size[pid] = 0

    while True:
        moves = 0
        for u in rcm:
            if len(nbr[u]) != 3:
                continue
            own = int(part[u])
            others = [int(part[w]) for w in nbr[u] if part[w] != own]
            if len(others) == 2 and others[0] == others[1] and size[others[0]] < tile_tris:
                part[u] = others[0]
                size[own] -= 1
                size[others[0]] += 1
                moves += 1
        if moves == 0:
            break

    order, offs = [], [0]
    for pid in range(len(parts)):
        ids = np.flatnonzero(part == pid)
        if ids.size:
            order.extend(ids[np.argsort(pos[ids])].tolist())
            offs.append(len(order))
    return np.asarray(order, np.int64), np.asarray(offs, np.int64)


def shared_edges(mesh: Mesh, order: np.ndarray, offs: np.ndarray) -> int:
    """Interior edges whose two triangles lie in different parts: the shared boundary length
    l_Sigma of Fig. 6, counted in edges."""
    tile = np.empty(mesh.n_tris, np.int64)
    for p in range(len(offs) - 1):
        tile[order[offs[p]:offs[p + 1]]] = p
    ii = mesh.interior_ids
    return int(np.count_nonzero(tile[mesh.R[ii]] != tile[mesh.L[ii]]))


def device_tables(mesh: Mesh, perm_tri: np.ndarray):
    """Connectivity tables for a given triangle order (see module docstring)."""
    n_t = mesh.n_tris
    new_of = np.empty(n_t, np.int64)
    new_of[perm_tri] = np.arange(n_t)
    tv = mesh.tris[perm_tri]
    rot = np.argmin(tv, axis=1)
    idx = (rot[:, None] + np.arange(3)[None, :]) % 3
    tv = np.take_along_axis(tv, idx, axis=1)
    te = np.take_along_axis(mesh.tri_edge[perm_tri], idx, axis=1)
    ts = np.take_along_axis(mesh.tri_sign[perm_tri], idx, axis=1)
    ie = mesh.interior_ids
    r = new_of[mesh.R[ie]]
    l = new_of[mesh.L[ie]]
    lo = np.minimum(r, l)
    hi = np.maximum(r, l)
    o = np.lexsort((hi, lo))
    edge_caller = ie[o]
    edge_tri = np.stack([r[o], l[o]], axis=1)
    n_ei = ie.size
    k_of_edge = np.full(mesh.n_edges, n_ei, np.int64)
    k_of_edge[edge_caller] = np.arange(n_ei)
    k = k_of_edge[te]
    code = 2 * k + ((ts < 0) & (k < n_ei))
    return dict(perm_tri=perm_tri.astype(np.int64), tri_nodes=tv, edge_caller=edge_caller,
                edge_tri=edge_tri, tri_code=code, n_ei=n_ei)
