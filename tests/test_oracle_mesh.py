"""Pins of the oracle's mesh symbols and reordering (CPU only)."""
import json
import os

import numpy as np
import pytest

import meshgen
from oracle import geometry, mesh as om, rcm

GOLD = os.path.join(os.path.dirname(__file__), "golden", "two_triangle.json")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def test_two_triangle_tables_match_hand_worked_values():
    g = _gold()
    m = om.canonicalize(np.array(g["xy"]), np.array(g["tris"]))
    assert m.edges.tolist() == g["edges"]
    assert m.interior.tolist() == g["interior"]
    assert m.tri_edge.tolist() == g["tri_edge"]
    assert m.tri_sign.tolist() == g["tri_sign"]
    assert m.R.tolist() == g["R"]
    assert m.L.tolist() == g["L"]
    O = geometry.circumcentres(m.xy, m.tris)
    np.testing.assert_allclose(O, g["circumcentres"], atol=1e-15)
    np.testing.assert_allclose(geometry.areas(m.xy, m.tris), g["areas"], rtol=1e-15)
    np.testing.assert_allclose(geometry.edge_lengths(m), g["edge_lengths"], rtol=1e-15)


def test_clockwise_input_is_reoriented():
    g = _gold()
    cw = np.array(g["tris"])[:, [0, 2, 1]]
    m = om.canonicalize(np.array(g["xy"]), cw)
    assert m.tri_sign.tolist() == g["tri_sign"]
    assert m.R.tolist() == g["R"] and m.L.tolist() == g["L"]


def test_left_triangle_is_R():
    """R(i) lies to the left of the directed edge (the side its circumcentre is on)."""
    ms = meshgen.random_delaunay(300, seed=5)
    m = om.canonicalize(ms.xy, ms.tris)
    ie = m.interior_ids
    v = geometry.edge_vectors(m)[ie]
    cR = m.xy[m.tris[m.R[ie]]].mean(axis=1) - m.xy[m.edges[ie, 0]]
    cL = m.xy[m.tris[m.L[ie]]].mean(axis=1) - m.xy[m.edges[ie, 0]]
    assert np.all(v[:, 0] * cR[:, 1] - v[:, 1] * cR[:, 0] > 0)
    assert np.all(v[:, 0] * cL[:, 1] - v[:, 1] * cL[:, 0] < 0)


@pytest.mark.parametrize("tris,code", [
    ([[0, 1, 4]], om.ERR_ARG),                               # index out of range
    ([[0, 1, 1]], om.ERR_DEGENERATE),                        # repeated vertex
    ([[0, 1, 2], [0, 1, 3]], om.ERR_NONMANIFOLD),             # two triangles on one side
])
def test_invalid_meshes_are_rejected(tris, code):
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    with pytest.raises(om.MeshError) as ei:
        om.canonicalize(xy, np.array(tris))
    assert ei.value.code == code


def test_collinear_triangle_is_degenerate():
    xy = np.array([[0, 0], [1, 0], [2, 0]], float)
    with pytest.raises(om.MeshError) as ei:
        om.canonicalize(xy, np.array([[0, 1, 2]]))
    assert ei.value.code == om.ERR_DEGENERATE


def test_three_triangles_on_one_edge_is_nonmanifold():
    xy = np.array([[0, 0], [1, 0], [0.5, 1], [0.5, -1], [0.5, 2]], float)
    with pytest.raises(om.MeshError) as ei:
        om.canonicalize(xy, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    assert ei.value.code == om.ERR_NONMANIFOLD


def test_rcm_on_a_strip_is_the_reversed_path():
    """One row of diagonal-cut squares: the dual graph is a path t1-t0-t3-t2-t5-t4-..."""
    ms = meshgen.right_split_lattice(7, 2, 6.0, 1.0)
    m = om.canonicalize(ms.xy, ms.tris)
    order = rcm.rcm_order(m)
    path = [1, 0]
    for c in range(1, 6):
        path += [2 * c + 1, 2 * c]
    # both ends have degree 1; the start is the end with the smaller id (t1)
    assert order.tolist() == path[::-1]


def test_rcm_is_a_permutation_and_reduces_bandwidth():
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=3)
    rng = np.random.default_rng(0)
    shuffle = rng.permutation(ms.n_tris)
    m = om.canonicalize(ms.xy, ms.tris[shuffle])
    order = rcm.rcm_order(m)
    assert np.array_equal(np.sort(order), np.arange(m.n_tris))
    t = rcm.device_tables(m, order)
    bw = np.abs(t["edge_tri"][:, 0] - t["edge_tri"][:, 1]).max()
    ie = m.interior_ids
    bw0 = np.abs(m.R[ie] - m.L[ie]).max()
    assert bw < bw0 / 4


def test_device_tables_are_consistent():
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=4)
    m = om.canonicalize(ms.xy, ms.tris)
    order = rcm.rcm_order(m)
    t = rcm.device_tables(m, order)
    n_ei = t["n_ei"]
    code = t["tri_code"]
    k = code >> 1
    neg = code & 1
    # every interior edge appears exactly twice, once with each sign, at R and at L
    inner = k < n_ei
    assert np.bincount(k[inner], minlength=n_ei).tolist() == [2] * n_ei
    rows = np.repeat(np.arange(m.n_tris), 3).reshape(-1, 3)
    R = t["edge_tri"][:, 0]
    L = t["edge_tri"][:, 1]
    assert np.all(R[k[inner & (neg == 0)]] == rows[inner & (neg == 0)])
    assert np.all(L[k[inner & (neg == 1)]] == rows[inner & (neg == 1)])
    # vertex rotation: smallest caller node id first, still counter-clockwise
    tv = t["tri_nodes"]
    assert np.all(tv[:, 0] < tv[:, 1]) and np.all(tv[:, 0] < tv[:, 2])
    assert np.all(om.orient2d(m.xy, tv) > 0)
    # interior edges sorted by (min, max) new triangle id
    lo = np.minimum(R, L)
    hi = np.maximum(R, L)
    key = lo * m.n_tris + hi
    assert np.all(np.diff(key) > 0)


def _parts(order, offs):
    return [order[offs[p]:offs[p + 1]] for p in range(len(offs) - 1)]


def _connected(m, ids):
    nbr = rcm.dual_adjacency(m)
    inside = set(int(i) for i in ids)
    seen, stack = {int(ids[0])}, [int(ids[0])]
    while stack:
        u = stack.pop()
        for w in nbr[u]:
            if w in inside and w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == len(inside)


def test_greedy_on_a_strip_cuts_consecutive_segments():
    """On a strip the dual graph is a path and every triangle has at most two neighbours, so
    the sharpest triangle is always the end of what is left: parts are consecutive segments of
    target = T - T//8 triangles in RCM order; a last segment of fewer than T//8 triangles joins
    the one before it (room for it by construction); no triangle can hang (degree < 3)."""
    ms = meshgen.right_split_lattice(30, 2, 29.0, 1.0)          # 58 triangles
    m = om.canonicalize(ms.xy, ms.tris)
    r = rcm.rcm_order(m)
    order, offs = rcm.greedy_order(m, r, 32)                     # target 28, theta 4
    assert order.tolist() == r.tolist()
    assert offs.tolist() == [0, 28, 58]                          # 28 + 28 + 2, the 2 joined
    assert rcm.shared_edges(m, order, offs) == 1
    order, offs = rcm.greedy_order(m, r, 16)                     # target 14, theta 2
    assert offs.tolist() == [0, 14, 28, 42, 56, 58]              # last 2 >= theta: kept
    assert rcm.shared_edges(m, order, offs) == 4                 # 5 segments of a path


def _holed():
    return meshgen.graded_square(0.01, 0.03, grade=0.3,
                                 holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=9)


@pytest.mark.parametrize("tile", [16, 64, 333])
def test_greedy_parts_are_connected_capped_and_without_hanging_triangles(tile):
    ms = _holed()
    m = om.canonicalize(ms.xy, ms.tris)
    order, offs = rcm.greedy_order(m, rcm.rcm_order(m), tile)
    assert np.array_equal(np.sort(order), np.arange(m.n_tris))
    sizes = np.diff(offs)
    assert sizes.min() >= 1 and sizes.max() <= tile
    part = np.empty(m.n_tris, np.int64)
    for p, ids in enumerate(_parts(order, offs)):
        assert _connected(m, ids), (tile, p)
        part[ids] = p
    # no triangle left hanging on a part that still has room
    for u, ws in enumerate(rcm.dual_adjacency(m)):
        if len(ws) != 3:
            continue
        other = [int(part[w]) for w in ws if part[w] != part[u]]
        if len(other) == 2 and other[0] == other[1]:
            assert sizes[other[0]] == tile
    # shared boundary from its definition: edges whose two triangles sit in different parts
    cut = sum(1 for i in m.interior_ids if part[m.R[i]] != part[m.L[i]])
    assert rcm.shared_edges(m, order, offs) == cut


def test_greedy_hanging_refinement_cuts_shared_edges():
    """Moving a hanging triangle turns its two edges on Q into inner edges and its one edge on
    its own part into a shared one: each move removes one shared edge, so the refined partition
    never shares more edges than the parts before the sweep.  The unrefined parts are rebuilt
    here from the growth rules alone (no joins happen at this size on this mesh)."""
    ms = _holed()
    m = om.canonicalize(ms.xy, ms.tris)
    r = rcm.rcm_order(m)
    order, offs = rcm.greedy_order(m, r, 64)
    refined = rcm.shared_edges(m, order, offs)
    # growth only: the hanging and small-part steps switched off by a tile cap they never meet
    nbr = rcm.dual_adjacency(m)
    pos = np.empty(m.n_tris, np.int64)
    pos[r] = np.arange(m.n_tris)
    part = np.full(m.n_tris, -1)
    free = np.array([len(a) for a in nbr])
    pid = 0
    while (part < 0).any():
        c = np.flatnonzero((part < 0) & (free < 3))
        root = int(c[np.lexsort((pos[c], free[c]))[0]])
        grown, front = [root], [root]
        part[root] = pid
        for w in nbr[root]:
            free[w] -= 1
        while front and len(grown) < 56:
            u = front.pop(0)
            for w in sorted(nbr[u], key=lambda x: pos[x]):
                if len(grown) < 56 and part[w] < 0:
                    part[w] = pid
                    grown.append(w)
                    front.append(w)
                    for x in nbr[w]:
                        free[x] -= 1
        pid += 1
    raw = sum(1 for i in m.interior_ids if part[m.R[i]] != part[m.L[i]])
    assert refined < raw


def test_greedy_and_kd_share_about_the_same_boundary():
    """Fig. 6: at nearly the same number of parts KD and greedy give nearly the same shared
    boundary; greedy reaches part counts that are not powers of two."""
    ms = meshgen.cavity_lattice(65, 33, 1.0, 0.5, jitter=0.2, seed=4)
    m = om.canonicalize(ms.xy, ms.tris)
    r = rcm.rcm_order(m)
    ko, koffs = rcm.kd_order(m, r, 256)
    n_kd = len(koffs) - 1
    tile = int(round(m.n_tris / n_kd * 8 / 7))
    go, goffs = rcm.greedy_order(m, r, tile)
    n_gr = len(goffs) - 1
    assert abs(n_gr - n_kd) <= n_kd // 4
    lk, lg = rcm.shared_edges(m, ko, koffs), rcm.shared_edges(m, go, goffs)
    assert 0.67 * lk < lg < 1.5 * lk, (lk, lg)
    _, o3 = rcm.greedy_order(m, r, 200)
    n3 = len(o3) - 1
    assert n3 & (n3 - 1) != 0


def test_kd_splits_along_the_longer_side():
    """Median splits along the longer side of the parts' centroid box: on a long thin lattice
    (16 x 2 squares) four KD parts are disjoint slabs in x, each a quarter of the triangles,
    sharing only the 2 edges that each of the three cuts crosses."""
    ms = meshgen.right_split_lattice(17, 3, 16.0, 2.0)      # 64 triangles
    m = om.canonicalize(ms.xy, ms.tris)
    order, offs = rcm.kd_order(m, rcm.rcm_order(m), 16)
    assert offs.tolist() == [0, 16, 32, 48, 64]
    cx = m.xy[m.tris].mean(axis=1)[:, 0]
    spans = [(cx[order[a:b]].min(), cx[order[a:b]].max()) for a, b in zip(offs[:-1], offs[1:])]
    spans.sort()
    assert all(spans[i][1] < spans[i + 1][0] for i in range(3))
    # each cut crosses the strip's 2 rows of squares: 2 vertical edges per cut
    assert rcm.shared_edges(m, order, offs) == 3 * 2
