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
