"""ue_triangulate (mesh generation, Section 3 and Fig. 5a) against the oracle, on the host.

The constrained Delaunay triangulation is unique where no four nodes are cocircular: there the
library's triangles must equal the oracle's exactly (as sets).  On lattices, where cocircular
quadrilaterals leave a choice of diagonal, both must pass the independent property check.
No GPU is used: the call runs on the host.
"""
import ctypes

import numpy as np
import pytest
from scipy.spatial import Delaunay

import meshgen
from oracle import mesh as om, triangulate as tr
from test_oracle_triangulate import (_zigzag_case, check_cdt, hull_area2, polygon_area2,
                                     square_with_hole)


@pytest.fixture(scope="module")
def ue():
    from paper_1812_01448_gb300 import build
    build.build()
    import paper_1812_01448_gb300 as ue
    return ue


@pytest.mark.parametrize("n", [3, 4, 7, 30, 500])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_clouds_equal_the_oracle(ue, n, seed):
    xy = np.random.default_rng(seed).random((n, 2))
    got, flips = ue.triangulate(xy)
    want, _ = tr.triangulate(xy)
    assert flips == 0
    assert np.array_equal(tr.canonical(got), want)


def test_segments_holes_and_exterior_equal_the_oracle(ue):
    xy, segs = _zigzag_case()
    got, flips = ue.triangulate(xy, segs)
    want, wflips = tr.triangulate(xy, segs)
    assert np.array_equal(tr.canonical(got), want) and flips > 20
    xy, segs, ol, hl = square_with_hole()
    got, _ = ue.triangulate(xy, segs, holes=[[0.5, 0.5]])
    want, _ = tr.triangulate(xy, segs, holes=[[0.5, 0.5]])
    assert np.array_equal(tr.canonical(got), want)
    check_cdt(xy, got, segs, area2=polygon_area2(xy, ol) - polygon_area2(xy, hl))
    # the same square with the hole contour reversed, and a second, empty hole point
    got2, _ = ue.triangulate(xy, segs[:, ::-1], holes=[[0.5, 0.5], [0.6, 0.6]])
    assert np.array_equal(tr.canonical(got2), want)


def test_non_convex_domain(ue):
    corners = [(0, 0), (1, 0), (1, 0.5), (0.5, 0.5), (0.5, 1), (0, 1)]
    loop = []
    for (x0, y0), (x1, y1) in zip(corners, corners[1:] + corners[:1]):
        k = int(round(max(abs(x1 - x0), abs(y1 - y0)) / 0.04))
        loop += [(x0 + (x1 - x0) * i / k, y0 + (y1 - y0) * i / k) for i in range(k)]
    rng = np.random.default_rng(11)
    pts = rng.random((2000, 2)) * 0.96 + 0.02
    pts = pts[~((pts[:, 0] > 0.48) & (pts[:, 1] > 0.48))][:600]
    xy = np.vstack([np.array(loop), pts])
    L = list(range(len(loop)))
    segs = np.array([(a, b) for a, b in zip(L, L[1:] + L[:1])])
    for drop in (False, True):
        got, _ = ue.triangulate(xy, segs, drop_exterior=drop)
        want, _ = tr.triangulate(xy, segs, drop_exterior=drop)
        assert np.array_equal(tr.canonical(got), want), drop
    check_cdt(xy, got, segs, area2=polygon_area2(xy, L))


@pytest.mark.parametrize("shape,h", [((9, 6), 0.1), ((30, 17), 1 / 3), ((4, 50), 0.7)])
def test_lattices_are_valid(ue, shape, h):
    g = np.stack(np.meshgrid(np.arange(shape[0]), np.arange(shape[1])), -1).reshape(-1, 2) * h
    got, _ = ue.triangulate(g)
    assert got.shape[0] == 2 * (shape[0] - 1) * (shape[1] - 1)
    check_cdt(g, got, area2=hull_area2(g))
    # a segment from the corner (0, 0) to the node (sx - 1, 1): it passes through no other
    # node, and the cells it cuts are split along it
    sx = shape[0]
    segs = [[0, sx + sx - 1]]
    got, flips = ue.triangulate(g, segs)
    want, wflips = tr.triangulate(g, segs)
    check_cdt(g, got, segs, area2=hull_area2(g))
    check_cdt(g, want, segs, area2=hull_area2(g))


def test_large_cloud_is_exactly_delaunay(ue):
    """100k random nodes: every triangle that differs from Qhull's must be the exact one (Qhull
    is not exact), and every interior edge passes the in-circle test."""
    xy = np.random.default_rng(12).random((100_000, 2))
    got, _ = ue.triangulate(xy)
    q = Delaunay(xy).simplices
    a = q[:, 0]
    neg = ((xy[q[:, 1], 0] - xy[a, 0]) * (xy[q[:, 2], 1] - xy[a, 1])
           - (xy[q[:, 1], 1] - xy[a, 1]) * (xy[q[:, 2], 0] - xy[a, 0])) < 0
    q[neg] = q[neg][:, [0, 2, 1]]
    G = {tuple(t) for t in tr.canonical(got).tolist()}
    Q = {tuple(t) for t in tr.canonical(q).tolist()}
    diff = sorted(G - Q)
    assert len(G) == len(Q) and len(diff) <= 8
    P = tr._F(xy)
    for t in diff:
        for u in sorted(Q - G):
            for w in u:
                if w not in t:
                    assert tr.incircle(P, *t, w) <= 0
    # every interior edge: the node across it is not inside the triangle's circle (double
    # precision with a margin, and exactly where the margin does not decide)
    t = got.astype(np.int64)
    a, b, c = (t[:, [0, 1, 2]].ravel(), t[:, [1, 2, 0]].ravel(), t[:, [2, 0, 1]].ravel())
    n = xy.shape[0]
    key = a * n + b
    twin = {k: i for i, k in enumerate((b * n + a).tolist())}
    j = np.array([twin.get(k, -1) for k in key.tolist()])
    inner = j >= 0
    d = c[j[inner]]
    A, B, C, D = xy[a[inner]], xy[b[inner]], xy[c[inner]], xy[d]
    ad, bd, cd = A - D, B - D, C - D
    la, lb, lc = (ad ** 2).sum(1), (bd ** 2).sum(1), (cd ** 2).sum(1)
    x = lambda u, v: u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]
    det = la * x(bd, cd) + lb * x(cd, ad) + lc * x(ad, bd)
    perm = la * np.abs(x(bd, cd)) + lb * np.abs(x(cd, ad)) + lc * np.abs(x(ad, bd))
    assert inner.sum() > 2.9 * len(t)
    unsure = np.nonzero(det > -1e-10 * perm)[0]
    ia, ib, ic = a[inner], b[inner], c[inner]
    for k in unsure:
        assert tr.incircle(P, int(ia[k]), int(ib[k]), int(ic[k]), int(d[k])) <= 0


def test_output_loads_as_a_mesh(ue):
    xy, segs, ol, hl = square_with_hole()
    tris, _ = ue.triangulate(xy, segs, holes=[[0.5, 0.5]])
    m = ue.Mesh(xy, tris)
    o = om.canonicalize(xy, tris)
    assert (m.n_tris, m.n_edges) == (o.n_tris, o.n_edges)
    m.close()


def test_fresh_triangulation_equals_lawson_remesh_on_a_convex_cloud(ue):
    """After jello relaxation (the oracle's), a fresh triangulation of the node cloud and the
    Lawson remesh of the relaxed triangulation agree where the boundary is convex."""
    from oracle import relax
    ms = meshgen.random_delaunay(400, seed=13)
    xy, tris, _ = relax.relax(ms.xy, ms.tris, 30, flip_every=0)
    flipped, _ = relax.lawson_flips(xy, tris)
    fresh, _ = ue.triangulate(xy)
    assert np.array_equal(tr.canonical(fresh), tr.canonical(flipped))


@pytest.mark.parametrize("case,code", [("repeat", -3), ("collinear", -3), ("on_segment", -1),
                                       ("crossing", -1), ("hole_outside", -1), ("bad_id", -1)])
def test_invalid_inputs_are_refused_like_the_oracle(ue, case, code):
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 0.5]], float)
    xy, kw = sq, {}
    if case == "repeat":
        xy = np.vstack([sq, sq[2:3]])
    elif case == "collinear":
        xy = np.array([[0, 0], [1, 1], [2, 2], [3, 3.0]])
    elif case == "on_segment":
        kw = dict(segs=[[0, 2]])
    elif case == "crossing":
        xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 0.2]], float)
        kw = dict(segs=[[0, 2], [1, 3]])
    elif case == "hole_outside":
        kw = dict(holes=[[2.0, 2.0]])
    else:
        kw = dict(segs=[[0, 5]])
    with pytest.raises(ue.UEError) as ei:
        ue.triangulate(xy, **kw)
    assert ei.value.code == code
    with pytest.raises(tr.TriangulationError):
        tr.triangulate(xy, **kw)


def test_capacity_and_flags_are_checked(ue):
    from paper_1812_01448_gb300 import _native as N
    xy = np.random.default_rng(14).random((50, 2))
    out = np.empty((10, 3), np.int32)
    nt = ctypes.c_int64()
    rc = N.lib().ue_triangulate(xy.ctypes.data_as(N.PD), 50, None, 0, None, 0, 0,
                                out.ctypes.data_as(N.PI32), 10, ctypes.byref(nt), None)
    assert rc == -1 and nt.value == ue.triangulate(xy)[0].shape[0] > 10
    rc = N.lib().ue_triangulate(xy.ctypes.data_as(N.PD), 50, None, 0, None, 0, 4,
                                out.ctypes.data_as(N.PI32), 10, ctypes.byref(nt), None)
    assert rc == -1


def test_exterior_flag_and_repeated_segments_change_nothing_on_a_closed_hull(ue):
    # every hull edge of the holed square is a segment: dropping the exterior drops nothing,
    # and listing segments twice, either way round, changes nothing
    xy, segs, ol, hl = square_with_hole(seed=15)
    want, _ = ue.triangulate(xy, segs, holes=[[0.5, 0.5]])
    got, _ = ue.triangulate(xy, segs, holes=[[0.5, 0.5]], drop_exterior=True)
    assert np.array_equal(tr.canonical(got), tr.canonical(want))
    twice = np.vstack([segs, segs[::-1, ::-1]])
    got, _ = ue.triangulate(xy, twice, holes=[[0.5, 0.5]])
    assert np.array_equal(tr.canonical(got), tr.canonical(want))
    o, _ = tr.triangulate(xy, twice, holes=[[0.5, 0.5]], drop_exterior=True)
    assert np.array_equal(o, tr.canonical(want))


def test_mesh_flip_equals_the_oracle_lawson_pass(ue):
    """ue_mesh_flip (the relaxation's remesh step) against the oracle's Lawson flips: a scrambled
    Delaunay triangulation comes back; with kept edges, a scrambled constrained triangulation
    comes back to the one flip refinement builds."""
    from oracle import relax
    from test_oracle_relax import _scramble
    ms = meshgen.random_delaunay(300, seed=17)
    bad = _scramble(ms.xy, relax.orient_ccw(ms.xy, ms.tris), 200, seed=3)
    got, flips = ue.mesh_flip(ms.xy, bad)
    want, wflips = relax.lawson_flips(ms.xy, bad)
    assert flips > 0 and np.array_equal(tr.canonical(got), tr.canonical(want))
    assert np.array_equal(tr.canonical(got), tr.canonical(relax.orient_ccw(ms.xy, ms.tris)))
    xy, segs = _zigzag_case(n=200)
    cdt, _ = tr.triangulate(xy, segs)
    bad = _scramble(xy, cdt, 150, seed=5, keep=segs)
    got, flips = ue.mesh_flip(xy, bad, keep=segs)
    assert flips > 0 and np.array_equal(tr.canonical(got), cdt)
    want, _ = relax.lawson_flips(xy, bad, keep=segs)
    assert np.array_equal(tr.canonical(want), cdt)


def test_mesh_flip_refuses_bad_input(ue):
    ms = meshgen.random_delaunay(50, seed=18)
    with pytest.raises(ue.UEError) as ei:
        ue.mesh_flip(ms.xy, ms.tris, keep=[[0, ms.xy.shape[0]]])
    assert ei.value.code == -1
    flat = ms.tris.copy()
    flat[0] = [0, 0, 1]
    with pytest.raises(ue.UEError) as ei:
        ue.mesh_flip(ms.xy, flat)
    assert ei.value.code == -3


def test_mesh_flip_along_the_oracle_relaxation_of_anchored_geometry(ue):
    """At every remesh of the oracle's anchored relaxation (contour nodes anchored, contour
    edges kept), the library's Lawson pass on the same positions gives the oracle's triangles;
    the flip counts may differ, since they depend on the order flips are taken in."""
    import oracle.relax as R
    from test_oracle_relax import ring_case
    xy, t0, ids, segs = ring_case()
    seen = []
    real = R.lawson_flips

    def both(x, t, keep=()):
        a, ka = real(x, t, keep)
        b, _ = ue.mesh_flip(x, t, keep=keep)
        seen.append(np.array_equal(tr.canonical(a), tr.canonical(b)))
        return a, ka

    R.lawson_flips = both
    try:
        R.relax(xy, t0, 60, flip_every=10, anchors=ids, keep=segs)
    finally:
        R.lawson_flips = real
    assert len(seen) == 6 and all(seen)


@pytest.mark.parametrize("case", ["circle", "circle_centre", "collinear_run", "tiny_box", "clusters",
                                  "lattice_diagonal"])
def test_degenerate_and_badly_scaled_clouds(ue, case):
    """Nodes all (nearly) on one circle, a long collinear run, 98 distinct nodes in a 1e-12 box
    at 1000, clusters over twelve orders of magnitude, and lattice cell diagonals as segments:
    the result always has the constrained Delaunay property and covers the hull exactly."""
    a = 2 * np.pi * np.arange(400) / 400
    circle = np.stack([np.cos(a), np.sin(a)], 1)
    x = np.linspace(0, 1, 300)
    r = np.random.default_rng(2)
    segs = ()
    xy = {
        "circle": circle,
        "circle_centre": np.vstack([circle, [[0.0, 0.0]]]),
        "collinear_run": np.vstack([np.stack([x, 0 * x], 1), [[0.3, 0.2], [0.7, -0.1], [0.5, 1e-9]]]),
        "tiny_box": np.unique(np.random.default_rng(1).random((500, 2)) * 1e-12 + 1e3, axis=0),
        "clusters": np.vstack([r.normal(0, 1e-6, (200, 2)), r.normal(5, 1, (200, 2)), r.random((50, 2)) * 1e6]),
        "lattice_diagonal": np.stack(np.meshgrid(np.arange(20), np.arange(20)), -1).reshape(-1, 2) * 0.1,
    }[case]
    if case == "lattice_diagonal":
        segs = [[i * 20 + i, (i + 1) * 20 + i + 1] for i in range(19)]
    got, _ = ue.triangulate(xy, segs)
    check_cdt(xy, got, segs, area2=hull_area2(xy))
    if xy.shape[0] <= 450 and case != "tiny_box":
        want, _ = tr.triangulate(xy, segs)
        check_cdt(xy, want, segs, area2=hull_area2(xy))


def test_mesh_generation_flow_gives_a_mesh_the_scheme_accepts(ue):
    """Section 3's flow: contours seeded at spacing h (the unit square, a square hole, and a
    circular object meshed on both sides), random area nodes, ue_triangulate with flip
    refinement and the hole dropped, then the jello relaxation (the oracle's: the object's
    contour anchored and its edges kept, Lawson remeshes every 10 steps).  The mesh loads,
    both contours are still edges, and every interior edge has a positive dual length (eq. 10
    needs d > 0), so the scheme can step it."""
    from oracle import geometry, relax
    xy0, segs0, ol, hl = square_with_hole(seed=19, n=0)
    h = 0.05
    k = 13
    ang = 2 * np.pi * np.arange(k) / k
    ring = np.stack([0.18 + 0.1 * np.cos(ang), 0.18 + 0.1 * np.sin(ang)], 1)
    rng = np.random.default_rng(19)
    pts = rng.random((3000, 2)) * 0.94 + 0.03
    keep_pt = ~np.all((pts > 0.33) & (pts < 0.67), 1)
    keep_pt &= np.abs(np.linalg.norm(pts - 0.18, axis=1) - 0.1) > 0.4 * h
    pts = pts[keep_pt]
    # thin the cloud to about the seeding spacing: drop nodes closer than 0.6 h to one kept
    # before them (contour nodes first)
    from scipy.spatial import cKDTree
    base = np.vstack([xy0, ring])
    chosen = []
    tree_base = cKDTree(base)
    for p in pts:
        if tree_base.query(p)[0] < 0.6 * h:
            continue
        if chosen and np.min(np.linalg.norm(np.asarray(chosen) - p, axis=1)) < 0.6 * h:
            continue
        chosen.append(p)
    xy = np.vstack([base, np.asarray(chosen)])
    rid = np.arange(len(xy0), len(xy0) + k)
    rsegs = np.stack([rid, np.roll(rid, -1)], 1)
    segs = np.vstack([segs0, rsegs])
    tris, flips = ue.triangulate(xy, segs, holes=[[0.5, 0.5]])
    check_cdt(xy, tris, segs, area2=polygon_area2(xy, ol) - polygon_area2(xy, hl))
    x1, t1, nf = relax.relax(xy, tris, 80, flip_every=10, anchors=rid, keep=rsegs)
    assert np.array_equal(x1[rid], xy[rid]) and np.array_equal(x1[:len(xy0)], xy0)
    edges = {frozenset(e) for r in t1.tolist() for e in ((r[0], r[1]), (r[1], r[2]), (r[2], r[0]))}
    assert all(frozenset((int(u), int(v))) in edges for u, v in segs)
    m = ue.Mesh(x1, t1)
    om_ = om.canonicalize(x1, t1)
    assert (m.n_tris, m.n_edges) == (om_.n_tris, om_.n_edges)
    m.close()
    d = geometry.Geometry(om_).d[om_.interior]
    assert d.min() > 0
