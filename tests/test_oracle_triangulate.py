"""Pins of the mesh-generation oracle (Section 3, "Mesh generation"; Fig. 5a), CPU only.

The oracle builds its triangulation by a sweep, Lawson flips, flip refinement of the segments
and a second Lawson pass.  These tests hold it to what fixes the answer independently of that
construction: the empty-circumcircle definition by brute force over all triples, Qhull's
triangulation of random clouds, a kite worked by hand, and `check_cdt`, which checks the
constrained Delaunay property directly (every triangle counter-clockwise, each directed edge
used once, every segment an edge, every other interior edge locally Delaunay, every boundary
edge a hull edge or a segment, and the covered area exactly the domain's).  A triangulation with
all of these properties is the constrained Delaunay triangulation.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.spatial import Delaunay

from oracle import triangulate as tr


def _q(xy):
    return [(Fraction(float(x)), Fraction(float(y))) for x, y in np.asarray(xy, np.float64)]


def _cross(P, a, b, c):
    return (P[b][0] - P[a][0]) * (P[c][1] - P[a][1]) - (P[b][1] - P[a][1]) * (P[c][0] - P[a][0])


def _in_circle(P, a, b, c, d):
    m = []
    for v in (a, b, c):
        x, y = P[v][0] - P[d][0], P[v][1] - P[d][1]
        m.append((x, y, x * x + y * y))
    return (m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0])
            - m[1][2] * (m[0][0] * m[2][1] - m[0][1] * m[2][0])
            + m[2][2] * (m[0][0] * m[1][1] - m[0][1] * m[1][0]))


def polygon_area2(xy, loop):
    """Twice the area of a closed CCW polygon (node ids), exactly."""
    P = _q(xy)
    return sum(P[a][0] * P[b][1] - P[b][0] * P[a][1] for a, b in zip(loop, loop[1:] + loop[:1]))


def hull_area2(xy):
    """Twice the area of the convex hull, exactly (Andrew's monotone chain over fractions)."""
    P = sorted(set(_q(xy)))

    def chain(pts):
        h = []
        for p in pts:
            while len(h) >= 2 and ((h[-1][0] - h[-2][0]) * (p[1] - h[-2][1])
                                   - (h[-1][1] - h[-2][1]) * (p[0] - h[-2][0])) <= 0:
                h.pop()
            h.append(p)
        return h

    h = chain(P)[:-1] + chain(P[::-1])[:-1]
    return sum(h[i][0] * h[(i + 1) % len(h)][1] - h[(i + 1) % len(h)][0] * h[i][1] for i in range(len(h)))


def check_cdt(xy, tris, segs=(), area2=None):
    P = _q(xy)
    tris = np.asarray(tris, np.int64).reshape(-1, 3)
    seg = {frozenset((int(u), int(v))) for u, v in np.asarray(segs, np.int64).reshape(-1, 2)}
    owner = {}
    total = Fraction(0)
    for i, (a, b, c) in enumerate(tris.tolist()):
        s = _cross(P, a, b, c)
        assert s > 0, f"triangle {i} is not counter-clockwise"
        total += s
        for e in ((a, b), (b, c), (c, a)):
            assert e not in owner, f"directed edge {e} used twice"
            owner[e] = (a, b, c)
    edges = {frozenset(e) for e in owner}
    for s_ in seg:
        assert s_ in edges, f"segment {tuple(s_)} is not an edge"
    for (a, b), t in owner.items():
        c = next(x for x in t if x != a and x != b)
        if (b, a) in owner:
            if frozenset((a, b)) in seg:
                continue
            d = next(x for x in owner[(b, a)] if x != a and x != b)
            assert _in_circle(P, a, b, c, d) <= 0, f"edge {(a, b)} is not locally Delaunay"
        elif frozenset((a, b)) not in seg:
            assert all(_cross(P, a, b, w) >= 0 for w in range(len(P))), f"boundary edge {(a, b)} is not on the hull"
    if area2 is not None:
        assert total == area2
    return edges


# ------------------------------------------------------------------ the definition


@pytest.mark.parametrize("n", [3, 4, 6, 9, 14, 20])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_delaunay_matches_the_empty_circle_definition(n, seed):
    xy = np.random.default_rng(seed).random((n, 2))
    got, flips = tr.triangulate(xy)
    assert flips == 0
    assert np.array_equal(got, tr.delaunay_brute(xy))
    check_cdt(xy, got, area2=hull_area2(xy))


def test_delaunay_matches_qhull_on_random_clouds():
    for seed in (3, 4):
        xy = np.random.default_rng(seed).random((400, 2))
        got, _ = tr.triangulate(xy)
        q = Delaunay(xy).simplices
        P = _q(xy)
        q = np.array([t if _cross(P, *t) > 0 else t[[0, 2, 1]] for t in q])
        assert np.array_equal(got, tr.canonical(q))


def test_hand_worked_kite():
    # A(0,0) B(4,0) C(2,1) D(2,-1): the circle through A, B, C has centre (2,-1.5) and radius
    # 2.5; D is 0.5 from the centre, inside it, so AB is not Delaunay and the diagonal is CD.
    xy = np.array([[0, 0], [4, 0], [2, 1], [2, -1.0]])
    dt, flips = tr.triangulate(xy)
    assert dt.tolist() == [[0, 3, 2], [1, 2, 3]] and flips == 0
    # AB as a segment: one flip restores it (Fig. 5a), and the quadrilateral stays split on it
    cdt, flips = tr.triangulate(xy, [[0, 1]])
    assert cdt.tolist() == [[0, 1, 2], [0, 3, 1]] and flips == 1
    check_cdt(xy, cdt, [[0, 1]], area2=Fraction(8))


def test_collinear_first_nodes_and_a_lattice():
    # every node of a lattice is cocircular with three others: no unique answer, but the
    # property holds and the count is two triangles per cell
    g = np.stack(np.meshgrid(np.arange(7), np.arange(5)), -1).reshape(-1, 2) * 0.1
    got, _ = tr.triangulate(g)
    assert got.shape[0] == 2 * 6 * 4
    check_cdt(g, got, area2=hull_area2(g))


# ------------------------------------------------------------------ segments


def _zigzag_case(seed=5, n=250):
    rng = np.random.default_rng(seed)
    cloud = rng.random((n, 2))
    line = np.array([[0.05, 0.1], [0.3, 0.9], [0.55, 0.12], [0.8, 0.88], [0.97, 0.2]])
    xy = np.vstack([cloud, line])
    k = np.arange(n, n + len(line))
    return xy, np.stack([k[:-1], k[1:]], 1)


def test_long_segments_through_a_cloud():
    xy, segs = _zigzag_case()
    dt, _ = tr.triangulate(xy)
    cdt, flips = tr.triangulate(xy, segs)
    assert flips > 20                                # many triangles cross each segment
    assert not np.array_equal(cdt, dt)
    check_cdt(xy, cdt, segs, area2=hull_area2(xy))


def test_segments_that_are_delaunay_edges_change_nothing():
    xy = np.random.default_rng(6).random((200, 2))
    dt, _ = tr.triangulate(xy)
    segs = [(int(t[0]), int(t[1])) for t in dt[::12]]
    cdt, flips = tr.triangulate(xy, segs)
    assert flips == 0 and np.array_equal(cdt, dt)


def square_with_hole(seed=7, n=300, h=0.05):
    """Unit square seeded along its sides at spacing h, a square hole [0.35, 0.65]^2 seeded at
    the same spacing, random nodes between them; returns xy, segments, outer loop, hole loop."""
    def loop(x0, x1, k):
        # k nodes per side, counter-clockwise from (x0, x0); every side exactly straight
        s = np.linspace(x0, x1, k + 1)[:-1]
        t = x1 - (s - x0)
        return np.concatenate([np.stack([s, np.full(k, x0)], 1), np.stack([np.full(k, x1), s], 1),
                               np.stack([t, np.full(k, x1)], 1), np.stack([np.full(k, x0), t], 1)])
    outer = loop(0.0, 1.0, int(round(1 / h)))
    hole = loop(0.35, 0.65, int(round(0.3 / h)))
    rng = np.random.default_rng(seed)
    pts = rng.random((4 * n, 2)) * 0.96 + 0.02
    inside = np.all((pts > 0.33) & (pts < 0.67), 1)
    pts = pts[~inside][:n]
    xy = np.vstack([outer, hole, pts])
    no, nh = len(outer), len(hole)
    ol = list(range(no))
    hl = list(range(no, no + nh))
    segs = [(a, b) for a, b in zip(ol, ol[1:] + ol[:1])] + [(a, b) for a, b in zip(hl, hl[1:] + hl[:1])]
    return xy, np.array(segs), ol, hl


def test_square_with_a_hole():
    xy, segs, ol, hl = square_with_hole()
    assert polygon_area2(xy, ol) == 2 and polygon_area2(xy, hl) > 0
    got, _ = tr.triangulate(xy, segs, holes=[[0.5, 0.5]])
    check_cdt(xy, got, segs, area2=polygon_area2(xy, ol) - polygon_area2(xy, hl))
    c = xy[got].mean(1)
    assert not np.any(np.all((c > 0.35) & (c < 0.65), 1))


def test_non_convex_domain_drops_its_exterior():
    # an L: the unit square without [0.5, 1]^2, its contour seeded at spacing 0.05
    h = 0.05
    corners = [(0, 0), (1, 0), (1, 0.5), (0.5, 0.5), (0.5, 1), (0, 1)]
    loop = []
    for (x0, y0), (x1, y1) in zip(corners, corners[1:] + corners[:1]):
        k = int(round(max(abs(x1 - x0), abs(y1 - y0)) / h))
        loop += [(x0 + (x1 - x0) * i / k, y0 + (y1 - y0) * i / k) for i in range(k)]
    rng = np.random.default_rng(8)
    pts = rng.random((600, 2)) * 0.96 + 0.02
    pts = pts[~((pts[:, 0] > 0.48) & (pts[:, 1] > 0.48))][:250]
    xy = np.vstack([np.array(loop), pts])
    L = list(range(len(loop)))
    segs = np.array([(a, b) for a, b in zip(L, L[1:] + L[:1])])
    full, _ = tr.triangulate(xy, segs)
    check_cdt(xy, full, segs, area2=hull_area2(xy))
    got, _ = tr.triangulate(xy, segs, drop_exterior=True)
    check_cdt(xy, got, segs, area2=polygon_area2(xy, L))
    assert polygon_area2(xy, L) == Fraction(3, 2)


# ------------------------------------------------------------------ errors


@pytest.mark.parametrize("case", ["repeat", "collinear", "on_segment", "crossing", "hole_outside"])
def test_invalid_inputs_are_refused(case):
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 0.5]], float)
    kw = {}
    xy = sq
    if case == "repeat":
        xy = np.vstack([sq, sq[2:3]])
    elif case == "collinear":
        xy = np.array([[0, 0], [1, 1], [2, 2], [3, 3.0]])
    elif case == "on_segment":
        kw = dict(segs=[[0, 2]])
    elif case == "crossing":
        xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.5, 0.2]], float)
        kw = dict(segs=[[0, 2], [1, 3]])
    else:
        kw = dict(holes=[[2.0, 2.0]])
    with pytest.raises(tr.TriangulationError):
        tr.triangulate(xy, **kw)
