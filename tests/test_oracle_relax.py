"""Jello-model relaxation and flip refinement (Section 3) oracle pins."""
import numpy as np

import meshgen
from oracle import relax


def _mesh_data(ms, h=None):
    t = relax.orient_ccw(ms.xy, ms.tris)
    hn = np.full(ms.xy.shape[0], h if h is not None else relax.uniform_size(ms.xy, t))
    edges, L0, H0 = relax.rest_lengths(t, hn)
    return t, edges, L0, H0


def test_forces_are_minus_the_energy_gradient():
    """Central differences of E against the forces (no node held fixed)."""
    ms = meshgen.random_delaunay(40, seed=3)
    t, edges, L0, H0 = _mesh_data(ms)
    xy = ms.xy.copy()
    F = relax.forces(xy, t, edges, L0, H0, np.zeros(xy.shape[0], bool))
    eps = 1e-6
    G = np.zeros_like(xy)
    for i in range(xy.shape[0]):
        for k in range(2):
            xp = xy.copy(); xp[i, k] += eps
            xm = xy.copy(); xm[i, k] -= eps
            G[i, k] = (relax.energy(xp, t, edges, L0, H0) - relax.energy(xm, t, edges, L0, H0)) / (2 * eps)
    assert np.abs(F + G).max() < 1e-6 * np.abs(G).max()


def test_equilateral_lattice_is_a_fixed_point():
    ms = meshgen.equilateral_lattice(8, 0.1)
    out, t, flips = relax.relax(ms.xy, ms.tris, 20, h_nodes=np.full(ms.xy.shape[0], 0.1), flip_every=5)
    assert np.abs(out - ms.xy).max() < 1e-10 and flips == 0


def test_relaxation_lowers_the_energy_and_restores_the_lattice():
    """A jittered lattice (boundary fixed) flows down E at every step, back towards the lattice."""
    ms = meshgen.equilateral_lattice(10, 0.1, jitter=0.2, seed=4)
    ref = meshgen.equilateral_lattice(10, 0.1).xy
    t, edges, L0, H0 = _mesh_data(ms, 0.1)
    bnd = relax.boundary_nodes(ms.xy.shape[0], t)
    xy = ms.xy.copy()
    E = [relax.energy(xy, t, edges, L0, H0)]
    for _ in range(400):
        xy = relax.relax(xy, t, 1, h_nodes=np.full(xy.shape[0], 0.1))[0]
        E.append(relax.energy(xy, t, edges, L0, H0))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-14 * E[0])
    assert E[-1] < 1e-8 * E[0]
    assert np.abs(xy - ref).max() < 1e-3 * 0.1
    assert np.array_equal(xy[bnd], ms.xy[bnd])


def _scramble(xy, tris, n, seed, keep=()):
    """Random flips of interior edges whose quad is convex (Delaunay or not), never of the
    node-id pairs in `keep`."""
    rng = np.random.default_rng(seed)
    fixed = {frozenset((int(u), int(v))) for u, v in np.asarray(keep, np.int64).reshape(-1, 2)}
    t = [list(r) for r in tris]
    done = 0
    while done < n:
        i = int(rng.integers(len(t)))
        q = int(rng.integers(3))
        a, b = t[i][q], t[i][(q + 1) % 3]
        c = t[i][(q + 2) % 3]
        if frozenset((a, b)) in fixed:
            continue
        js = [j for j in range(len(t)) if j != i and a in t[j] and b in t[j]]
        if not js:
            continue
        j = js[0]
        d = [x for x in t[j] if x != a and x != b][0]
        cr = lambda p, r, s: (xy[r][0] - xy[p][0]) * (xy[s][1] - xy[p][1]) - (xy[r][1] - xy[p][1]) * (xy[s][0] - xy[p][0])
        if cr(a, d, c) <= 0 or cr(d, b, c) <= 0:
            continue
        t[i], t[j] = [a, d, c], [d, b, c]
        done += 1
    return np.asarray(t)


def test_lawson_flips_recover_the_delaunay_triangulation():
    """Qhull's Delaunay triangulation of random points, scrambled by 150 convex flips, comes
    back exactly (as a set of triangles) from Lawson's flips."""
    ms = meshgen.random_delaunay(150, seed=9)
    ref = {tuple(sorted(r)) for r in ms.tris}
    bad = _scramble(ms.xy, relax.orient_ccw(ms.xy, ms.tris), 150, seed=2)
    assert {tuple(sorted(r)) for r in bad} != ref
    out, flips = relax.lawson_flips(ms.xy, bad)
    assert flips > 0
    assert {tuple(sorted(r)) for r in out} == ref


def test_kept_edges_give_the_constrained_delaunay_triangulation():
    """Lawson flips that keep the segments of a zigzag through a cloud, run on a scrambled copy
    of its constrained Delaunay triangulation (built independently, by flip refinement), come
    back to that triangulation; without `keep` they leave it."""
    from oracle import triangulate as tri
    from test_oracle_triangulate import _zigzag_case
    xy, segs = _zigzag_case(n=150)
    cdt, _ = tri.triangulate(xy, segs)
    bad = _scramble(xy, cdt, 120, seed=4, keep=segs)
    assert not np.array_equal(tri.canonical(bad), cdt)
    out, flips = relax.lawson_flips(xy, bad, keep=segs)
    assert flips > 0 and np.array_equal(tri.canonical(out), cdt)
    free, _ = relax.lawson_flips(xy, bad)
    assert np.array_equal(tri.canonical(free), tri.triangulate(xy)[0])


def ring_case():
    """A unit square with a circle of 24 seeded nodes inside (an object's contour, meshed on
    both sides) and 300 random nodes: (xy, its constrained Delaunay triangulation, the contour's
    node ids, the contour's edges)."""
    from oracle import triangulate as tri
    rng = np.random.default_rng(16)
    k = 24
    ang = 2 * np.pi * np.arange(k) / k
    ring = np.stack([0.5 + 0.2 * np.cos(ang), 0.5 + 0.2 * np.sin(ang)], 1)
    pts = rng.random((500, 2)) * 0.96 + 0.02
    pts = pts[np.abs(np.linalg.norm(pts - 0.5, axis=1) - 0.2) > 0.02][:300]
    xy = np.vstack([np.array([[0, 0], [1, 0], [1, 1], [0, 1.0]]), ring, pts])
    ids = np.arange(4, 4 + k)
    segs = np.stack([ids, np.roll(ids, -1)], 1)
    return xy, tri.triangulate(xy, segs)[0], ids, segs


def test_anchored_geometry_stays_put():
    """The ring's nodes anchored and its edges kept: the nodes do not move and the contour
    survives the remesh, while the cloud around it relaxes; unanchored, the contour nodes move."""
    xy, t0, ids, segs = ring_case()
    x1, t1, flips = relax.relax(xy, t0, 60, flip_every=10, anchors=ids, keep=segs)
    assert np.array_equal(x1[ids], xy[ids])
    edges = {frozenset(e) for r in t1 for e in ((r[0], r[1]), (r[1], r[2]), (r[2], r[0]))}
    assert all(frozenset((int(u), int(v))) in edges for u, v in segs)
    moved = np.linalg.norm(x1 - xy, axis=1)
    assert moved[4 + len(ids):].max() > 1e-3 and flips > 0
    x2, _, _ = relax.relax(xy, t0, 60, flip_every=10)
    assert np.linalg.norm(x2[ids] - xy[ids], axis=1).max() > 1e-3
