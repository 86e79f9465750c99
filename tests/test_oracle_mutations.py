"""Planted mistakes in copies of the oracle (CPU only): each plausible slip must fail the pin
that guards it, so that the pins are known to see it.  The oracle itself is not modified: the
mutant is compiled from its source with one textual change."""
import inspect
import math
import textwrap

import numpy as np

import meshgen
from oracle import mesh as om, operators, pml, rcm, spectral


def _mutant(obj, old: str, new: str):
    """obj (function or class) recompiled from its source with `old` replaced by `new`."""
    src = textwrap.dedent(inspect.getsource(obj))
    assert src.count(old) == 1, old
    ns = dict(vars(inspect.getmodule(obj)))
    exec(compile(src.replace(old, new), f"<mutant of {obj.__name__}>", "exec"), ns)
    return ns[obj.__name__]


def test_greedy_small_part_join_is_pinned():
    """Dropping the join of small parts leaves the strip's 2-triangle tail as its own part."""
    bad = _mutant(rcm.greedy_order, "if size[pid] == 0 or size[pid] >= theta:",
                  "if True:")
    ms = meshgen.right_split_lattice(30, 2, 29.0, 1.0)
    m = om.canonicalize(ms.xy, ms.tris)
    order, offs = bad(m, rcm.rcm_order(m), 32)
    assert offs.tolist() != [0, 28, 58]


def _yee_error(cls):
    h, nx, ny = 0.125, 9, 7
    ms = meshgen.right_split_lattice(nx, ny, (nx - 1) * h, (ny - 1) * h)
    m = om.canonicalize(ms.xy, ms.tris)
    fo = cls(m, 3, sigma_max=0.0, inner=operators.MergedOperators(m))
    lam = np.sort(np.linalg.eigvalsh(spectral.symmetric_K(fo)))
    M, N = np.meshgrid(np.arange(fo.NX), np.arange(fo.NY))
    yee = np.sort(((4 / h ** 2) * (np.sin(M * np.pi / (2 * fo.NX)) ** 2
                                   + np.sin(N * np.pi / (2 * fo.NY)) ** 2)).ravel())
    return np.abs(lam - yee).max() / yee.max()


def test_frame_interface_dual_length_is_pinned():
    """The interface edge's dual length with the frame cell's half counted twice
    (d = (O - C) . n + h) breaks Yee's closed form for the framed lattice."""
    assert _yee_error(pml.FramedOperators) < 1e-12
    bad = _mutant(pml.FramedOperators, "d = float(np.dot(geom.O[t] - C, nin) + 0.5 * h)",
                  "d = float(np.dot(geom.O[t] - C, nin) + 1.0 * h)")
    assert _yee_error(bad) > 1e-3


def test_frame_interface_sign_is_pinned():
    """The frame cell taking the triangle's orientation sign for the shared edge (instead of
    the opposite one) breaks the adjointness of the coupled operators."""
    bad = _mutant(pml.FramedOperators, "iface_of[(fc, s)] = (n_ie + k, -1.0 if tri_is_R else 1.0, el)",
                  "iface_of[(fc, s)] = (n_ie + k, 1.0 if tri_is_R else -1.0, el)")
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0, seed=5)
    m = om.canonicalize(ms.xy, ms.tris)
    for cls, ok in ((pml.FramedOperators, True), (bad, False)):
        fo = cls(m, 4, sigma_max=0.0)
        LB, LE = fo.L_B.toarray(), fo.L_E.toarray()
        adj = np.abs(fo.w_E[:, None] * LB + (fo.w_B[:, None] * LE).T).max() / np.abs(LB).max()
        assert (adj < 1e-12) == ok


def test_framed_plasma_drain_sign_is_pinned():
    """A current that feeds E instead of draining it breaks the static-field closed form."""
    bad = _mutant(pml.step_plasma, "E[:ni] -= dt * j", "E[:ni] += dt * j")
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0, seed=5)
    m = om.canonicalize(ms.xy, ms.tris)
    fo = pml.FramedOperators(m, 4)
    rng = np.random.default_rng(6)
    bnd = np.zeros(m.n_nodes, bool)
    bnd[m.edges[~m.interior].ravel()] = True
    phi = np.where(bnd, 0.0, rng.standard_normal(m.n_nodes))
    e = m.edges[fo.inner.ie]
    E0 = np.zeros(fo.n_ei)
    E0[:fo.inner.n_ei] = (phi[e[:, 1]] - phi[e[:, 0]]) / fo.inner.elen
    n0 = 3.0e3
    rho, _ = spectral.power_iteration(fo, 300)
    dt = 0.5 * 2.0 / math.sqrt(rho * rho + n0)
    nbar = pml.inner_nbar(fo, np.full(m.n_nodes, n0))

    def resid(step):
        E, Bs, j = E0.copy(), np.zeros(fo.n_s), np.zeros(fo.inner.n_ei)
        hist = [E.copy()]
        for k in range(20):
            E, Bs, j = step(fo, E, Bs, j, dt, nbar, 0.0, n=k)
            hist.append(E.copy())
        H = np.asarray(hist)
        return np.abs(H[2:] + H[:-2] - (2.0 - n0 * dt * dt) * H[1:-1]).max() / np.abs(H).max()

    assert resid(pml.step_plasma) < 1e-12
    assert resid(bad) > 1e-6


def test_greedy_hanging_refinement_is_pinned():
    """Without the hanging-triangle moves, triangles hanging on a neighbouring part that has room
    are left: the invariant the holed-mesh test checks."""
    bad = _mutant(rcm.greedy_order,
                  "if len(others) == 2 and others[0] == others[1] and size[others[0]] < tile_tris:",
                  "if False:")

    def hanging_with_room(fn):
        ms = meshgen.graded_square(0.01, 0.03, grade=0.3,
                                   holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=9)
        m = om.canonicalize(ms.xy, ms.tris)
        order, offs = fn(m, rcm.rcm_order(m), 64)
        sizes = np.diff(offs)
        part = np.empty(m.n_tris, np.int64)
        for p in range(len(offs) - 1):
            part[order[offs[p]:offs[p + 1]]] = p
        n = 0
        for u, ws in enumerate(rcm.dual_adjacency(m)):
            other = [int(part[w]) for w in ws if part[w] != part[u]]
            if len(ws) == 3 and len(other) == 2 and other[0] == other[1] and sizes[other[0]] < 64:
                n += 1
        return n

    assert hanging_with_room(rcm.greedy_order) == 0
    assert hanging_with_room(bad) > 0


def test_relax_height_spring_sign_is_pinned():
    """A height spring that pushes the apex the wrong way is not -grad E."""
    from oracle import relax
    bad = _mutant(relax.forces, "np.add.at(F, v, -g)", "np.add.at(F, v, g)")
    ms = meshgen.random_delaunay(40, seed=3)
    t = relax.orient_ccw(ms.xy, ms.tris)
    h = np.full(ms.xy.shape[0], relax.uniform_size(ms.xy, t))
    edges, L0, H0 = relax.rest_lengths(t, h)
    xy = ms.xy.copy()
    eps = 1e-6
    G = np.zeros_like(xy)
    for i in range(xy.shape[0]):
        for k in range(2):
            xp = xy.copy(); xp[i, k] += eps
            xm = xy.copy(); xm[i, k] -= eps
            G[i, k] = (relax.energy(xp, t, edges, L0, H0) - relax.energy(xm, t, edges, L0, H0)) / (2 * eps)
    free = np.zeros(xy.shape[0], bool)
    for fn, ok in ((relax.forces, True), (bad, False)):
        F = fn(xy, t, edges, L0, H0, free)
        assert (np.abs(F + G).max() < 1e-6 * np.abs(G).max()) == ok


def test_triangle_operator_sign_is_pinned():
    """L_E with the orientation signs flipped breaks the adjointness of eq. 10."""
    bad = _mutant(operators.Operators, "vals = (-mesh.tri_sign * geom.elen[mesh.tri_edge] / geom.S[:, None]).reshape(-1)",
                  "vals = (mesh.tri_sign * geom.elen[mesh.tri_edge] / geom.S[:, None]).reshape(-1)")
    ms = meshgen.cavity_te11_mesh()
    m = om.canonicalize(ms.xy, ms.tris)
    for cls, ok in ((operators.Operators, True), (bad, False)):
        o = cls(m)
        A = (o.L_B.multiply(o.w_E[:, None])).tocsr()
        Bm = (o.L_E.multiply(o.w_B[:, None])).T.tocsr()
        assert (np.abs((A + Bm).toarray()).max() <= 1e-15 * np.abs(A.toarray()).max()) == ok


def _small_ops():
    ms = meshgen.cavity_lattice(9, 5, 1.0, 0.5, jitter=0.2, dual_floor=0.05, seed=7)
    return ms, operators.Operators(om.canonicalize(ms.xy, ms.tris))


def test_source_time_is_pinned():
    """Evaluating the soft source at n dt instead of (n + 1/2) dt changes the first step."""
    from oracle import leapfrog as lf
    bad = _mutant(lf.step, "t = (st.n + 0.5) * dt", "t = st.n * dt")
    ms, ops = _small_ops()
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    src = lf.Source(ids, amp, 2 * math.pi * 3, 0.2, 0.1)
    dt = 1e-3
    g = math.sin(src.omega0 * 0.5 * dt) * math.exp(-((0.5 * dt - 0.2) / 0.1) ** 2)
    exp = np.zeros(ops.mesh.n_edges)
    exp[ids] = dt * amp * g
    for fn, ok in ((lf.step, True), (bad, False)):
        E = ops.extend(fn(ops, lf.initial_state(ops), dt, source=src).E)
        assert np.allclose(E, exp, rtol=1e-15, atol=0) == ok


def test_power_iteration_metric_is_pinned():
    """A Rayleigh quotient without the S metric of eq. 7 is no longer a lower bound on the
    dense rho (the operator is self-adjoint only in that metric)."""
    bad = _mutant(spectral.power_iteration, "lam = float(np.dot(S * v, w))", "lam = float(np.dot(v, w))")
    ms, ops = _small_ops()
    rho_dense = spectral.dense_rho(ops)
    good, _ = spectral.power_iteration(ops, 200, seed=3)
    assert rho_dense * (1 - 2e-3) <= good <= rho_dense * (1 + 1e-12)
    worse, _ = bad(ops, 200, seed=3)
    assert not (rho_dense * (1 - 2e-3) <= worse <= rho_dense * (1 + 1e-12))


def _kd_slabs_ok(kd):
    ms = meshgen.right_split_lattice(17, 3, 16.0, 2.0)
    m = om.canonicalize(ms.xy, ms.tris)
    order, offs = kd(m, rcm.rcm_order(m), 16)
    cx = m.xy[m.tris].mean(axis=1)[:, 0]
    spans = sorted((cx[order[a:b]].min(), cx[order[a:b]].max()) for a, b in zip(offs[:-1], offs[1:]))
    return (offs.tolist() == [0, 16, 32, 48, 64] and all(spans[i][1] < spans[i + 1][0] for i in range(3))
            and rcm.shared_edges(m, order, offs) == 6)


def test_kd_split_axis_is_pinned():
    """Splitting along the SHORTER side of the centroid box breaks the slab pin."""
    assert _kd_slabs_ok(rcm.kd_order)
    bad = _mutant(rcm.kd_order, "key = cx if ex >= ey else cy", "key = cy if ex >= ey else cx")
    assert not _kd_slabs_ok(bad)


def test_rcm_start_rule_is_pinned():
    """Starting a component at its triangle of MAXIMUM degree breaks the strip's closed form."""
    bad = _mutant(rcm.rcm_order, "start = min(comp, key=lambda v: (deg[v], v))",
                  "start = max(comp, key=lambda v: (deg[v], -v))")
    ms = meshgen.right_split_lattice(7, 2, 6.0, 1.0)
    m = om.canonicalize(ms.xy, ms.tris)
    path = [1, 0]
    for c in range(1, 6):
        path += [2 * c + 1, 2 * c]
    assert rcm.rcm_order(m).tolist() == path[::-1]
    assert bad(m).tolist() != path[::-1]


def test_mlp_backward_layer_transpose_is_pinned():
    """Back-propagating through W2 transposed (d2 @ W2.T) is caught by central differences of
    the first layer's gradient."""
    from oracle import mlp
    bad = _mutant(mlp.backward, "d1 = (d2 @ W2) * (a1 > 0)", "d1 = (d2 @ W2.T) * (a1 > 0)")
    rng = np.random.default_rng(0)
    p = mlp.init_params(3) + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((7, 12))
    c = rng.standard_normal(7)
    z, cache = mlp.forward(p, X)
    idx = range(0, 64 * 12, 37)                       # entries of W1
    h = 1e-6

    def worst(back):
        g = back(p, cache, c)
        err = 0.0
        for i in idx:
            e = np.zeros(mlp.N_PARAMS)
            e[i] = h
            fd = (np.dot(c, mlp.forward(p + e, X)[0]) - np.dot(c, mlp.forward(p - e, X)[0])) / (2 * h)
            err = max(err, abs(fd - g[i]) / max(1.0, abs(g[i])))
        return err

    assert worst(mlp.backward) <= 1e-6
    assert worst(bad) > 1e-3


def test_lawson_incircle_sign_is_pinned():
    """Flipping edges whose opposite vertex lies OUTSIDE the circumcircle does not reach Qhull's
    Delaunay triangulation."""
    from oracle import relax
    bad_in = _mutant(relax._in_circle, "return det > 1e-10 * s * s", "return det < -1e-10 * s * s")
    ns = dict(vars(relax))
    ns["_in_circle"] = bad_in
    src = textwrap.dedent(inspect.getsource(relax.lawson_flips))
    exec(compile(src, "<mutant of lawson_flips>", "exec"), ns)
    bad = ns["lawson_flips"]
    from test_oracle_relax import _scramble
    ms = meshgen.random_delaunay(150, seed=9)
    xy = ms.xy
    want = {tuple(sorted(r)) for r in ms.tris}
    start = np.asarray(_scramble(xy, relax.orient_ccw(xy, ms.tris), 150, seed=2))
    assert {tuple(sorted(r)) for r in start} != want
    good_t, _ = relax.lawson_flips(xy, start)
    bad_t, _ = bad(xy, start)
    assert {tuple(sorted(r)) for r in good_t} == want
    assert {tuple(sorted(r)) for r in bad_t} != want


def _triangulate_with(**swap):
    """oracle.triangulate.triangulate compiled with some of its helpers replaced."""
    from oracle import triangulate as tr
    ns = dict(vars(tr))
    ns.update(swap)
    src = textwrap.dedent(inspect.getsource(tr.triangulate))
    exec(compile(src, "<mutant of triangulate>", "exec"), ns)
    return ns["triangulate"]


def _refused_by_pins(run, check):
    try:
        check(*run())
    except AssertionError:
        return True
    return False


def test_lawson_requeue_is_pinned():
    """A Lawson pass that does not look again at the four edges around each flip stops short
    of the empty-circle definition."""
    from oracle import triangulate as tr
    bad = _triangulate_with(lawson=_mutant(tr.lawson, "todo += [(c, a), (a, d), (d, b), (b, c)]", "pass"))
    caught = 0
    for seed in range(6):
        xy = np.random.default_rng(seed).random((20, 2))
        want = tr.delaunay_brute(xy)
        assert np.array_equal(tr.triangulate(xy)[0], want)
        caught += not np.array_equal(bad(xy)[0], want)
    assert caught >= 3


def test_flip_refinement_retry_is_pinned():
    """Dropping a crossing edge whose quadrilateral is not convex, instead of trying it again
    after the others, does not restore the segments of a zigzag through a cloud."""
    from oracle import triangulate as tr
    from test_oracle_triangulate import _zigzag_case, check_cdt, hull_area2
    xy, segs = _zigzag_case()
    bad = _triangulate_with(recover_segment=_mutant(tr.recover_segment, "queue.append((a, b))", "pass"))
    check_cdt(xy, tr.triangulate(xy, segs)[0], segs, area2=hull_area2(xy))
    assert _refused_by_pins(lambda: (xy, bad(xy, segs)[0], segs, hull_area2(xy)), check_cdt)


def test_region_flood_stops_at_segments_is_pinned():
    """A flood that crosses segments empties the whole square instead of the hole."""
    from oracle import triangulate as tr
    from test_oracle_triangulate import check_cdt, polygon_area2, square_with_hole
    xy, segs, ol, hl = square_with_hole()
    area = polygon_area2(xy, ol) - polygon_area2(xy, hl)
    bad = _triangulate_with(drop_regions=_mutant(
        tr.drop_regions, "if j is not None and j not in gone and frozenset((a, b)) not in fixed:",
        "if j is not None and j not in gone:"))
    check_cdt(xy, tr.triangulate(xy, segs, holes=[[0.5, 0.5]])[0], segs, area2=area)
    assert _refused_by_pins(lambda: (xy, bad(xy, segs, holes=[[0.5, 0.5]])[0], segs, area), check_cdt)


def test_sweep_strict_visibility_is_pinned():
    """Joining hull edges that the new node sees only at a grazing angle (collinear) makes flat
    triangles on a lattice."""
    from oracle import triangulate as tr
    from test_oracle_triangulate import check_cdt, hull_area2
    g = np.stack(np.meshgrid(np.arange(5), np.arange(4)), -1).reshape(-1, 2) * 0.25
    bad_sweep = _mutant(tr.sweep_triangulation, "p) < 0 for i in range(m)]", "p) <= 0 for i in range(m)]")
    bad = _triangulate_with(sweep_triangulation=bad_sweep)
    check_cdt(g, tr.triangulate(g)[0], area2=hull_area2(g))
    assert _refused_by_pins(lambda: (g, bad(g)[0], (), hull_area2(g)), check_cdt)
