"""C-ABI checks that need no GPU: symbol exports and the host ingest tables (bit-exact)."""
import ctypes
import os
import re

import numpy as np
import pytest

import meshgen
from oracle import mesh as om, rcm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ue():
    from paper_1812_01448_gb300 import build
    build.build()
    import paper_1812_01448_gb300 as ue
    return ue


def _declared():
    src = open(os.path.join(ROOT, "include", "ue.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ue_[a-z_0-9]+)\s*\(", src)) - {"ue_alloc_fn", "ue_free_fn"})


def test_library_exports_every_declared_symbol(ue):
    from paper_1812_01448_gb300 import _native
    L = ctypes.CDLL(_native.LIB_PATH)
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n
    assert sorted(s[0] for s in _native.SIGNATURES) == names


def _meshes():
    yield "cavity", meshgen.cavity_te11_mesh()
    yield "random", meshgen.random_delaunay(2000, seed=21)
    yield "hole", meshgen.graded_square(0.01, 0.03, grade=0.3,
                                         holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=9)


@pytest.mark.parametrize("reorder", [0, 1])
def test_tables_bit_exact_against_oracle(ue, reorder):
    for name, ms in _meshes():
        # shuffle caller numbering and flip half the triangles to exercise orientation
        rng = np.random.default_rng(1)
        tris = ms.tris[rng.permutation(ms.n_tris)].copy()
        flip = rng.random(ms.n_tris) < 0.5
        tris[flip] = tris[flip][:, [0, 2, 1]]
        m = ue.Mesh(ms.xy, tris, reorder=reorder)
        t = m.tables()
        om_ = om.canonicalize(ms.xy, tris)
        order = rcm.rcm_order(om_) if reorder == 1 else np.arange(om_.n_tris)
        ref = rcm.device_tables(om_, order)
        assert m.n_edges == om_.n_edges and m.n_ei == ref["n_ei"], name
        assert np.array_equal(t["perm_tri"], ref["perm_tri"]), name
        assert np.array_equal(t["edge_caller"], ref["edge_caller"]), name
        assert np.array_equal(t["edge_tri"], ref["edge_tri"]), name
        assert np.array_equal(t["tri_code"], ref["tri_code"]), name
        m.close()


def test_kd_tiles_bit_exact_against_oracle(ue):
    for name, ms in _meshes():
        m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_KD, tile_tris=300)
        t = m.tables()
        om_ = om.canonicalize(ms.xy, ms.tris)
        order, offs = rcm.kd_order(om_, rcm.rcm_order(om_), 300)
        ref = rcm.device_tables(om_, order)
        assert np.diff(offs).max() <= 300
        for k in ("perm_tri", "edge_caller", "edge_tri", "tri_code"):
            assert np.array_equal(t[k], ref[k]), (name, k)
        assert np.array_equal(m.tiles(), offs), name
        m.close()


@pytest.mark.parametrize("tile", [16, 97, 300])
def test_greedy_tiles_bit_exact_against_oracle(ue, tile):
    for name, ms in _meshes():
        rng = np.random.default_rng(2)
        tris = ms.tris[rng.permutation(ms.n_tris)].copy()
        m = ue.Mesh(ms.xy, tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=tile)
        t = m.tables()
        om_ = om.canonicalize(ms.xy, tris)
        order, offs = rcm.greedy_order(om_, rcm.rcm_order(om_), tile)
        ref = rcm.device_tables(om_, order)
        for k in ("perm_tri", "edge_caller", "edge_tri", "tri_code"):
            assert np.array_equal(t[k], ref[k]), (name, tile, k)
        assert np.array_equal(m.tiles(), offs), (name, tile)
        m.close()


@pytest.mark.parametrize("tile", [40, 300])
def test_ring_ordered_tiles_follow_their_rule(ue, tile):
    """UE_REORDER_GREEDY_RINGS: the greedy tiles of the oracle (offsets and sets); inside each
    tile the ring index (0: a neighbour in another tile; breadth first inside the tile, capped
    at 15) never decreases; within a ring below the cap the angle of the centroids around the
    tile's mean centroid never decreases; the triangles at the cap keep the greedy order."""
    for name, ms in _meshes():
        m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY_RINGS, tile_tris=tile)
        perm, offs = m.tables()["perm_tri"], m.tiles()
        m.close()
        om_ = om.canonicalize(ms.xy, ms.tris)
        order, ref_offs = rcm.greedy_order(om_, rcm.rcm_order(om_), tile)
        assert np.array_equal(offs, ref_offs), name
        tile_of = np.empty(ms.n_tris, np.int64)
        rank = np.empty(ms.n_tris, np.int64)
        rank[order] = np.arange(ms.n_tris)
        for t in range(offs.size - 1):
            a, b = offs[t], offs[t + 1]
            assert set(perm[a:b].tolist()) == set(order[a:b].tolist()), (name, t)
            tile_of[perm[a:b]] = t
        nbrs = [[] for _ in range(ms.n_tris)]
        for R, L in zip(om_.R, om_.L):
            if R >= 0 and L >= 0:
                nbrs[R].append(L)
                nbrs[L].append(R)
        cen = ms.xy[om_.tris].mean(axis=1)
        for t in range(offs.size - 1):
            mem = perm[offs[t]:offs[t + 1]]
            ring = {j: 15 for j in mem.tolist()}
            frontier = [j for j in mem.tolist() if any(tile_of[o] != t for o in nbrs[j])]
            for j in frontier:
                ring[j] = 0
            for r in range(1, 15):
                nxt = []
                for j in frontier:
                    for o in nbrs[j]:
                        if tile_of[o] == t and ring[o] == 15:
                            ring[o] = r
                            nxt.append(o)
                frontier = nxt
            rr = np.array([ring[j] for j in mem.tolist()])
            assert np.all(np.diff(rr) >= 0), (name, t)
            c = cen[mem].mean(axis=0)
            ang = np.arctan2(cen[mem, 1] - c[1], cen[mem, 0] - c[0])
            for r in np.unique(rr):
                sel = rr == r
                if r < 15:
                    assert np.all(np.diff(ang[sel]) >= -1e-9), (name, t, r)
                else:
                    assert np.all(np.diff(rank[mem[sel]]) > 0), (name, t)


@pytest.mark.parametrize("reorder", [0, 1, 2, 3])
def test_unused_nodes_keep_tables_bit_exact(ue, reorder):
    # nodes that no triangle uses, before and after the used ones: they shift the caller ids
    # that order the edges but must create no edge
    ms = meshgen.random_delaunay(300, seed=3)
    extra = np.random.default_rng(0).random((50, 2)) * 10 + 5
    xy = np.vstack([extra[:20], ms.xy, extra[20:]])
    tris = ms.tris + 20
    kw = dict(reorder=reorder, tile_tris=40) if reorder >= 2 else dict(reorder=reorder)
    m = ue.Mesh(xy, tris, **kw)
    t = m.tables()
    o = om.canonicalize(xy, tris)
    if reorder == 0:
        order = np.arange(o.n_tris)
    elif reorder == 1:
        order = rcm.rcm_order(o)
    elif reorder == 2:
        order, _ = rcm.kd_order(o, rcm.rcm_order(o), 40)
    else:
        order, _ = rcm.greedy_order(o, rcm.rcm_order(o), 40)
    ref = rcm.device_tables(o, order)
    assert m.n_edges == o.n_edges == om.canonicalize(ms.xy, ms.tris).n_edges
    for k in ("perm_tri", "edge_caller", "edge_tri", "tri_code"):
        assert np.array_equal(t[k], ref[k]), k
    m.close()


def test_smallest_meshes(ue):
    # no triangle: refused on both sides; one triangle: three PEC edges, no unknown
    ms = meshgen.cavity_te11_mesh()
    with pytest.raises(ue.UEError) as ei:
        ue.Mesh(ms.xy, np.zeros((0, 3), np.int64))
    assert ei.value.code == -1
    with pytest.raises(om.MeshError):
        om.canonicalize(ms.xy, np.zeros((0, 3), np.int64))
    xy = np.array([[0, 0], [1, 0], [0, 1.0]])
    m = ue.Mesh(xy, np.array([[0, 2, 1]]))
    o = om.canonicalize(xy, np.array([[0, 2, 1]]))
    assert (m.n_tris, m.n_edges, m.n_ei) == (1, 3, 0) == (o.n_tris, o.n_edges, 0)
    assert m.tables()["edge_caller"].size == 0
    m.close()


def test_tiles_empty_without_partition(ue):
    ms = meshgen.cavity_te11_mesh()
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_RCM)
    assert m.tiles().size == 0
    m.close()


@pytest.mark.parametrize("tris,code", [
    ([[0, 1, 4]], -1),
    ([[0, 1, 1]], -3),
    ([[0, 1, 2], [0, 1, 3]], -2),
])
def test_ingest_errors_match_oracle_classification(ue, tris, code):
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    with pytest.raises(ue.UEError) as ei:
        ue.Mesh(xy, np.array(tris))
    assert ei.value.code == code
    with pytest.raises(om.MeshError) as eo:
        om.canonicalize(xy, np.array(tris))
    assert eo.value.code == code


def test_collinear_and_nonmanifold_rejected(ue):
    with pytest.raises(ue.UEError) as ei:
        ue.Mesh(np.array([[0, 0], [1, 0], [2, 0]], float), np.array([[0, 1, 2]]))
    assert ei.value.code == -3
    xy = np.array([[0, 0], [1, 0], [0.5, 1], [0.5, -1], [0.5, 2]], float)
    with pytest.raises(ue.UEError) as ei:
        ue.Mesh(xy, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    assert ei.value.code == -2


def test_frame_layout_and_interface_match_oracle(ue):
    from oracle import pml
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=5)
    m = ue.Mesh(ms.xy, ms.tris)
    m.frame_attach(6)
    info = m.frame_info()
    fo = pml.FramedOperators(om.canonicalize(ms.xy, ms.tris), 6)
    assert (info["W"], info["nx"], info["ny"], info["NX"], info["NY"]) == (6, fo.nx, fo.ny, fo.NX, fo.NY)
    assert info["n_cells"] == fo.n_fc and info["n_interface"] == fo.n_if
    assert abs(info["h"] - fo.h) <= 1e-12 * fo.h
    assert abs(info["sigma_max"] - fo.sigma_max) <= 1e-12 * fo.sigma_max
    edge, cell = m.frame_interface()
    cid = {c: k for k, c in enumerate(fo.frame_cells)}
    assert np.array_equal(edge, [rec[0] for rec in fo.iface])
    assert np.array_equal(cell, [cid[rec[7]] for rec in fo.iface])
    m.frame_attach(6, sigma_max=0.0)
    assert m.frame_info()["sigma_max"] == 0.0
    m.frame_attach(0)
    with pytest.raises(ue.UEError):
        m.frame_info()
    m.close()


def test_frame_refuses_a_boundary_that_is_not_a_divided_rectangle(ue):
    from test_oracle_pml import _not_a_divided_rectangle
    for xy, tris in _not_a_divided_rectangle():
        m = ue.Mesh(xy, tris)
        with pytest.raises(ue.UEError):
            m.frame_attach(4)
        m.close()
    ms = meshgen.cavity_te11_mesh()                     # boundary spacing 1/32 on all sides
    m = ue.Mesh(ms.xy, ms.tris)
    m.frame_attach(4)
    for bad in ((-1, -1.0, 3), (4, -1.0, 0), (4, float("nan"), 3), (300, -1.0, 3)):
        with pytest.raises(ue.UEError):
            m.frame_attach(*bad)
    m.close()


@pytest.mark.parametrize("reorder,tile", [(2, 64), (3, 64), (3, 16), (3, 100000)])
def test_partitions_of_a_mesh_in_two_pieces(ue, reorder, tile):
    """Two disjoint meshes in one load: RCM runs per component and both partitions cover them;
    tables and tile offsets bit-exact against the oracle (KD = 2, greedy = 3); a tile larger
    than the mesh gives one part per the greedy rules."""
    a = meshgen.cavity_te11_mesh()
    b = meshgen.random_delaunay(150, seed=12)
    xy = np.vstack([a.xy, b.xy + [3.0, 0.0]])
    tris = np.vstack([a.tris, b.tris + a.xy.shape[0]])
    m = ue.Mesh(xy, tris, reorder=reorder, tile_tris=tile)
    om_ = om.canonicalize(xy, tris)
    r = rcm.rcm_order(om_)
    order, offs = (rcm.kd_order if reorder == 2 else rcm.greedy_order)(om_, r, tile)
    t = m.tables()
    ref = rcm.device_tables(om_, order)
    for k in ("perm_tri", "edge_caller", "edge_tri", "tri_code"):
        assert np.array_equal(t[k], ref[k]), k
    assert np.array_equal(m.tiles(), offs)
    assert np.diff(offs).max() <= tile
    m.close()


@pytest.mark.parametrize("tile,k", [(128, 8), (256, 4), (400, 3), (4096, 4)])
def test_frame_region_plan(ue, tile, k):
    """The host plan of blocked stepping with a frame against a breadth-first search written
    here: tiles within k-1 rings of a triangle on the outer edges form the region; its local
    triangles are k rings around it, its local edges those with a triangle within k-1 rings."""
    ms = meshgen.graded_square(1 / 32, 1 / 32, grade=0.0,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=5)
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=tile)
    m.frame_attach(6)
    got = m.frame_region(k)
    t = m.tables()
    off = m.tiles()
    om_ = om.canonicalize(ms.xy, ms.tris)
    stored = np.empty(m.n_tris, np.int64)
    stored[t["perm_tri"]] = np.arange(m.n_tris)
    edge, _ = m.frame_interface()
    seeds = {int(stored[om_.R[e] if om_.R[e] >= 0 else om_.L[e]]) for e in edge}
    R, L = t["edge_tri"][:, 0].astype(np.int64), t["edge_tri"][:, 1].astype(np.int64)
    nbr = [[] for _ in range(m.n_tris)]
    for r, l in zip(R, L):
        nbr[r].append(l)
        nbr[l].append(r)

    def rings(start, depth):
        lvl = {s: 0 for s in start}
        front = list(start)
        for d in range(1, depth + 1):
            nxt = []
            for u in front:
                for w in nbr[u]:
                    if w not in lvl:
                        lvl[w] = d
                        nxt.append(w)
            front = nxt
        return lvl

    near = rings(seeds, k - 1)
    tile_of = np.searchsorted(off, np.arange(m.n_tris), side="right") - 1
    region_tiles = {int(tile_of[j]) for j in near}
    owned = np.isin(tile_of, list(region_tiles))
    lvl = rings(set(np.flatnonzero(owned).tolist()), k)
    edges = [i for i in range(len(R)) if min(lvl.get(R[i], 99), lvl.get(L[i], 99)) <= k - 1]
    own_e = [i for i in edges if owned[min(R[i], L[i])]]
    want = {"tiles": len(off) - 1, "blocked_tiles": len(off) - 1 - len(region_tiles),
            "region_owned_tris": int(owned.sum()), "region_tris": len(lvl),
            "region_edges": len(edges), "region_owned_edges": len(own_e)}
    assert got == want
    m.close()


def test_bench_partition_stats_match_the_oracle(ue):
    """The Fig. 6 quantities the bench reports (parts, part sizes, shared edges) from the
    library's tables agree with the oracle's definitions on the same partition."""
    import bench
    ms = meshgen.graded_square(0.01, 0.03, grade=0.3,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=9)
    for reorder, fn in ((ue.UE_REORDER_KD, rcm.kd_order), (ue.UE_REORDER_GREEDY, rcm.greedy_order)):
        m = ue.Mesh(ms.xy, ms.tris, reorder=reorder, tile_tris=300)
        st = bench.partition_stats(m)
        om_ = om.canonicalize(ms.xy, ms.tris)
        order, offs = fn(om_, rcm.rcm_order(om_), 300)
        sizes = np.diff(offs)
        assert st["parts"] == sizes.size and st["tris_max"] == sizes.max()
        assert abs(st["tris_mean"] - sizes.mean()) < 1e-9 and abs(st["tris_rms"] - sizes.std()) < 1e-9
        assert st["shared_edges"] == rcm.shared_edges(om_, order, offs)
        m.close()


def test_frame_calls_refuse_bad_arguments(ue):
    ms = meshgen.graded_square(1 / 16, 1 / 16, grade=0.0, seed=5)
    plain = ue.Mesh(ms.xy, ms.tris)                                   # no tiles, no frame
    for call in (lambda: plain.frame_region(4), lambda: plain.frame_interface(), lambda: plain.frame_info()):
        with pytest.raises(ue.UEError):
            call()
    plain.frame_attach(4)
    with pytest.raises(ue.UEError):                                   # a frame but no tiles
        plain.frame_region(4)
    tiled = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=128)
    tiled.frame_attach(4)
    for k in (0, 16):
        with pytest.raises(ue.UEError):
            tiled.frame_region(k)
    assert tiled.frame_region(15)["tiles"] == tiled.tiles().size - 1
    for m in (plain, tiled):
        with pytest.raises(ue.UEError):                               # nothing built yet
            m.frame_fields()
        m.close()


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "ue.h"
int main(void) {
    const double xy[8] = {0, 0, 4, 0, 2, 1, 2, -1};
    const int32_t seg[2] = {0, 1};
    int32_t tris[8 * 3];
    int64_t nt = 0, nf = 0;
    if (ue_triangulate(xy, 4, seg, 1, NULL, 0, 0, tris, 8, &nt, &nf) != UE_OK) return 1;
    printf("%lld %lld", (long long)nt, (long long)nf);
    for (int64_t i = 0; i < 3 * nt; ++i) printf(" %d", (int)tris[i]);
    if (ue_triangulate(xy, 2, NULL, 0, NULL, 0, 0, tris, 8, &nt, NULL) != UE_ERR_ARG) return 2;
    printf("|%s\n", ue_last_error());
    return strlen(ue_last_error()) > 0 ? 0 : 3;
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(ue, tmp_path):
    """include/ue.h compiles as C99 with -pedantic-errors, and a C program linked against the
    library runs a host-only call (the kite of the triangulation pins: one flip restores its
    long diagonal) and reads the thread's error text after a refused call."""
    import shutil
    import subprocess
    from paper_1812_01448_gb300 import _native
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    lib_dir = os.path.dirname(_native.LIB_PATH)
    cuda_inc = "/usr/local/cuda/include"
    exe = tmp_path / "caller"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic-errors", f"-I{ROOT}/include",
                        f"-I{cuda_inc}", str(src), "-o", str(exe), f"-L{lib_dir}", "-lue",
                        f"-Wl,-rpath,{lib_dir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    head, err = r.stdout.strip().split("|")
    vals = [int(v) for v in head.split()]
    assert vals[:2] == [2, 1]
    from oracle import triangulate as tr
    got = tr.canonical(np.array(vals[2:]).reshape(-1, 3))
    assert got.tolist() == [[0, 1, 2], [0, 3, 1]]
    assert "ue_triangulate" in err


def test_error_text_is_per_thread(ue):
    """Two threads refused for different reasons, many times over: each reads its own text
    (the error string is thread-local)."""
    import threading
    xy_dup = np.array([[0, 0], [1, 0], [0, 1], [1, 0.0]])
    xy_ok = np.random.default_rng(20).random((30, 2))
    seen = {"dup": set(), "seg": set()}

    def run(kind):
        for _ in range(200):
            try:
                if kind == "dup":
                    ue.triangulate(xy_dup)
                else:
                    ue.triangulate(xy_ok, [[0, 0]])
            except ue.UEError as e:
                seen[kind].add(str(e).split(": ", 1)[1])

    ts = [threading.Thread(target=run, args=(k,)) for k in ("dup", "seg")]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert len(seen["dup"]) == 1 and "repeats another node" in next(iter(seen["dup"]))
    assert len(seen["seg"]) == 1 and "bad node id" in next(iter(seen["seg"]))


@pytest.mark.parametrize("bad", ["anchor_range", "keep_self", "keep_range", "tau", "iters", "flat", "sizes"])
def test_mesh_relax_refuses_bad_input_before_the_gpu(ue, bad):
    """ue_mesh_relax checks its arguments on the host before any device call: each refusal
    comes back as its error code with no GPU present."""
    ms = meshgen.random_delaunay(60, seed=21)
    n = ms.xy.shape[0]
    tris = ms.tris.copy()
    kw = dict(iters=5)
    code = -1
    if bad == "anchor_range":
        kw["anchors"] = [n]
    elif bad == "keep_self":
        kw["keep"] = [[3, 3]]
    elif bad == "keep_range":
        kw["keep"] = [[0, -1]]
    elif bad == "tau":
        kw["tau"] = 0.2
    elif bad == "iters":
        kw["iters"] = -1
    elif bad == "flat":
        tris[0] = [0, 0, 1]
        code = -3
    else:
        kw["h_nodes"] = np.zeros(n)
    with pytest.raises(ue.UEError) as ei:
        ue.mesh_relax(ms.xy, tris, kw.pop("iters"), **kw)
    assert ei.value.code == code


def test_every_entry_point_refuses_null_arguments(ue):
    """Each declared function called with NULL pointers and zero sizes returns UE_ERR_ARG (the
    void ones return, ue_last_error gives text): no call dereferences an absent argument."""
    import ctypes as C
    from paper_1812_01448_gb300 import _native as N
    L = N.lib()
    checked = 0
    for name, res, argtypes in N.SIGNATURES:
        args = []
        for t in argtypes:
            if t in (C.c_double, C.c_float):
                args.append(0.0)
            elif t in (C.c_int, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t):
                args.append(0)
            elif isinstance(t, type) and issubclass(t, C._CFuncPtr):
                args.append(t())          # a NULL callback
            else:
                args.append(None)
        r = getattr(L, name)(*args)
        if name in ("ue_options_default", "ue_mesh_free"):
            assert r is None
        elif name == "ue_last_error":
            assert isinstance(r, bytes)
        else:
            assert r == -1, name
            assert L.ue_last_error(), name
        checked += 1
    assert checked == len(N.SIGNATURES) >= 38


@pytest.mark.parametrize("bad", ["dtype", "shape", "strided", "cpu"])
def test_power_iteration_static_checks_its_tensors_before_the_library(ue, bad):
    """The binding refuses a wrong dtype, a shape that does not match the sizes taken from S
    and elen, a strided tensor, and host tensors, with ValueError and before any call into
    the library (these run without a GPU)."""
    torch = pytest.importorskip("torch")
    n_t, n_ei = 8, 6
    a = dict(edge_tri=torch.zeros((n_ei, 2), dtype=torch.int32), elen=torch.ones(n_ei, dtype=torch.float64),
             d=torch.ones(n_ei, dtype=torch.float64), tri_code=torch.zeros((n_t, 3), dtype=torch.int32),
             S=torch.ones(n_t, dtype=torch.float64), tri_caller=torch.arange(n_t, dtype=torch.int64))
    if bad == "dtype":
        a["tri_caller"] = a["tri_caller"].to(torch.int32)
        msg = "tri_caller must be"
    elif bad == "shape":
        a["edge_tri"] = torch.zeros((n_ei + 1, 2), dtype=torch.int32)
        msg = "edge_tri must be"
    elif bad == "strided":
        a["d"] = torch.ones(2 * n_ei, dtype=torch.float64)[::2]
        msg = "d must be contiguous"
    else:
        msg = "must be a CUDA tensor"
    with pytest.raises(ValueError, match=msg):
        ue.power_iteration_static(**a)


def test_stepping_calls_refuse_a_mesh_without_geometry(ue):
    """Before ue_geometry_build the stepping calls and the step counter return UE_ERR_ARG with a
    text, touching no device state (runs without a GPU): ue_step_n, ue_step_prepare,
    ue_set_step, ue_get_step."""
    import ctypes as C
    import meshgen
    from paper_1812_01448_gb300 import _native as N
    ms = meshgen.cavity_te11_mesh()
    m = ue.Mesh(ms.xy, ms.tris)
    L = N.lib()
    step = C.c_int64(-1)
    try:
        for rc in (L.ue_step_n(m._h, 5, None), L.ue_step_prepare(m._h, None), L.ue_set_step(m._h, 3),
                   L.ue_get_step(m._h, C.byref(step))):
            assert rc == N.UE_ERR_ARG
            assert b"geometry not built" in L.ue_last_error()
        assert step.value == -1
    finally:
        m.close()
