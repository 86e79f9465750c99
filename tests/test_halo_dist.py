"""One mesh split across ranks with a halo exchange every step (paper_1812_01448_gb300.halo), on
CPU: two gloo ranks (127.0.0.1) each step their part with the FP64 oracle and exchange the B
values of their rings by point-to-point messages.  Checked: the partition (parts from the
greedy tiler, rings, exchange lists that name the same triangles on both sides, l_Sigma), and
the stitched fields after 60 steps with a soft source and a plasma current, which must equal the
single-rank oracle run bit for bit (the local meshes keep the global numbering's order, so
every sum is evaluated in the same order)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_STEPS = 60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import math

    import meshgen
    import paper_1812_01448_gb300 as ue
    from paper_1812_01448_gb300 import halo
    ms = meshgen.graded_square(0.012, 0.03, grade=0.3, seed=9,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)])
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=400)   # host ingest only
    part = halo.parts_from_tiles(m.tiles(), m.tables()["perm_tri"], 2)
    m.close()
    plan = halo.Plan(ms.xy, ms.tris, part)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    return ms, plan, ids, amp, w0, dens


class OraclePart:
    """A part stepped by the FP64 oracle (the CPU stand-in for GpuPart)."""

    def __init__(self, plan, p, dt, E, B, j, ids, amp, w0, dens):
        import torch
        from oracle import leapfrog as lf, mesh as om, operators
        self.ops = operators.Operators(om.canonicalize(plan.local_xy(p), plan.local_tris(p)))
        self.src = lf.Source(*plan.local_sources(p, ids, amp), w0, 0.1, 0.05)
        self.pl = lf.Plasma(dens[plan.nodes[p]], 0.01 * w0)
        self.st = lf.initial_state(self.ops, E_all=plan.local_field_edges(p, E),
                                   B=plan.local_field_tris(p, B), j_all=plan.local_field_edges(p, j))
        self.dt = dt
        self.dtype = torch.float64

    def step(self, n=1):
        from oracle import leapfrog as lf
        self.st = lf.run(self.ops, self.st, self.dt, n, plasma=self.pl, source=self.src)

    def gather(self, ids):
        import torch
        return torch.from_numpy(self.st.B[ids].copy())

    def scatter(self, ids, buf):
        self.st.B[ids] = buf.numpy()


def _initial(ms, plan, seed=5):
    rng = np.random.default_rng(seed)
    n_e = plan.edge_keys.size
    E, j = rng.standard_normal(n_e), rng.standard_normal(n_e)
    from oracle import mesh as om
    inner = om.canonicalize(ms.xy, ms.tris).interior
    E[~inner] = 0.0
    j[~inner] = 0.0
    return E, rng.standard_normal(ms.tris.shape[0]), j


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1812_01448_gb300 import halo
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, plan, ids, amp, w0, dens = _case()
        E, B, j = _initial(ms, plan)
        # both sides name the same triangles: send our lists' global ids, compare with theirs
        mine = {k: plan.tris_global[rank][v].tolist() for k, v in plan.send[rank].items()}
        objs = [None, None]
        dist.all_gather_object(objs, mine)
        other = objs[1 - rank]
        recv_g = {k: plan.tris_global[rank][v].tolist() for k, v in plan.recv[rank].items()}
        tables_agree = other.get(rank, []) == recv_g.get(1 - rank, [])
        eng = OraclePart(plan, rank, 1.0 / 2200.0, E, B, j, ids, amp, w0, dens)
        for _ in range(N_STEPS):
            eng.step(1)
            halo.exchange_dist(eng, plan, rank, dist)
        own_t = plan.tris_global[rank][plan.owned[rank]]
        own_e = plan.owned_edges(rank)
        ge = plan.global_edges_of(rank)
        out = (rank, tables_agree, own_t, eng.st.B[plan.owned[rank]],
               ge[own_e], eng.ops.extend(eng.st.E)[own_e], eng.ops.extend(eng.st.j)[own_e])
        q.put(out)
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_two_gloo_ranks_match_the_single_rank_run_bit_for_bit():
    sys.path.insert(0, ROOT)
    from oracle import leapfrog as lf, mesh as om, operators
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms, plan, ids, amp, w0, dens = _case()
    # the partition: two compact parts of near-equal size, a ring on each side
    sizes = np.bincount(plan.part)
    assert sizes.size == 2 and abs(sizes[0] - sizes[1]) < 0.2 * sizes.mean()
    l_sigma = plan.shared_boundary()
    assert 0 < l_sigma < 0.05 * ms.tris.shape[0]
    assert all(r[1] for r in res)
    for p in range(2):
        assert sum(v.size for v in plan.send[p].values()) <= l_sigma
    # the single-rank oracle run on the whole mesh
    E, B, j = _initial(ms, plan)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    st = lf.initial_state(ops, E_all=E, B=B, j_all=j)
    st = lf.run(ops, st, 1.0 / 2200.0, N_STEPS, plasma=lf.Plasma(dens, 0.01 * w0),
                source=lf.Source(ids, amp, w0, 0.1, 0.05))
    Bs = np.full(ms.tris.shape[0], np.nan)
    Es = np.full(plan.edge_keys.size, np.nan)
    js = np.full(plan.edge_keys.size, np.nan)
    for r in res:
        Bs[r[2]] = r[3]
        Es[r[4]] = r[5]
        js[r[4]] = r[6]
    assert not np.isnan(Bs).any() and not np.isnan(Es).any()
    assert np.array_equal(Bs, st.B)
    assert np.array_equal(Es, ops.extend(st.E)) and np.array_equal(js, ops.extend(st.j))
    # a stable run (dt rho ~ 0.9 < 2) with fields of order one
    assert 0 < np.abs(st.B).max() < 100 and 0 < np.abs(st.E).max() < 100


def test_parts_in_one_process_match_and_a_skipped_exchange_breaks_it():
    """The same two parts stepped in one process (halo.run with exchange_local) equal the
    single-rank oracle run bit for bit; with the exchange left out (a planted mistake) the
    rings go stale and the stitched B differs."""
    sys.path.insert(0, ROOT)
    from oracle import leapfrog as lf, mesh as om, operators
    from paper_1812_01448_gb300 import halo
    ms, plan, ids, amp, w0, dens = _case()
    E, B, j = _initial(ms, plan)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    st = lf.initial_state(ops, E_all=E, B=B, j_all=j)
    st = lf.run(ops, st, 1.0 / 2200.0, 20, plasma=lf.Plasma(dens, 0.01 * w0),
                source=lf.Source(ids, amp, w0, 0.1, 0.05))

    def stitched(exchange):
        parts = [OraclePart(plan, p, 1.0 / 2200.0, E, B, j, ids, amp, w0, dens) for p in range(2)]
        halo.run(parts, plan, 20, exchange=exchange)
        Bs = np.full(ms.tris.shape[0], np.nan)
        for p, e in enumerate(parts):
            Bs[plan.tris_global[p][plan.owned[p]]] = e.st.B[plan.owned[p]]
        return Bs

    assert np.array_equal(stitched(halo.exchange_local), st.B)
    stale = stitched(lambda engines, plan: None)
    assert not np.array_equal(stale, st.B)
