"""One mesh split into parts with a halo exchange every step (paper_1812_01448_gb300.halo), on
one GPU: three parts, each a libue.so mesh of its owned triangles and their ring, stepped by
ue_step_n and exchanging the ring's B through ue_exchange_tris (device copies between the parts
of one process stand in for the messages between ranks).  The stitched fields equal the whole
mesh's run bit for bit, with a soft source and a plasma current, in FP32 and in FP64."""
import math

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ue():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_01448_gb300 import build
    build.build()
    import paper_1812_01448_gb300 as ue
    return ue


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_three_parts_match_the_whole_mesh_bit_for_bit(ue, precision):
    from paper_1812_01448_gb300 import halo
    prec = ue.UE_PREC_FP32 if precision == "fp32" else ue.UE_PREC_FP64
    ms = meshgen.graded_square(0.006, 0.02, grade=0.3, seed=9,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)])
    g = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=800)
    plan = halo.Plan(ms.xy, ms.tris, halo.parts_from_tiles(g.tiles(), g.tables()["perm_tri"], 3))
    g.close()
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    rng = np.random.default_rng(4)
    whole = ue.Mesh(ms.xy, ms.tris)
    whole.geometry_build(precision=prec)
    dt = whole.get_dt()[0]
    E0 = rng.standard_normal(whole.n_edges)
    B0 = rng.standard_normal(whole.n_tris)
    j0 = rng.standard_normal(whole.n_edges)
    whole.set_source(ids, amp, w0, 0.1, 0.05)
    whole.set_plasma(dens, 0.01 * w0)
    whole.write_fields(E0, B0, j0)
    E_ref0, _, _ = whole.read_fields()
    whole.write_fields(E_ref0, B0, j0)        # E on boundary edges as the library keeps it
    whole.step_n(150)
    E_ref, B_ref, j_ref = whole.read_fields(j=True)
    whole.close()
    parts = []
    for p in range(plan.n_parts):
        e = halo.GpuPart(plan, p, dt, precision=prec)
        e.m.set_source(*plan.local_sources(p, ids, amp), w0, 0.1, 0.05)
        e.m.set_plasma(dens[plan.nodes[p]], 0.01 * w0)
        e.m.write_fields(plan.local_field_edges(p, E_ref0), plan.local_field_tris(p, B0),
                         plan.local_field_edges(p, j0))
        parts.append(e)
    halo.run(parts, plan, 150)
    E = np.full(E_ref.size, np.nan)
    B = np.full(B_ref.size, np.nan)
    J = np.full(j_ref.size, np.nan)
    for p, e in enumerate(parts):
        El, Bl, jl = e.m.read_fields(j=True)
        own_e = plan.owned_edges(p)
        ge = plan.global_edges_of(p)
        E[ge[own_e]] = El[own_e]
        J[ge[own_e]] = jl[own_e]
        B[plan.tris_global[p][plan.owned[p]]] = Bl[plan.owned[p]]
        e.close()
    assert not np.isnan(E).any() and not np.isnan(B).any()
    assert np.array_equal(B, B_ref) and np.array_equal(E, E_ref) and np.array_equal(J, j_ref)
    assert 0 < np.abs(B_ref).max() < 1e3
    assert plan.shared_boundary() > 0
