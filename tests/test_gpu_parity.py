"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same inputs.

Tolerances: FP32 product <= 1e-4 relative L2 of each field after the stated number of steps;
FP64 check build <= 1e-12; geometry and power iteration are FP64 on both sides; connectivity,
graph replay and checkpoint/resume are bit-exact.
"""
import math

import numpy as np
import pytest

import meshgen
from oracle import leapfrog as lf, mesh as om, operators, spectral

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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle(ms):
    return operators.Operators(om.canonicalize(ms.xy, ms.tris))


@pytest.fixture(scope="module")
def cavity(cavity_mesh):
    return cavity_mesh, _oracle(cavity_mesh)


def test_geometry_matches_oracle(ue, cavity):
    ms, ops = cavity
    for mesh in (ms, meshgen.graded_square(0.01, 0.03, grade=0.3, seed=9,
                                           holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)])):
        o = ops if mesh is ms else _oracle(mesh)
        m = ue.Mesh(mesh.xy, mesh.tris)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-3)
        g = m.geometry()
        np.testing.assert_allclose(g["O"], o.geom.O, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(g["S"], o.geom.S, rtol=1e-12)
        ie = o.ie
        np.testing.assert_allclose(g["elen"][ie], o.geom.elen[ie], rtol=1e-14)
        np.testing.assert_allclose(g["d"][ie], o.geom.d[ie], rtol=1e-9)
        assert rel_l2(g["d"][ie], o.geom.d[ie]) < 1e-12
        assert np.all(np.isnan(g["d"][~o.mesh.interior]))
        m.close()


def test_power_iteration_matches_oracle(ue, cavity):
    ms, ops = cavity
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(power_iters=200, power_seed=7, safety=0.5)
    dt, rho, src = m.get_dt()
    rho_o, _ = spectral.power_iteration(ops, 200, seed=7)
    assert src == 1
    assert abs(rho / rho_o - 1) < 1e-10
    assert abs(dt - 1.0 / rho) < 1e-15 / rho
    lo, hi = spectral.certified_bracket(ops)
    assert lo <= rho <= hi


def _cavity_run(ue, ms, ops, precision, nsteps, graph_chunk=0, reorder=1):
    rho, _ = spectral.power_iteration(ops, 200)
    dt = 1.0 / rho
    B0 = meshgen.te_mode_b(ops.geom.O, 1, 1, 1.0, 0.5)
    m = ue.Mesh(ms.xy, ms.tris, reorder=reorder)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, precision=precision, graph_chunk=graph_chunk)
    m.write_fields(E=np.zeros(m.n_edges), B=B0)
    m.step_n(nsteps)
    E, B, _ = m.read_fields()
    m.close()
    st = lf.run(ops, lf.initial_state(ops, B=B0), dt, nsteps)
    return E, B, ops.extend(st.E), st.B


def test_cavity_te11_fp32_1000_steps(ue, cavity):
    ms, ops = cavity
    E, B, Eo, Bo = _cavity_run(ue, ms, ops, ue.UE_PREC_FP32, 1000)
    eE, eB = rel_l2(E, Eo), rel_l2(B, Bo)
    print(f"cavity fp32 1000 steps: rel L2 E {eE:.2e} B {eB:.2e}")
    assert eE <= 1e-4 and eB <= 1e-4
    assert np.all(E[~ops.mesh.interior] == 0)


def test_cavity_te11_fp64_check_1000_steps(ue, cavity):
    ms, ops = cavity
    E, B, Eo, Bo = _cavity_run(ue, ms, ops, ue.UE_PREC_FP64, 1000)
    eE, eB = rel_l2(E, Eo), rel_l2(B, Bo)
    print(f"cavity fp64 1000 steps: rel L2 E {eE:.2e} B {eB:.2e}")
    assert eE <= 1e-12 and eB <= 1e-12


def test_graph_replay_is_bit_identical_to_plain_launches(ue, cavity):
    ms, ops = cavity
    a = _cavity_run(ue, ms, ops, ue.UE_PREC_FP32, 100, graph_chunk=32)
    b = _cavity_run(ue, ms, ops, ue.UE_PREC_FP32, 100, graph_chunk=-1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_reorder_does_not_change_results_beyond_rounding(ue, cavity):
    ms, ops = cavity
    a = _cavity_run(ue, ms, ops, ue.UE_PREC_FP64, 300, reorder=0)
    b = _cavity_run(ue, ms, ops, ue.UE_PREC_FP64, 300, reorder=1)
    assert rel_l2(a[0], b[0]) < 1e-13 and rel_l2(a[1], b[1]) < 1e-13


def _plasma_case(n_tris=20000, seed=1003):
    ms = meshgen.plasma_square_mesh(n_tris, seed=seed)
    ops = _oracle(ms)
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    return ms, ops, w0, dens, ids, amp


@pytest.mark.parametrize("precision,nsteps,tol", [(0, 20000, 1e-4), (1, 2000, 1e-12)])
def test_plasma_with_source_downscale(ue, precision, nsteps, tol):
    """Plasma workload at 20k triangles: Gaussian density, nu = 0.01 w0, line source."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 200)
    pl = lf.Plasma(dens, 0.01 * w0)
    dt = spectral.stable_dt(rho, 0.5, pl.nbar(ops).max())
    src = lf.Source(ids, amp, w0, 0.1, 0.05)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, precision=precision)
    m.set_plasma(dens, 0.01 * w0)
    m.set_source(ids, amp, w0, 0.1, 0.05)
    m.step_n(nsteps)
    E, B, J = m.read_fields(j=True)
    assert m.get_step() == nsteps
    m.close()
    st = lf.run(ops, lf.initial_state(ops), dt, nsteps, plasma=pl, source=src)
    Eo, Bo, Jo = ops.extend(st.E), st.B, ops.extend(st.j)
    assert np.linalg.norm(Bo) > 0 and np.linalg.norm(Jo) > 0
    errs = rel_l2(E, Eo), rel_l2(B, Bo), rel_l2(J, Jo)
    print(f"plasma prec={precision} {nsteps} steps: rel L2 E {errs[0]:.2e} B {errs[1]:.2e} j {errs[2]:.2e}")
    assert max(errs) <= tol


def test_checkpoint_resume_is_bit_identical(ue):
    ms, ops, w0, dens, ids, amp = _plasma_case(5000, seed=77)
    rho, _ = spectral.power_iteration(ops, 100)
    dt = 0.5 / rho

    def fresh():
        m = ue.Mesh(ms.xy, ms.tris)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt)
        m.set_plasma(dens, 0.01 * w0)
        m.set_source(ids, amp, w0, 0.1, 0.05)
        return m

    a = fresh()
    a.step_n(400)
    Ea, Ba, Ja = a.read_fields(j=True)
    b = fresh()
    b.step_n(200)
    E1, B1, J1 = b.read_fields(j=True)
    step = b.get_step()
    b.close()
    c = fresh()
    c.write_fields(E1, B1, J1)
    c.set_step(step)
    c.step_n(200)
    Ec, Bc, Jc = c.read_fields(j=True)
    assert np.array_equal(Ea, Ec) and np.array_equal(Ba, Bc) and np.array_equal(Ja, Jc)


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_set_step_reaches_the_next_stepping_call(ue, variant):
    """ue_set_step is recorded on the host and written to the device counter by the next
    stepping call: get_step reads it back before any step, and after n steps it has advanced
    by n; a second set before stepping replaces the first."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY_RINGS, tile_tris=300)
    code = ue.UE_VARIANT_BLOCKED if variant == "blocked" else ue.UE_VARIANT_PLAIN
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-6, variant=code, block_depth=4)
    assert m.get_step() == 0
    m.set_step(1000)
    m.set_step(123)
    assert m.get_step() == 123
    m.step_n(7)
    assert m.get_step() == 130
    m.step_n(0)
    assert m.get_step() == 130
    m.close()


def test_non_delaunay_mesh_is_rejected(ue):
    # a quad split along its long diagonal: the two opposite angles sum to more than pi
    xy = np.array([[0, 0], [2, 0], [2.2, 1], [0.2, 1]], float) * [1, 0.3]
    m = ue.Mesh(xy, np.array([[0, 1, 2], [0, 2, 3]]))
    with pytest.raises(ue.UEError) as ei:
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-3)
    assert ei.value.code == -4


@pytest.mark.slow
@pytest.mark.parametrize("variant", ["plain", "blocked", "blocked-k8", "blocked-fused"])
def test_full_size_scatterer_window(ue, scatterer_window, variant):
    """Full size in the bench's launch configurations (plain: RCM, graphs of 32 steps;
    blocked: ring-ordered greedy tiles of <= 2500, k = 10 (and 8), 512 threads, split or fused
    kernel, the step graphs captured ahead by step_prepare) against the
    oracle on the whole mesh: relative L2 of each field, and per element the largest error
    against the field's largest value (an error confined to a few elements, such as the source
    edges or the hole's ring, would not move the L2 norm over 6M edges)."""
    ms, ops, ids, amp, w0, dt, Eo, Bo = scatterer_window
    blocked = variant != "plain"
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY_RINGS if blocked else ue.UE_REORDER_RCM,
                tile_tris=2500)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt,
                     variant=ue.UE_VARIANT_BLOCKED if blocked else ue.UE_VARIANT_PLAIN,
                     block_depth=8 if variant == "blocked-k8" else 10,
                     tb_kernel=ue.UE_TB_FUSED if variant == "blocked-fused" else ue.UE_TB_SPLIT)
    m.set_source(ids, amp, w0, 0.1, 0.05)
    if blocked:
        assert m.stats()["tb_kernel_used"] == (4 if variant == "blocked-fused" else 3)
    m.set_step(5000)
    m.step_prepare()
    m.step_n(200)
    E, B, _ = m.read_fields()
    m.close()
    eE, eB = rel_l2(E, Eo), rel_l2(B, Bo)
    iE = float(np.abs(E - Eo).max() / np.abs(Eo).max())
    iB = float(np.abs(B - Bo).max() / np.abs(Bo).max())
    src = np.asarray(ids)
    iS = float(np.abs(E[src] - Eo[src]).max() / np.abs(Eo[src]).max())
    print(f"scatterer {variant} n_t={ms.n_tris} 200 steps: rel L2 E {eE:.2e} B {eB:.2e}; "
          f"max per element E {iE:.2e} B {iB:.2e}, on the source edges {iS:.2e}")
    assert np.linalg.norm(Bo) > 0
    assert eE <= 1e-4 and eB <= 1e-4
    assert iE <= 1e-4 and iB <= 1e-4 and iS <= 1e-4


@pytest.mark.slow
def test_full_size_plasma_window(ue):
    """plasma-1M in the bench's launch configuration (ring-ordered greedy tiles <= 2700, k = 8,
    the one-CTA-per-tile kernel) against the oracle on the whole mesh over a 200-step window
    from step 5000 (source mid-pulse, current growing): relative L2 of E, B and j, and per
    element the largest error against each field's largest value."""
    ms = meshgen.cached("plasma_1003", meshgen.plasma_square_mesh)
    ops = _oracle(ms)
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    rho, _ = spectral.power_iteration(ops, 200)
    pl = lf.Plasma(dens, 0.01 * w0)
    dt = spectral.stable_dt(rho, 0.5, pl.nbar(ops).max())
    st = lf.initial_state(ops)
    st.n = 5000
    st = lf.run(ops, st, dt, 200, plasma=pl, source=lf.Source(ids, amp, w0, 0.1, 0.05))
    Eo, Bo, Jo = ops.extend(st.E), st.B, ops.extend(st.j)
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY_RINGS, tile_tris=2700)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, variant=ue.UE_VARIANT_BLOCKED, block_depth=8)
    m.set_plasma(dens, 0.01 * w0)
    m.set_source(ids, amp, w0, 0.1, 0.05)
    assert m.stats()["tb_kernel_used"] == 1
    m.set_step(5000)
    m.step_prepare()
    m.step_n(200)
    E, B, J = m.read_fields(j=True)
    m.close()
    assert np.linalg.norm(Bo) > 0 and np.linalg.norm(Jo) > 0
    errs = [rel_l2(E, Eo), rel_l2(B, Bo), rel_l2(J, Jo)]
    maxe = [float(np.abs(x - y).max() / np.abs(y).max()) for x, y in ((E, Eo), (B, Bo), (J, Jo))]
    print(f"plasma-1M n_t={ms.n_tris} 200 steps: rel L2 E {errs[0]:.2e} B {errs[1]:.2e} j {errs[2]:.2e}; "
          f"max per element {maxe[0]:.2e} {maxe[1]:.2e} {maxe[2]:.2e}")
    assert max(errs) <= 1e-4 and max(maxe) <= 1e-4


def _run_variant(ue, ms, dt, nsteps, variant, tile, k, dens=None, nu=0.0, src=None, graph_chunk=0,
                 B0=None, threads=0, reorder=None, kernel=0, expect_kernel=None):
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_KD if reorder is None else reorder,
                tile_tris=tile)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, variant=variant, block_depth=k,
                     graph_chunk=graph_chunk, tb_threads=threads, tb_kernel=kernel)
    if dens is not None:
        m.set_plasma(dens, nu)
    if src is not None:
        m.set_source(*src)
    if expect_kernel is not None:
        assert m.stats()["tb_kernel_used"] in expect_kernel, m.stats()["tb_kernel_used"]
    if B0 is not None:
        m.write_fields(B=B0)
    m.step_n(nsteps)
    out = m.read_fields(j=dens is not None)
    step = m.get_step()
    m.close()
    return out, step


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_step_prepare_is_bit_identical(ue, variant):
    """Step graphs captured ahead by step_prepare (once before set_plasma and set_source, which
    make the next step_n capture again, and once after them) give the fields of the lazily
    captured run bit for bit, over graph chunks and a remainder, plasma current included."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 50)
    dt = 0.45 / rho
    code = ue.UE_VARIANT_BLOCKED if variant == "blocked" else ue.UE_VARIANT_PLAIN
    B0 = np.sin(7 * ms.xy[ms.tris].mean(axis=1)[:, 0])
    out = []
    for prepare in (False, True):
        m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY_RINGS, tile_tris=300)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, variant=code, block_depth=5, graph_chunk=32)
        if prepare:
            m.step_prepare()
        m.set_plasma(dens, 0.01 * w0)
        m.set_source(ids, amp, w0, 0.0, 0.05)
        m.write_fields(B=B0)
        if prepare:
            m.step_prepare()
        m.step_n(71)
        out.append((m.read_fields(j=True), m.get_step()))
        m.close()
    (Ea, Ba, Ja), sa = out[0]
    (Eb, Bb, Jb), sb = out[1]
    assert sa == sb == 71
    assert np.array_equal(Ea, Eb) and np.array_equal(Ba, Bb) and np.array_equal(Ja, Jb)


@pytest.mark.parametrize("tile,k,nsteps,threads", [(512, 4, 14, 0), (1024, 8, 40, 0), (300, 1, 5, 0),
                                                   (2048, 3, 64, 0), (1500, 6, 23, 1024),
                                                   (64, 5, 31, 0)])
@pytest.mark.parametrize("plasma", [False, True])
@pytest.mark.parametrize("kernel", ["split", "fused"])
def test_blocked_is_bit_identical_to_plain(ue, tile, k, nsteps, threads, plasma, kernel):
    """Temporal blocking on KD tiles reproduces the plain two-kernel step bit for bit
    (partial last launch, double buffering, halo recompute, source and current included).
    Tiles of 64 triangles give more tiles than SMs, so the pipelined persistent form loads
    each CTA's next tile while it steps the current one (including a 1-step last launch)."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 50)
    dt = 0.45 / rho
    kw = dict(dens=dens if plasma else None, nu=0.01 * w0, src=(ids, amp, w0, 0.0, 0.05),
              B0=np.sin(7 * ms.xy[ms.tris].mean(axis=1)[:, 0]))
    (Ep, Bp, Jp), sp = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_PLAIN, tile, k, **kw)
    tbk = ue.UE_TB_FUSED if kernel == "fused" else ue.UE_TB_SPLIT
    # the fused kernel runs vacuum media with 512 threads; plasma and 1024 threads run the split
    # forms (1: one CTA per tile, 2: records in shared memory, 3: pipelined)
    expect = {4} if (kernel == "fused" and not plasma and threads != 1024) else {1, 2, 3}
    if tile == 64:
        expect &= {3, 4}     # more tiles than SMs: the pipelined form (plasma included) or the fused one
    for gc in (0, -1):
        (Eb, Bb, Jb), sb = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_BLOCKED, tile, k,
                                        graph_chunk=gc, threads=threads, kernel=tbk,
                                        expect_kernel=expect, **kw)
        assert sp == sb == nsteps
        assert np.array_equal(Ep, Eb) and np.array_equal(Bp, Bb)
        if plasma:
            assert np.array_equal(Jp, Jb)


@pytest.mark.parametrize("tile,k,nsteps", [(64, 5, 31), (1024, 8, 40), (300, 3, 13), (64, 10, 47),
                                           (1024, 10, 43)])
@pytest.mark.parametrize("kernel", ["split", "fused"])
@pytest.mark.parametrize("tiler", ["greedy", "rings"])
def test_blocked_on_greedy_tiles_is_bit_identical_to_plain(ue, tile, k, nsteps, kernel, tiler):
    """Greedy tiles (connected parts of any size up to the cap, small parts and hanging
    triangles joined), also with each tile's boundary rings stored first (rings), feed the
    same blocked kernel; it must reproduce the plain step on the same stored order bit for
    bit, with plasma, source and current."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 50)
    dt = 0.45 / rho
    reorder = ue.UE_REORDER_GREEDY if tiler == "greedy" else ue.UE_REORDER_GREEDY_RINGS
    kw = dict(dens=dens, nu=0.01 * w0, src=(ids, amp, w0, 0.0, 0.05),
              B0=np.sin(7 * ms.xy[ms.tris].mean(axis=1)[:, 0]), reorder=reorder)
    (Ep, Bp, Jp), sp = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_PLAIN, tile, k, **kw)
    (Eb, Bb, Jb), sb = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_BLOCKED, tile, k, **kw)
    assert sp == sb == nsteps
    assert np.array_equal(Ep, Eb) and np.array_equal(Bp, Bb) and np.array_equal(Jp, Jb)
    kw.pop("dens")
    kw["reorder"] = reorder
    tbk = ue.UE_TB_FUSED if kernel == "fused" else ue.UE_TB_SPLIT
    # the fused kernel holds at most 1023 source records per tile: tiles of 1024 with a 10-ring
    # halo hold up to 1038 copies of this mesh's 2873 source edges, so the split kernel runs
    fused = {3} if (tile, k) == (1024, 10) else {4}
    (Ep, Bp, _), _ = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_PLAIN, tile, k, **kw)
    (Eb, Bb, _), _ = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_BLOCKED, tile, k, kernel=tbk,
                                  expect_kernel=fused if kernel == "fused" else {1, 3}, **kw)
    assert np.array_equal(Ep, Eb) and np.array_equal(Bp, Bb)


def test_blocked_against_oracle(ue):
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 200)
    pl = lf.Plasma(dens, 0.01 * w0)
    dt = spectral.stable_dt(rho, 0.5, pl.nbar(ops).max())
    (E, B, J), _ = _run_variant(ue, ms, dt, 3001, ue.UE_VARIANT_BLOCKED, 1024, 4, dens=dens,
                                nu=0.01 * w0, src=(ids, amp, w0, 0.1, 0.05))
    st = lf.run(ops, lf.initial_state(ops), dt, 3001, plasma=pl,
                source=lf.Source(ids, amp, w0, 0.1, 0.05))
    errs = rel_l2(E, ops.extend(st.E)), rel_l2(B, st.B), rel_l2(J, ops.extend(st.j))
    print(f"blocked plasma 3001 steps: rel L2 E {errs[0]:.2e} B {errs[1]:.2e} j {errs[2]:.2e}")
    assert max(errs) <= 1e-4


def _batch_members():
    specs = meshgen.batch_specs(5, seed=31, n_min=1500, n_max=12000)
    out = []
    for sp in specs:
        ms = meshgen.batch_mesh(sp)
        ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.3, ms.h)
        out.append((ms, ids, amp, sp["omega0"]))
    return out


@pytest.mark.parametrize("variant", ["plain", "blocked", "persistent"])
def test_batch_is_bit_identical_to_single_meshes(ue, variant):
    """Every mesh of a batch (own dt from its own power iteration, own source frequency) ends
    bit-identical to the same mesh stepped alone; sizes and scatterers differ per mesh.  The
    persistent batch advances all meshes in one cooperative launch per chunk of steps."""
    blocked = variant == "blocked"
    code = {"plain": ue.UE_VARIANT_PLAIN, "blocked": ue.UE_VARIANT_BLOCKED,
            "persistent": ue.UE_VARIANT_PERSISTENT}[variant]
    singles = []
    for i, (ms, ids, amp, w0) in enumerate(_batch_members()):
        m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_KD if blocked else ue.UE_REORDER_RCM,
                    tile_tris=400)
        m.geometry_build(power_iters=60, variant=code, block_depth=3)
        m.set_source(ids, amp, w0, 0.0, 0.05)
        m.write_fields(B=np.cos(3.0 * ms.xy[ms.tris].mean(axis=1)[:, 1] + i))
        singles.append(m)
    dts = [m.get_dt()[0] for m in singles]
    assert len(set(dts)) == len(dts)
    b = ue.batch_create(singles)
    assert b.n_tris == sum(m.n_tris for m in singles)
    for n in (37, 64):        # plain launches, then graph chunks
        for m in singles:
            m.step_n(n)
        b.step_n(n)
    E, B, _ = b.read_fields()
    eo = to = 0
    for m in singles:
        Es, Bs, _ = m.read_fields()
        assert np.array_equal(E[eo:eo + m.n_edges], Es)
        assert np.array_equal(B[to:to + m.n_tris], Bs)
        assert np.linalg.norm(Es) > 0
        eo += m.n_edges
        to += m.n_tris
    b.close()
    for m in singles:
        m.close()


@pytest.mark.parametrize("plasma", [False, True])
def test_persistent_is_bit_identical_to_plain(ue, plasma):
    """One cooperative launch per chunk with timed grid barriers between the half-steps gives
    the plain kernels' results bit for bit."""
    ms, ops, w0, dens, ids, amp = _plasma_case()
    rho, _ = spectral.power_iteration(ops, 50)
    dt = 0.45 / rho
    out = []
    for variant in (ue.UE_VARIANT_PLAIN, ue.UE_VARIANT_PERSISTENT):
        m = ue.Mesh(ms.xy, ms.tris)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, variant=variant)
        if plasma:
            m.set_plasma(dens, 0.01 * w0)
        m.set_source(ids, amp, w0, 0.0, 0.05)
        m.write_fields(B=np.sin(5 * ms.xy[ms.tris].mean(axis=1)[:, 1]))
        m.step_n(101)
        assert m.check()[0]
        out.append(m.read_fields(j=plasma) + (m.get_step(),))
        m.close()
    (Ea, Ba, Ja, sa), (Eb, Bb, Jb, sb) = out
    assert sa == sb == 101
    assert np.array_equal(Ea, Eb) and np.array_equal(Ba, Bb)
    if plasma:
        assert np.array_equal(Ja, Jb)


@pytest.mark.parametrize("form", ["plain", "blocked", "plasma", "fp64"])
def test_pinned_host_arrays_move_in_place_with_the_same_results(ue, cavity, form):
    """ue_write_fields / ue_read_fields with pinned host arrays: the kernels read and write them
    in place (the stats count each array moved that way), and every field equals the run
    through pageable arrays, bit for bit."""
    torch = pytest.importorskip("torch")
    ms, ops = cavity
    rng = np.random.default_rng(11)
    E0 = rng.standard_normal(ops.mesh.n_edges)
    E0[~ops.mesh.interior] = 0.0
    B0 = rng.standard_normal(ms.tris.shape[0])
    j0 = rng.standard_normal(ops.mesh.n_edges) if form == "plasma" else None
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)

    def pinned(a):
        t = torch.empty(a.size, dtype=torch.float64, pin_memory=True).numpy()
        t[:] = a
        return t

    out = []
    for pin in (False, True):
        load = dict(reorder=ue.UE_REORDER_GREEDY, tile_tris=256) if form == "blocked" else {}
        opts = dict(variant=ue.UE_VARIANT_BLOCKED, block_depth=4) if form == "blocked" else {}
        if form == "fp64":
            opts["precision"] = ue.UE_PREC_FP64
        m = ue.Mesh(ms.xy, ms.tris, **load)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=2e-3, **opts)
        m.set_source(ids, amp, 2 * math.pi * 20, 0.1, 0.05)
        if form == "plasma":
            m.set_plasma(np.full(ms.xy.shape[0], 400.0), 3.0)
        conv = pinned if pin else (lambda a: a)
        m.write_fields(E=conv(E0), B=conv(B0), j=None if j0 is None else conv(j0))
        m.step_n(37)
        o = {"E": conv(np.empty(m.n_edges)), "B": conv(np.empty(m.n_tris))}
        if form == "plasma":
            o["j"] = conv(np.empty(m.n_edges))
        E, B, j = m.read_fields(j=form == "plasma", out=o)
        direct = m.stats()["direct_fields"]
        m.close()
        assert direct == (0 if not pin else (6 if form == "plasma" else 4))
        out.append((E.copy(), B.copy(), None if j is None else j.copy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    if form == "plasma":
        assert np.array_equal(out[0][2], out[1][2])
    assert np.all(out[1][0][~ops.mesh.interior] == 0)


@pytest.mark.parametrize("nsteps", [1, 7, 1000])
def test_whole_mesh_in_one_cta_is_bit_identical_to_plain(ue, cavity, nsteps):
    """A mesh that is a single tile without a halo (the 1,024-triangle cavity, greedy tiles of
    up to 4096 triangles) runs all its steps in one launch of one CTA with the whole mesh in
    shared memory; with a source it equals the plain step bit for bit, and after 1000 steps it
    matches the FP64 oracle as the plain step does."""
    ms, ops = cavity
    rho, _ = spectral.power_iteration(ops, 200)
    dt = 1.0 / rho
    B0 = meshgen.te_mode_b(ops.geom.O, 1, 1, 1.0, 0.5)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    src = (ids, amp, 2 * math.pi * 2, 0.0, 0.5)
    (Ep, Bp, _), sp = _run_variant(ue, ms, dt, nsteps, ue.UE_VARIANT_PLAIN, 0, 1, src=src, B0=B0,
                                   reorder=ue.UE_REORDER_RCM)
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=4096)
    assert m.tiles().size == 2                      # one tile
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, variant=ue.UE_VARIANT_BLOCKED, block_depth=8)
    m.set_source(*src)
    m.write_fields(B=B0)
    launches0 = m.stats()["kernel_launches"]
    assert m.stats()["tb_kernel_used"] == 5
    m.step_n(nsteps)
    Eb, Bb, _ = m.read_fields()
    assert m.stats()["kernel_launches"] - launches0 == 1
    assert m.get_step() == sp == nsteps
    m.close()
    assert np.array_equal(Ep, Eb) and np.array_equal(Bp, Bb)
    assert np.linalg.norm(Eb) > 0


@pytest.mark.parametrize("pin", [False, True])
@pytest.mark.parametrize("form", ["plain", "blocked", "plasma"])
def test_float32_field_transfers_equal_the_double_ones(ue, cavity, pin, form):
    """ue_write_fields_f32 / ue_read_fields_f32 with float values equal the double calls given
    the same values (written: U = |e| E in FP64 rounded once; read: E = U / |e| rounded to
    float), with pageable arrays (through a device copy) and pinned ones (in place)."""
    torch = pytest.importorskip("torch")
    ms, ops = cavity
    rng = np.random.default_rng(12)
    E0 = rng.standard_normal(ops.mesh.n_edges).astype(np.float32)
    E0[~ops.mesh.interior] = 0.0
    B0 = rng.standard_normal(ms.tris.shape[0]).astype(np.float32)
    j0 = rng.standard_normal(ops.mesh.n_edges).astype(np.float32) if form == "plasma" else None

    def conv(a):
        if a is None or not pin:
            return a
        t = torch.empty(a.size, dtype=torch.float32, pin_memory=True).numpy()
        t[:] = a
        return t

    def run(f32):
        load = dict(reorder=ue.UE_REORDER_GREEDY, tile_tris=256) if form == "blocked" else {}
        opts = dict(variant=ue.UE_VARIANT_BLOCKED, block_depth=4) if form == "blocked" else {}
        m = ue.Mesh(ms.xy, ms.tris, **load)
        m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=2e-3, **opts)
        if form == "plasma":
            m.set_plasma(np.full(ms.xy.shape[0], 400.0), 3.0)
        if f32:
            m.write_fields_f32(conv(E0), conv(B0), conv(j0))
        else:
            m.write_fields(E0.astype(np.float64), B0.astype(np.float64),
                           None if j0 is None else j0.astype(np.float64))
        m.step_n(23)
        if f32:
            o = {"E": conv(np.empty(m.n_edges, np.float32)), "B": conv(np.empty(m.n_tris, np.float32))}
            if form == "plasma":
                o["j"] = conv(np.empty(m.n_edges, np.float32))
            out = m.read_fields_f32(j=form == "plasma", out=o)
        else:
            out = m.read_fields(j=form == "plasma")
        direct = m.stats()["direct_fields"]
        m.close()
        return [None if a is None else np.array(a) for a in out], direct

    (E32, B32, j32), d32 = run(True)
    (E64, B64, j64), _ = run(False)
    assert d32 == ((6 if form == "plasma" else 4) if pin else 0)
    assert np.array_equal(E32, E64.astype(np.float32)) and np.array_equal(B32, B64.astype(np.float32))
    if form == "plasma":
        assert np.array_equal(j32, j64.astype(np.float32))
    assert np.abs(B32).max() > 0
