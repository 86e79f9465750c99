"""PML frame on the GPU (ue_frame_attach) against the oracle's framed operators."""
import math

import numpy as np
import pytest

import meshgen
from oracle import geometry, leapfrog as lf, mesh as om, pml, spectral

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


def _square(h=1 / 32, seed=5):
    ms = meshgen.graded_square(h, h, grade=0.0,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)], seed=seed)
    return ms, om.canonicalize(ms.xy, ms.tris)


def _pulse(m, x0=(0.3, 0.3)):
    C = m.xy[m.tris].mean(axis=1)
    r2 = ((C - np.asarray(x0)) ** 2).sum(axis=1)
    return (C[:, 0] - x0[0]) * np.exp(-r2 / 0.12 ** 2)


def _oracle_fields(fo, E, Bs, n_edges):
    """Oracle state in the library's output layout: (E per caller edge, B per triangle, frame B
    in strip order, Ex [NY+1, NX], Ey [NY, NX+1])."""
    Ec = np.zeros(n_edges)
    Ec[fo.inner.ie] = E[:fo.inner.n_ei]
    for k, rec in enumerate(fo.iface):
        Ec[rec[0]] = E[fo.inner.n_ei + k]
    B = fo.P @ Bs
    Ex = np.zeros((fo.NY + 1, fo.NX))
    Ey = np.zeros((fo.NY, fo.NX + 1))
    for (I, J), row in fo.H.items():
        Ex[J, I] = E[row]
    for (I, J), row in fo.V.items():
        Ey[J, I] = E[row]
    return Ec, B[:fo.n_in], B[fo.n_in:], Ex, Ey


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_framed_power_iteration_matches_oracle(ue):
    """The power iteration covers the coupled system (triangles + frame cells, same start
    vector keyed by caller triangle id and n_t + frame cell)."""
    ms, m = _square()
    fo = pml.FramedOperators(m, 8)
    rho_o, _ = spectral.power_iteration(fo, 200)
    mesh = ue.Mesh(ms.xy, ms.tris)
    mesh.frame_attach(8)
    mesh.geometry_build(precision=ue.UE_PREC_FP64)
    dt, rho, src = mesh.get_dt()
    mesh.close()
    assert abs(rho - rho_o) <= 1e-10 * rho_o
    # dense check of the coupled operator's top mode (the iteration converged)
    lam = np.linalg.eigvalsh(spectral.symmetric_K(fo))
    assert abs(rho - math.sqrt(lam[-1])) <= 1e-3 * rho


@pytest.mark.parametrize("precision,nsteps,tol", [(1, 600, 1e-12), (0, 2000, 1e-4)])
def test_framed_pulse_matches_oracle(ue, precision, nsteps, tol):
    """A pulse in the holed square, W = 8 layer with the default decay, against the oracle:
    mesh E (interior and outer edges), mesh B, frame B and frame E."""
    ms, m = _square()
    fo = pml.FramedOperators(m, 8)
    rho_o, _ = spectral.power_iteration(fo, 200)
    dt = 0.5 * 2 / rho_o
    b = _pulse(m)
    E, Bs = np.zeros(fo.n_ei), fo.start_split(np.concatenate([b, np.zeros(fo.n_fc)]))
    E, Bs = pml.run(fo, E, Bs, dt, nsteps)
    ref = _oracle_fields(fo, E, Bs, m.n_edges)
    mesh = ue.Mesh(ms.xy, ms.tris)
    mesh.frame_attach(8)
    mesh.geometry_build(precision=precision, dt_mode=ue.UE_DT_GIVEN, dt=dt)
    mesh.write_fields(B=b)
    mesh.step_n(nsteps)
    Eg, Bg, _ = mesh.read_fields()
    Bf, Ex, Ey = mesh.frame_fields()
    mesh.close()
    got = (Eg, Bg, Bf, Ex, Ey)
    errs = [_rel(g, r) for g, r in zip(got, ref)]
    print("framed pulse rel L2 (E, B, frame B, Ex, Ey):", ["%.2e" % e for e in errs])
    assert np.linalg.norm(ref[2]) > 1e-3 * np.linalg.norm(b)      # the pulse reached the frame
    assert max(errs) <= tol


def test_framed_graphs_are_bit_identical_to_plain_launches(ue):
    ms, m = _square()
    b = _pulse(m)
    out = []
    for gc in (32, -1):
        mesh = ue.Mesh(ms.xy, ms.tris)
        mesh.frame_attach(6)
        mesh.geometry_build(graph_chunk=gc)
        mesh.write_fields(B=b)
        mesh.step_n(100)
        E, B, _ = mesh.read_fields()
        Bf, Ex, Ey = mesh.frame_fields()
        out.append((E, B, Bf, Ex, Ey))
        mesh.close()
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_pml_follows_a_large_undamped_frame_until_its_echo(ue):
    """The oracle's absorption pin, on the GPU in FP32: a 12-cell layer stays within 5e-4 of the
    same mesh in a 48-cell undamped frame up to t = 2.4."""
    ms, m = _square()
    b = _pulse(m)
    runs = {}
    dt = None
    for W, sm in ((48, 0.0), (12, -1.0)):
        mesh = ue.Mesh(ms.xy, ms.tris)
        mesh.frame_attach(W, sigma_max=sm)
        if dt is None:
            mesh.geometry_build()
            dt = mesh.get_dt()[0]
        mesh.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt)
        mesh.write_fields(B=b)
        snaps = []
        n = int(2.4 / dt)
        for _ in range(4):
            mesh.step_n(n // 4)
            snaps.append(mesh.read_fields()[1])
        runs[W] = snaps
        mesh.close()
    S = geometry.areas(m.xy, m.tris)
    nb = math.sqrt(np.dot(S, b * b))
    err = max(math.sqrt(np.dot(S, (p - r) ** 2)) / nb for p, r in zip(runs[12], runs[48]))
    print(f"PML W=12 vs undamped W=48: {err:.2e}")
    assert err < 5e-4


@pytest.mark.parametrize("tile,k,nsteps", [(256, 4, 61), (128, 8, 50), (400, 3, 37), (4096, 4, 22)])
def test_blocked_framed_is_bit_identical_to_plain(ue, tile, k, nsteps):
    """Blocked stepping of a framed mesh: tiles whose k rings stay off the outer edges run in the
    blocked kernel, the rest (with the frame) as one region advanced k steps by the plain
    kernels on local copies.  Same fields as plain stepping, bit for bit, with a line source
    (a step count that is not a multiple of k; the last case has no blocked tiles at all)."""
    ms, m = _square()
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    b = _pulse(m)
    out = []
    for variant in (ue.UE_VARIANT_PLAIN, ue.UE_VARIANT_BLOCKED):
        mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=tile)
        mesh.frame_attach(6)
        mesh.geometry_build(variant=variant, block_depth=k)
        mesh.set_source(ids, amp, 2 * math.pi * 20, 0.0, 0.05)
        mesh.write_fields(B=b)
        mesh.step_n(nsteps)
        E, B, _ = mesh.read_fields()
        out.append((E, B) + mesh.frame_fields() + (mesh.get_step(),))
        mesh.close()
    for a, c in zip(out[0][:5], out[1][:5]):
        assert np.array_equal(a, c)
    assert out[0][5] == out[1][5] == nsteps


def test_framed_write_fields_sets_the_outer_edges(ue):
    """E written on the mesh's outer edges (the frame's interface) reaches the step in both
    launch forms (in the blocked one it lives in the region's slots): plain and blocked stay
    bit-identical, and reading back right after writing returns what was written."""
    ms, m = _square()
    rng = np.random.default_rng(8)
    E0 = rng.standard_normal(m.n_edges) * 0.1
    B0 = _pulse(m)
    outer = ~m.interior
    out = []
    for variant in (ue.UE_VARIANT_PLAIN, ue.UE_VARIANT_BLOCKED):
        mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=256)
        mesh.frame_attach(6)
        mesh.geometry_build(variant=variant, block_depth=4)
        info = mesh.frame_info()
        mesh.write_fields(E=E0, B=B0)
        E1, _, _ = mesh.read_fields()
        on_frame = np.abs(E1[outer]) > 0
        assert on_frame.sum() == info["n_interface"]       # the outer edges that face the frame
        np.testing.assert_allclose(E1[outer][on_frame], E0[outer][on_frame], rtol=1e-6)
        mesh.step_n(30)
        E, B, _ = mesh.read_fields()
        out.append((E, B) + mesh.frame_fields())
        mesh.close()
    for a, c in zip(*out):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("precision,nsteps,tol", [(1, 400, 1e-12), (0, 1500, 1e-4)])
def test_framed_plasma_matches_oracle(ue, precision, nsteps, tol):
    """Plasma medium (Gaussian density, nu = 0.01 w0, line source) in the holed square with an
    8-cell PML frame, plain variant: E, B, j and the frame's fields against the oracle's framed
    plasma step."""
    ms, m = _square()
    fo = pml.FramedOperators(m, 8)
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    nu = 0.01 * w0
    nbar = pml.inner_nbar(fo, dens)
    rho_o, _ = spectral.power_iteration(fo, 200)
    dt = 0.5 * 2 / math.sqrt(rho_o ** 2 + nbar.max())
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    src = lf.Source(ids, amp, w0, 0.0, 0.05)
    b = _pulse(m)
    E, Bs = np.zeros(fo.n_ei), fo.start_split(np.concatenate([b, np.zeros(fo.n_fc)]))
    j = np.zeros(fo.inner.n_ei)
    rows = fo.inner.col_of_edge[ids]
    for k in range(nsteps):
        E, Bs, j = pml.step_plasma(fo, E, Bs, j, dt, nbar, nu, src=(rows, amp, src.g), n=k)
    ref = _oracle_fields(fo, E, Bs, m.n_edges)
    jref = np.zeros(m.n_edges)
    jref[fo.inner.ie] = j
    mesh = ue.Mesh(ms.xy, ms.tris)
    mesh.frame_attach(8)
    mesh.geometry_build(precision=precision, dt_mode=ue.UE_DT_GIVEN, dt=dt)
    mesh.set_plasma(dens, nu)
    mesh.set_source(ids, amp, w0, 0.0, 0.05)
    mesh.write_fields(B=b)
    mesh.step_n(nsteps)
    Eg, Bg, Jg = mesh.read_fields(j=True)
    got = (Eg, Bg) + mesh.frame_fields()
    mesh.close()
    errs = [_rel(g, r) for g, r in zip(got, ref)] + [_rel(Jg, jref)]
    print("framed plasma rel L2 (E, B, frame B, Ex, Ey, j):", ["%.2e" % e for e in errs])
    assert np.linalg.norm(jref) > 0 and np.linalg.norm(ref[2]) > 0
    assert max(errs) <= tol


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_framed_checkpoint_resume_is_bit_identical(ue, variant):
    """Fields, step and the frame's own state (ue_frame_state) saved after 23 steps and
    restored into a fresh mesh continue exactly as the uninterrupted run."""
    ms, m = _square()
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    code = ue.UE_VARIANT_BLOCKED if variant == "blocked" else ue.UE_VARIANT_PLAIN

    def fresh():
        mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=256)
        mesh.frame_attach(6)
        mesh.geometry_build(variant=code, block_depth=4)
        mesh.set_source(ids, amp, 2 * math.pi * 20, 0.0, 0.05)
        return mesh

    a = fresh()
    a.write_fields(B=_pulse(m))
    a.step_n(23)
    E, B, _ = a.read_fields()
    state = a.frame_state()
    step = a.get_step()
    a.step_n(37)
    want = a.read_fields()[:2] + a.frame_fields()
    a.close()
    b = fresh()
    b.write_fields(E=E, B=B)
    b.frame_state(state)
    b.set_step(step)
    b.step_n(37)
    got = b.read_fields()[:2] + b.frame_fields()
    b.close()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_framed_mesh_refuses_other_variants(ue):
    ms, m = _square(1 / 16)
    mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=256)
    mesh.frame_attach(4)
    with pytest.raises(ue.UEError):
        mesh.geometry_build(variant=ue.UE_VARIANT_PERSISTENT)
    mesh.geometry_build()
    with pytest.raises(ue.UEError):           # modes of the closed cavity only
        mesh.modes(2, iters=5)
    import torch
    X = torch.empty((mesh.n_tris, 12), dtype=torch.float32, device="cuda")
    base = torch.empty(mesh.n_tris, dtype=torch.float32, device="cuda")
    with pytest.raises(ue.UEError):           # features describe unframed meshes
        mesh.rho_features(X, base)
    mesh.close()


@pytest.mark.parametrize("tile,k,nsteps", [(256, 4, 45), (4096, 3, 20)])
def test_blocked_framed_plasma_is_bit_identical_to_plain(ue, tile, k, nsteps):
    """Plasma with a frame in both launch forms: the region next to the frame carries its own
    current and the mesh's coefficients; E, B, j and the frame bit for bit."""
    ms, m = _square()
    w0 = 2 * math.pi * 20
    dens = meshgen.plasma_density_nodes(ms.xy, w0)
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    b = _pulse(m)
    out = []
    for variant in (ue.UE_VARIANT_PLAIN, ue.UE_VARIANT_BLOCKED):
        mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=tile)
        mesh.frame_attach(6)
        mesh.geometry_build(variant=variant, block_depth=k)
        mesh.set_plasma(dens, 0.01 * w0)
        mesh.set_source(ids, amp, w0, 0.0, 0.05)
        mesh.write_fields(B=b)
        mesh.step_n(nsteps)
        out.append(mesh.read_fields(j=True) + mesh.frame_fields())
        mesh.close()
    assert np.linalg.norm(out[0][2]) > 0
    for a, c in zip(*out):
        assert np.array_equal(a, c)


@pytest.fixture(scope="module")
def framed_window(scatterer_window):
    """The oracle's 200-step window of the framed scatterer (16-cell frame, line source from step
    5000) from a smooth field that is non-zero at the outer boundary."""
    ms, ops, ids, amp, w0, dt, _, _ = scatterer_window
    m = ops.mesh
    fo = pml.FramedOperators(m, 16, inner=ops, geom=ops.geom)
    C = m.xy[m.tris].mean(axis=1)
    b = np.cos(2 * np.pi * C[:, 0]) * np.cos(3 * np.pi * C[:, 1])
    src = lf.Source(ids, amp, w0, 0.1, 0.05)
    E, Bs = np.zeros(fo.n_ei), fo.start_split(np.concatenate([b, np.zeros(fo.n_fc)]))
    E, Bs = pml.run(fo, E, Bs, dt, 200, src=(ops.col_of_edge[ids], amp, src.g), n0=5000)
    return b, _oracle_fields(fo, E, Bs, m.n_edges)


@pytest.mark.slow
@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_full_size_scatterer_with_frame(ue, scatterer_window, framed_window, variant):
    """The bench's framed configurations at full size (3.96M triangles, 16-cell frame, FP32, line
    source from step 5000; plain: CUDA graphs of 32 steps; blocked: greedy tiles <= 2500, k = 8,
    the region next to the frame beside the blocked kernel): every field within 1e-4 of the
    oracle after 200 steps."""
    ms, ops, ids, amp, w0, dt, _, _ = scatterer_window
    b, ref = framed_window
    blocked = variant == "blocked"
    mesh = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY if blocked else ue.UE_REORDER_RCM,
                   tile_tris=2500)
    mesh.frame_attach(16)
    mesh.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=dt, block_depth=8,
                        variant=ue.UE_VARIANT_BLOCKED if blocked else ue.UE_VARIANT_PLAIN)
    mesh.set_source(ids, amp, w0, 0.1, 0.05)
    mesh.set_step(5000)
    mesh.write_fields(B=b)
    mesh.step_n(200)
    got = mesh.read_fields()[:2] + mesh.frame_fields()
    mesh.close()
    errs = [_rel(g, r) for g, r in zip(got, ref)]
    print(f"full-size framed window, {variant}, rel L2 (E, B, frame B, Ex, Ey):", ["%.2e" % e for e in errs])
    assert np.linalg.norm(ref[2]) > 1e-3 * np.linalg.norm(b)
    assert max(errs) <= 1e-4
