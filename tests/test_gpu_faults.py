"""Failure detection on the GPU path, made on the host or by the method's own physics:
the energy watchdog against a time step above the stability bound of eq. 20, the device
energy against the oracle, and an allocator that runs out.  Nothing here faults the GPU."""
import ctypes as C

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


@pytest.fixture(scope="module")
def small():
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    return ms, ops, spectral.dense_rho(ops)


def test_device_energy_matches_oracle(ue, small):
    ms, ops, rho = small
    rng = np.random.default_rng(0)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho)
    E0 = np.zeros(m.n_edges)
    E0[ops.ie] = rng.standard_normal(ops.n_ei)
    m.write_fields(E=E0, B=rng.standard_normal(m.n_tris))
    m.step_n(100)
    E, B, _ = m.read_fields()
    W = m.energy()
    Wo = lf.energy_W(ops, ops.restrict(E), B)
    assert abs(W / Wo - 1) < 1e-6


@pytest.mark.parametrize("factor,unstable", [(0.95, False), (1.05, True)])
def test_watchdog_flags_a_time_step_above_the_stability_bound(ue, small, factor, unstable):
    """Eq. 20: dt = 1.05 * 2/rho grows without bound and the watchdog flags it; 0.95 does not."""
    ms, ops, rho = small
    rng = np.random.default_rng(1)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=factor * 2.0 / rho, watchdog_every=20,
                     watchdog_growth=10.0)
    E0 = np.zeros(m.n_edges)
    E0[ops.ie] = rng.standard_normal(ops.n_ei)
    m.write_fields(E=E0, B=rng.standard_normal(m.n_tris))
    m.step_n(6000)
    ok, W, flag = m.check()
    if unstable:
        assert not ok and flag in (1, 2)
        with pytest.raises(ue.UEError) as ei:
            m.read_fields()
        assert ei.value.code == -7
    else:
        assert ok and flag == 0 and np.isfinite(W)
        m.read_fields()


def test_allocator_returning_null_is_reported(ue, small):
    """A device allocator callback that runs out after a few blocks: ue_geometry_build returns
    UE_ERR_ALLOC and frees what it had; the mesh can be rebuilt once memory is back."""
    import torch
    from paper_1812_01448_gb300 import _native as N
    ms, ops, rho = small
    state = {"left": 5, "live": {}}

    def alloc(nbytes, stream, ctx):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, stream, ctx):
        state["live"].pop(ptr, None)

    fa, ff = N.ALLOC_FN(alloc), N.FREE_FN(free)
    L = N.lib()
    xy = np.ascontiguousarray(ms.xy)
    t = np.ascontiguousarray(ms.tris, dtype=np.int32)
    h = C.c_void_p()
    o = N.Options()
    L.ue_options_default(C.byref(o))
    N.check(L.ue_mesh_load(xy.ctypes.data_as(N.PD), xy.shape[0], t.ctypes.data_as(N.PI32), t.shape[0],
                           C.byref(o), fa, ff, None, C.byref(h)), "load")
    o.dt_mode = ue.UE_DT_GIVEN
    o.dt = 0.5 / rho
    rc = L.ue_geometry_build(h, C.byref(o), None)
    assert rc == -6
    assert not state["live"]                     # everything it got was handed back
    state["left"] = 10 ** 6
    assert L.ue_geometry_build(h, C.byref(o), None) == 0
    L.ue_mesh_free(h)
    assert not state["live"]


def test_persistent_barrier_timeout_is_reported(ue, small):
    """A CTA that never reaches the grid barrier (test hook): the others give up after
    timeout_ms, the launch ends, UE_ERR_TIMEOUT is reported, and the context stays usable."""
    ms, ops, rho = small
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho, variant=ue.UE_VARIANT_PERSISTENT,
                     timeout_ms=50, test_skip_cta=3)
    m.write_fields(B=np.ones(m.n_tris))
    m.step_n(5)
    ok, W, flag = m.check()
    assert not ok and flag == 3
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho, variant=ue.UE_VARIANT_PERSISTENT)
    m.write_fields(B=np.ones(m.n_tris))
    m.step_n(5)
    assert m.check() [0]
    E, B, _ = m.read_fields()
    assert np.all(np.isfinite(B))
    m.close()


@pytest.mark.parametrize("kernel", ["split", "fused"])
def test_blocked_copy_wait_timeout_is_reported(ue, small, kernel):
    """A CTA of the pipelined blocked kernels whose barrier is armed for record bytes that never
    arrive (test hook): its bounded wait runs out after about a second, all its threads agree
    to stop before using the staged records, it waits (bounded) for its copies in flight and
    returns; the launch ends, UE_ERR_TIMEOUT is reported, and the same mesh then steps
    normally, equal to the plain step."""
    ms, ops, rho = small
    tbk = ue.UE_TB_FUSED if kernel == "fused" else ue.UE_TB_SPLIT
    m = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=64)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho, variant=ue.UE_VARIANT_BLOCKED,
                     block_depth=4, tb_kernel=tbk, test_skip_cta=1)
    assert m.stats()["tb_kernel_used"] == (4 if kernel == "fused" else 3)
    assert m.tiles().size - 1 > 1
    m.write_fields(B=np.ones(m.n_tris))
    m.step_n(4)
    ok, W, flag = m.check()
    assert not ok and flag == 3
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho, variant=ue.UE_VARIANT_BLOCKED,
                     block_depth=4, tb_kernel=tbk)
    B0 = np.sin(9 * ms.xy[ms.tris].mean(axis=1)[:, 0])
    m.write_fields(B=B0)
    m.step_n(9)
    assert m.check()[0]
    E, B, _ = m.read_fields()
    m.close()
    p = ue.Mesh(ms.xy, ms.tris, reorder=ue.UE_REORDER_GREEDY, tile_tris=64)
    p.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=0.5 / rho)
    p.write_fields(B=B0)
    p.step_n(9)
    Ep, Bp, _ = p.read_fields()
    p.close()
    assert np.array_equal(E, Ep) and np.array_equal(B, Bp)
