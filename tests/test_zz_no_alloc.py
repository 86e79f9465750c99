"""The power iteration that allocates no device memory (ue_power_iteration_static).

Callers that cannot allocate device memory while they run use this entry point: code held to a
memory budget reserved up front, plug-ins whose host process owns the allocator, or code that
must not take cudaMalloc's implicit synchronisation.  Its work vectors live in one array that
the library holds for the process lifetime.  Here it is checked, on two calls in a row, against
the power iteration that ue_geometry_build runs (same seed and iteration count), through the
C ABI.  This file sorts last so that a run stopping at its first failure has run every other
test first.
"""
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


def _device_inputs(ue, ms, seed):
    import torch
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(power_iters=200, power_seed=seed)
    _, rho_ref, _ = m.get_dt()
    t = m.tables()
    g = m.geometry()
    m.close()
    ec, perm = t["edge_caller"], t["perm_tri"]
    dev = dict(
        edge_tri=torch.from_numpy(np.ascontiguousarray(t["edge_tri"])).cuda(),
        elen=torch.from_numpy(np.ascontiguousarray(g["elen"][ec])).cuda(),
        d=torch.from_numpy(np.ascontiguousarray(g["d"][ec])).cuda(),
        tri_code=torch.from_numpy(np.ascontiguousarray(t["tri_code"])).cuda(),
        S=torch.from_numpy(np.ascontiguousarray(g["S"][perm])).cuda(),
        tri_caller=torch.from_numpy(np.ascontiguousarray(perm)).cuda(),
    )
    return rho_ref, dev


@pytest.mark.parametrize("which", ["cavity", "graded"])
def test_static_power_iteration_matches_geometry_build(ue, which):
    ms = (meshgen.cavity_te11_mesh() if which == "cavity" else
          meshgen.graded_square(0.004, 0.01, grade=0.1, seed=5,
                                holes=[meshgen.polygon_triangle((0.5, 0.5), 0.2)]))
    rho_ref, dev = _device_inputs(ue, ms, seed=7)
    for _ in range(2):
        rho = ue.power_iteration_static(**dev, iters=200, seed=7)
        assert abs(rho / rho_ref - 1.0) <= 1e-12, (rho, rho_ref)


def test_static_power_iteration_takes_no_device_memory(ue):
    """After a warm-up call (which places the work array on the device under lazy module
    loading), a call changes neither the device's free memory nor torch's allocations."""
    import torch
    ms = meshgen.cavity_te11_mesh()
    rho_ref, dev = _device_inputs(ue, ms, seed=3)
    ue.power_iteration_static(**dev, iters=50, seed=3)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    rho = ue.power_iteration_static(**dev, iters=200, seed=3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert (free1, torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == (free0, alloc0, reserved0)
    assert abs(rho / rho_ref - 1.0) <= 1e-12


def _sized(n_t, n_ei):
    import torch
    f = dict(dtype=torch.float64, device="cuda")
    return dict(edge_tri=torch.zeros((n_ei, 2), dtype=torch.int32, device="cuda"),
                elen=torch.ones(n_ei, **f), d=torch.ones(n_ei, **f),
                tri_code=torch.zeros((n_t, 3), dtype=torch.int32, device="cuda"),
                S=torch.ones(n_t, **f), tri_caller=torch.arange(n_t, dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("which", ["tris", "edges"])
def test_static_power_iteration_rejects_oversize(ue, which):
    n_t = ue._native.UE_STATIC_MAX_TRIS + (1 if which == "tris" else 0)
    n_ei = ue._native.UE_STATIC_MAX_EDGES + (1 if which == "edges" else 0)
    with pytest.raises(ue.UEError) as ei:
        ue.power_iteration_static(**_sized(n_t, n_ei))
    assert ei.value.code == -1


@pytest.mark.parametrize("bad", ["edge_tri", "tri_code"])
def test_static_power_iteration_refuses_out_of_range_indices(ue, bad):
    """Indices that leave the caller's arrays are checked in the kernels before any access
    (the element is skipped) and the call returns UE_ERR_ARG; the next good call is exact."""
    a = _sized(64, 32)
    a["tri_code"].fill_(2 * 32)       # every edge a boundary edge: valid
    if bad == "edge_tri":
        a["edge_tri"][5, 1] = 64      # one past the last triangle
    else:
        a["tri_code"][7, 2] = 2 * 33  # one past the zero slot
    with pytest.raises(ue.UEError) as ei:
        ue.power_iteration_static(**a)
    assert ei.value.code == -1
    ms = meshgen.cavity_te11_mesh()
    rho_ref, dev = _device_inputs(ue, ms, seed=9)
    assert abs(ue.power_iteration_static(**dev, iters=200, seed=9) / rho_ref - 1.0) <= 1e-12
