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


def test_static_power_iteration_rejects_oversize(ue):
    import torch
    n = ue._native.UE_STATIC_MAX_TRIS + 1
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = torch.zeros(n, dtype=torch.float64, device="cuda")
    i32 = torch.zeros(2, dtype=torch.int32, device="cuda")
    i64 = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(ue.UEError) as ei:
        ue.power_iteration_static(i32, z, z, i32, big, i64)
    assert ei.value.code == -1
