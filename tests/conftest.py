import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def cavity_mesh():
    import meshgen
    return meshgen.cavity_te11_mesh()


@pytest.fixture(scope="session")
def scatterer_window():
    """The benchmarked workload (~4M triangles) and the oracle's 200-step window from step 5000
    (mid-pulse, so that the line source is far from zero)."""
    import math

    import meshgen
    from oracle import leapfrog as lf, mesh as om, operators, spectral
    ms = meshgen.cached("scatterer_1002", meshgen.scatterer_mesh)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, 2e-4)
    w0 = 2 * math.pi * 20
    rho, _ = spectral.power_iteration(ops, 200)
    dt = 1.0 / rho
    src = lf.Source(ids, amp, w0, 0.1, 0.05)
    st = lf.initial_state(ops)
    st.n = 5000
    st = lf.run(ops, st, dt, 200, source=src)
    return ms, ops, ids, amp, w0, dt, ops.extend(st.E), st.B
