"""The compiled oracle step (oracle/cstep.c) against the numpy oracle (oracle/leapfrog.py).

The compiled copy only times the CPU baseline; these tests pin it to the numpy oracle, whose own
pins are the invariants of test_oracle_invariants.py: 100 cavity steps agree to 1e-15 relative
(vacuum, with a soft source, and with plasma current), and one thread and four threads give
identical results.
"""
import numpy as np
import pytest

import meshgen
from oracle import cstep, leapfrog as lf, mesh as om, operators, spectral


@pytest.fixture(scope="module")
def cavity():
    ms = meshgen.cavity_te11_mesh()
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    rho, _ = spectral.power_iteration(ops, 200)
    return ms, ops, 1.0 / rho


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["vacuum", "source", "plasma"])
def test_compiled_step_matches_numpy_oracle(cavity, kind):
    ms, ops, dt = cavity
    rng = np.random.default_rng(3)
    st = lf.initial_state(ops, E_all=rng.standard_normal(ops.mesh.n_edges), B=rng.standard_normal(ops.n_t))
    plasma = source = None
    if kind == "plasma":
        plasma = lf.Plasma(rng.uniform(0.5, 2.0, ops.mesh.n_nodes) * 1e4, nu=30.0)
        st.j[:] = rng.standard_normal(ops.n_ei)
    if kind == "source":
        ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
        source = lf.Source(ids, amp, 2 * np.pi * 20, 0.1, 0.05)
    ref = lf.run(ops, st, dt, 100, plasma=plasma, source=source)
    got, _ = cstep.Stepper(ops).run(st, dt, 100, plasma=plasma, source=source)
    assert _rel(got.E, ref.E) <= 1e-15 and _rel(got.B, ref.B) <= 1e-15
    if plasma is not None:
        assert _rel(got.j, ref.j) <= 1e-15
    assert got.n == ref.n == 100


def test_thread_count_does_not_change_results(cavity):
    _, ops, dt = cavity
    rng = np.random.default_rng(4)
    st = lf.initial_state(ops, E_all=rng.standard_normal(ops.mesh.n_edges), B=rng.standard_normal(ops.n_t))
    s = cstep.Stepper(ops)
    a, _ = s.run(st, dt, 50, threads=1)
    b, used = s.run(st, dt, 50, threads=4)
    assert np.array_equal(a.E, b.E) and np.array_equal(a.B, b.B)
    assert used >= 1
