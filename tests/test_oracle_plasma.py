"""Plasma current (eqs. 5-6) and soft source pins on the oracle: closed-form recurrences."""
import math

import numpy as np
import pytest

import meshgen
from oracle import leapfrog as lf, mesh as om, operators, spectral


@pytest.fixture(scope="module")
def small():
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7)
    return operators.Operators(om.canonicalize(ms.xy, ms.tris)), ms


def _gradient_field(ops, seed=0):
    rng = np.random.default_rng(seed)
    m = ops.mesh
    phi = rng.standard_normal(m.n_nodes)
    phi[~np.isin(np.arange(m.n_nodes), lf.interior_nodes(ops))] = 0.0
    e = m.edges[ops.ie]
    return (phi[e[:, 1]] - phi[e[:, 0]]) / ops.elen


def test_static_field_oscillates_at_the_plasma_frequency(small):
    """Uniform n0, nu = 0, B = 0, E = grad phi: B stays 0 and E^{n+1} + E^{n-1} =
    (2 - n0 dt^2) E^n, i.e. a leap-frog oscillation at sqrt(n0)."""
    ops, ms = small
    n0 = 40.0 ** 2
    dt = 0.01
    pl = lf.Plasma(np.full(ms.n_nodes, n0), 0.0)
    E0 = _gradient_field(ops)
    hist = []
    st = lf.State(E0.copy(), np.zeros(ops.n_t), np.zeros(ops.n_ei), 0)
    hist.append(st.E)
    lf.run(ops, st, dt, 50, plasma=pl, record=lambda s: hist.append(s.E))
    H = np.array(hist)
    np.testing.assert_allclose(H[2:] + H[:-2], (2 - n0 * dt * dt) * H[1:-1], atol=1e-11 * np.abs(E0).max())


def test_em_mode_in_uniform_plasma_has_w2_plus_n0(small):
    """A K-eigenmode in uniform n0: the E amplitude obeys cos(W dt) = 1 - dt^2 (w_k^2 + n0)/2."""
    ops, ms = small
    lam, V = np.linalg.eigh(spectral.symmetric_K(ops))
    k = len(lam) // 2
    v = V[:, k] / np.sqrt(ops.w_B)
    n0 = 0.3 * lam[k]
    dt = 0.5 * 2 / math.sqrt(lam[-1] + n0)
    pl = lf.Plasma(np.full(ms.n_nodes, n0), 0.0)
    u = ops.L_B @ v
    st = lf.State(np.zeros(ops.n_ei), v.copy(), np.zeros(ops.n_ei), 0)
    amp = [0.0]
    lf.run(ops, st, dt, 80, plasma=pl, record=lambda s: amp.append(np.dot(ops.w_E * s.E, u)))
    a = np.array(amp)
    c = 2 - dt * dt * (lam[k] + n0)
    np.testing.assert_allclose(a[2:] + a[:-2], c * a[1:-1], atol=1e-10 * np.abs(a).max())


def test_collisions_damp_at_half_the_rate(small):
    """With collisions nu the plasma oscillation decays like exp(-nu t / 2)."""
    ops, ms = small
    n0, nu, dt = 50.0 ** 2, 2.0, 0.002
    pl = lf.Plasma(np.full(ms.n_nodes, n0), nu)
    E0 = _gradient_field(ops, 1)
    st = lf.State(E0.copy(), np.zeros(ops.n_t), np.zeros(ops.n_ei), 0)
    en = []
    lf.run(ops, st, dt, 1500, plasma=pl,
           record=lambda s: en.append(lf.energy_W(ops, s.E, s.B) + np.dot(ops.w_E, s.j ** 2) / n0))
    t = (np.arange(len(en)) + 1) * dt
    # energy ~ exp(-nu t): fit the slope of log energy over whole periods
    slope = np.polyfit(t, np.log(en), 1)[0]
    assert abs(slope + nu) < 0.02 * nu


def test_soft_source_first_step(small):
    """From zero fields one step adds dt a_i g(dt/2) on the source edges and nothing else."""
    ops, ms = small
    ids, amp = meshgen.source_line_amplitudes(ms.xy, ms.tris, 0.35, ms.h)
    src = lf.Source(ids, amp, 2 * math.pi * 3, 0.2, 0.1)
    dt = 1e-3
    st = lf.initial_state(ops)
    st = lf.step(ops, st, dt, source=src)
    E = ops.extend(st.E)
    g = math.sin(src.omega0 * 0.5 * dt) * math.exp(-((0.5 * dt - 0.2) / 0.1) ** 2)
    exp = np.zeros(ms.n_tris * 0 + ops.mesh.n_edges)
    exp[ids] = dt * amp * g
    np.testing.assert_allclose(E, exp, rtol=1e-15, atol=0)
    np.testing.assert_allclose(st.B, dt * (ops.L_E @ ops.restrict(exp)), rtol=1e-15, atol=1e-300)
