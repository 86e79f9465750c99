"""Exact invariants of the scheme, checked on the oracle (Section 1 remark on div E, eqs. 7-10)."""
import numpy as np
import pytest

import meshgen
from oracle import leapfrog as lf, mesh as om, operators, spectral


@pytest.fixture(scope="module")
def ops(cavity_mesh):
    m = om.canonicalize(cavity_mesh.xy, cavity_mesh.tris)
    return operators.Operators(m)


def test_discrete_gradient_is_in_the_kernel_of_L_E(ops):
    """E_i = (phi_hi - phi_lo)/|e_i| with phi = 0 on the walls gives L_E E = 0 (curl grad = 0)."""
    rng = np.random.default_rng(0)
    m = ops.mesh
    phi = rng.standard_normal(m.n_nodes)
    phi[~np.isin(np.arange(m.n_nodes), lf.interior_nodes(ops))] = 0.0
    e = m.edges[ops.ie]
    E = (phi[e[:, 1]] - phi[e[:, 0]]) / ops.elen
    r = ops.L_E @ E
    scale = abs(ops.L_E) @ np.abs(E)
    assert np.max(np.abs(r)) < 1e-14 * np.max(scale)


def test_gradient_check_detects_a_flipped_sign(ops):
    """The same check fails if one triangle's sign table is wrong (the pin has teeth)."""
    m = ops.mesh
    bad = om.Mesh(m.xy, m.tris, m.edges, m.tri_edge, m.tri_sign.copy(), m.R, m.L, m.interior)
    j = int(np.nonzero(m.interior[m.tri_edge].all(axis=1))[0][0])
    bad.tri_sign[j, 0] *= -1
    ops2 = operators.Operators(bad)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(m.n_nodes)
    phi[~np.isin(np.arange(m.n_nodes), lf.interior_nodes(ops))] = 0.0
    e = m.edges[ops.ie]
    E = (phi[e[:, 1]] - phi[e[:, 0]]) / ops.elen
    assert np.max(np.abs(ops2.L_E @ E)) > 1e-3


def test_adjointness_from_energy_conservation(ops):
    """Eq. 10: W_E L_B = -(W_B L_E)^T exactly."""
    A = (ops.L_B.multiply(ops.w_E[:, None])).tocsr()
    Bm = (ops.L_E.multiply(ops.w_B[:, None])).T.tocsr()
    diff = (A + Bm).toarray()
    assert np.max(np.abs(diff)) <= 1e-15 * np.max(np.abs(A.toarray()))


def test_div_E_flux_is_unchanged_by_the_E_update(ops):
    """Remark after eq. 4: the Voronoi-cell flux of E is constant in time at interior nodes."""
    rng = np.random.default_rng(1)
    E0 = rng.standard_normal(ops.n_ei)
    B = rng.standard_normal(ops.n_t)
    E1 = E0 + 0.01 * (ops.L_B @ B)
    nodes = lf.interior_nodes(ops)
    f0 = lf.node_flux(ops, E0)[nodes]
    f1 = lf.node_flux(ops, E1)[nodes]
    assert np.max(np.abs(f1 - f0)) < 1e-14 * np.max(np.abs(f0))


def test_staggered_energy_is_conserved_and_W_bounded(ops, cavity_mesh):
    """Leap-frog conserves Q = <E,E>_W + <B^{n-1/2},B^{n+1/2}>_S exactly; W (eq. 8) stays bounded."""
    rho, _ = spectral.power_iteration(ops, 200)
    dt = spectral.stable_dt(rho, 0.5)
    O = ops.geom.O
    B0 = meshgen.te_mode_b(O, 1, 1, 1.0, 0.5)
    rng = np.random.default_rng(2)
    st = lf.State(rng.standard_normal(ops.n_ei) * 0.1, B0 + 0.1 * rng.standard_normal(ops.n_t),
                  np.zeros(ops.n_ei), 0)
    Qs, Ws = [], []
    prevB = [st.B]

    def rec(s):
        Qs.append(lf.energy_Q(ops, s.E, prevB[0], s.B))
        Ws.append(lf.energy_W(ops, s.E, s.B))
        prevB[0] = s.B

    lf.run(ops, st, dt, 1000, record=rec)
    Qs = np.array(Qs)
    assert np.max(np.abs(Qs - Qs[0])) / Qs[0] < 1e-12
    Ws = np.array(Ws)
    assert Ws.max() / Ws.min() < 1.5
