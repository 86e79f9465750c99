"""Pins of the PML frame oracle (CPU only)."""
import math

import numpy as np
import pytest

import meshgen
from oracle import mesh as om, operators, pml, spectral


def test_framed_right_split_lattice_is_yee_for_every_mode():
    """A right-split lattice of square cells (cocircular pairs merged) inside a frame without
    decay is Yee's mesh of the whole box: its modes are
    w^2 = (4/h^2) (sin^2(m pi / 2 NX) + sin^2(n pi / 2 NY)), m < NX, n < NY, PEC outer walls.
    This fixes the frame's geometry, the dual lengths at the mesh boundary and every sign."""
    h, nx, ny = 0.125, 9, 7
    ms = meshgen.right_split_lattice(nx, ny, (nx - 1) * h, (ny - 1) * h)
    m = om.canonicalize(ms.xy, ms.tris)
    fo = pml.FramedOperators(m, 3, sigma_max=0.0, inner=operators.MergedOperators(m))
    assert (fo.NX, fo.NY, fo.n_if) == (14, 12, 28)
    lam = np.sort(np.linalg.eigvalsh(spectral.symmetric_K(fo)))
    M, N = np.meshgrid(np.arange(fo.NX), np.arange(fo.NY))
    yee = np.sort(((4 / h ** 2) * (np.sin(M * np.pi / (2 * fo.NX)) ** 2
                                   + np.sin(N * np.pi / (2 * fo.NY)) ** 2)).ravel())
    np.testing.assert_allclose(lam, yee, rtol=1e-10, atol=1e-10 * yee.max())


def _square(h=1 / 32, hole=False, seed=5):
    holes = [meshgen.polygon_triangle((0.5, 0.5), 0.2)] if hole else []
    ms = meshgen.graded_square(h, h, grade=0.0, holes=holes, seed=seed)
    return ms, om.canonicalize(ms.xy, ms.tris)


def test_framed_operators_are_adjoint_and_conserve_the_staggered_energy():
    """Without decay the combined operators keep eq. 10's adjointness
    W_E L_B = -(W_B L_E)^T, so the staggered energy sum w_E E^2 + sum S B^- B^+ is exact."""
    ms, m = _square(1 / 16, hole=True)
    fo = pml.FramedOperators(m, 4, sigma_max=0.0)
    LB, LE = fo.L_B.toarray(), fo.L_E.toarray()
    assert np.abs(fo.w_E[:, None] * LB + (fo.w_B[:, None] * LE).T).max() < 1e-12 * np.abs(LB).max()
    rho, _ = spectral.power_iteration(fo, 300)
    dt = 0.9 * 2 / rho
    rng = np.random.default_rng(4)
    E = np.zeros(fo.n_ei)
    Bs = fo.start_split(rng.standard_normal(fo.n_c))
    Q = []
    for _ in range(400):
        B_before = fo.P @ Bs
        E, Bs = pml.step(fo, E, Bs, dt)
        Q.append(np.dot(fo.w_E, E * E) + np.dot(fo.w_B, B_before * (fo.P @ Bs)))
    Q = np.asarray(Q)
    assert np.abs(Q - Q[0]).max() < 1e-12 * Q[0]


def _pulse_run(fo, b, dt, n_steps, n_samples):
    B0 = np.zeros(fo.n_c)
    B0[:fo.n_in] = b
    E, Bs = np.zeros(fo.n_ei), fo.start_split(B0)
    out = []
    for k in range(n_steps):
        E, Bs = pml.step(fo, E, Bs, dt)
        if (k + 1) % (n_steps // n_samples) == 0:
            out.append((fo.P @ Bs)[:fo.n_in].copy())
    return out


@pytest.mark.slow
def test_pml_matches_a_large_domain_until_its_echo_returns():
    """A pulse in the unit square: with a 12-cell layer the field inside stays within 5e-4
    (S-norm, relative to the start) of the same mesh in a 48-cell frame without decay, whose
    PEC wall echoes back only after t = 3; wider layers do better, and a layer whose Bx and By
    decay rates are swapped (a planted mistake) is more than 20 times worse; no layer at all
    reflects everything."""
    ms, m = _square()
    ref = pml.FramedOperators(m, 48, sigma_max=0.0)
    rho, _ = spectral.power_iteration(ref, 300)
    dt = 0.5 * 2 / rho
    C = m.xy[m.tris].mean(axis=1)
    r2 = ((C - 0.5) ** 2).sum(axis=1)
    b = (C[:, 0] - 0.5) * np.exp(-r2 / 0.12 ** 2)
    S = ref.w_B[:ref.n_in]
    nb = math.sqrt(np.dot(S, b * b))
    n = int(2.4 / dt)
    R = _pulse_run(ref, b, dt, n, 4)

    def err(fo):
        P = _pulse_run(fo, b, dt, n, 4)
        return max(math.sqrt(np.dot(S, (p - r) ** 2)) / nb for p, r in zip(P, R))

    e12 = err(pml.FramedOperators(m, 12))
    e8 = err(pml.FramedOperators(m, 8))
    e16 = err(pml.FramedOperators(m, 16))
    swapped = pml.FramedOperators(m, 12)
    k = swapped.n_in
    sx, sy = swapped.sigB[k:k + swapped.n_fc].copy(), swapped.sigB[k + swapped.n_fc:].copy()
    swapped.sigB[k:k + swapped.n_fc], swapped.sigB[k + swapped.n_fc:] = sy, sx
    e_sw = err(swapped)
    e_none = err(pml.FramedOperators(m, 12, sigma_max=0.0))
    assert e12 < 5e-4
    assert e16 < e12 < e8
    assert e_sw > 20 * e12
    assert e_none > 0.1


def _not_a_divided_rectangle():
    """A rotated cavity (sides not along the axes) and a square whose bottom nodes are not
    uniformly spaced."""
    c = meshgen.cavity_te11_mesh()
    R = np.array([[math.cos(0.5), -math.sin(0.5)], [math.sin(0.5), math.cos(0.5)]])
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.3, 0], [0.5, 1], [0, 0.5], [1, 0.5], [0.5, 0.5]])
    from scipy.spatial import Delaunay
    return [(c.xy @ R.T, c.tris), (xy, Delaunay(xy).simplices.astype(np.int32))]


def test_frame_needs_a_uniform_rectangular_boundary():
    for xy, tris in _not_a_divided_rectangle():
        with pytest.raises(ValueError):
            pml.FramedOperators(om.canonicalize(xy, tris), 4)


def test_framed_plasma_static_field_closed_form():
    """A discrete gradient E = G phi (phi zero on every boundary node) is curl-free, so B stays 0
    and the frame and the outer edges see nothing (to rounding); with uniform density n0 and nu = 0 the
    current makes every edge oscillate as E^{n+1} + E^{n-1} = (2 - n0 dt^2) E^n."""
    ms, m = _square(1 / 16, hole=True)
    fo = pml.FramedOperators(m, 4)
    rng = np.random.default_rng(6)
    bnd = np.zeros(m.n_nodes, bool)
    bnd[m.edges[~m.interior].ravel()] = True
    phi = np.where(bnd, 0.0, rng.standard_normal(m.n_nodes))
    e = m.edges[fo.inner.ie]
    E = np.zeros(fo.n_ei)
    E[:fo.inner.n_ei] = (phi[e[:, 1]] - phi[e[:, 0]]) / fo.inner.elen
    n0 = 3.0e3
    rho, _ = spectral.power_iteration(fo, 300)
    dt = 0.5 * 2.0 / math.sqrt(rho * rho + n0)
    nbar = pml.inner_nbar(fo, np.full(m.n_nodes, n0))
    Bs, j = np.zeros(fo.n_s), np.zeros(fo.inner.n_ei)
    hist = [E.copy()]
    for k in range(60):
        E, Bs, j = pml.step_plasma(fo, E, Bs, j, dt, nbar, 0.0, n=k)
        hist.append(E.copy())
    H = np.asarray(hist)
    assert np.abs(Bs).max() < 1e-12 * np.abs(H).max()
    assert np.abs(H[:, fo.inner.n_ei:]).max() < 1e-12 * np.abs(H).max()   # rounding only
    resid = H[2:] + H[:-2] - (2.0 - n0 * dt * dt) * H[1:-1]
    assert np.abs(resid).max() < 1e-12 * np.abs(H).max()
