"""Spectrum, stability bound (eq. 20), dispersion (eqs. 18-19) and cavity convergence pins."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import meshgen
from oracle import leapfrog as lf, mesh as om, operators, spectral


def _ops(ms):
    return operators.Operators(om.canonicalize(ms.xy, ms.tris))


@pytest.fixture(scope="module")
def small():
    return _ops(meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7))   # 256 triangles


def test_power_iteration_and_bracket_against_dense_eigenvalues(small):
    rho_dense = spectral.dense_rho(small)
    rho_pi, hist = spectral.power_iteration(small, 200, seed=3)
    lo, hi = spectral.certified_bracket(small)
    assert lo <= rho_dense <= hi
    assert rho_pi <= rho_dense * (1 + 1e-12)           # Rayleigh quotient: a lower bound
    assert rho_pi >= rho_dense * (1 - 2e-3)
    assert np.all(np.diff(hist) >= -1e-9 * hist[-1])    # monotone for a PSD operator


def test_complex_time_modes_against_dense_eigenpairs(small):
    """Section 2's method with deflation: the 6 highest omegas equal the dense ones, the modes
    are S-orthonormal, and each is an eigenvector of K (a dropped deflation collapses every mode
    onto the first; an unweighted one breaks the orthonormality)."""
    w, V = spectral.complex_time_modes(small, 6, iters=2000, seed=1)
    dense = spectral.dense_omegas(small)[::-1][:6]
    assert np.abs(w / dense - 1).max() < 1e-12
    G = V.T @ (small.w_B[:, None] * V)
    assert np.abs(G - np.eye(6)).max() < 1e-10
    for i in range(6):
        r = spectral.apply_K(small, V[:, i]) - w[i] ** 2 * V[:, i]
        assert np.sqrt(np.dot(small.w_B * r, r)) < 1e-6 * w[i] ** 2


def test_local_rayleigh_against_eigendecomposition(small):
    """v = K^p delta_j: in the symmetric frame u = S^(1/2) v = Kt^p sqrt(S_j) e_j, so the
    quotient is sum c_i^2 lam_i^(2p+1) / sum c_i^2 lam_i^(2p) with c_i = phi_i[j] (eigh of
    Kt = S^(1/2) K S^(-1/2)).  It is a lower bound of lambda_max and grows with p."""
    lam, phi = np.linalg.eigh(spectral.symmetric_K(small))
    lam = np.clip(lam, 0.0, None)
    for j in (0, 57, 131, small.n_t - 1):
        c2 = phi[j] ** 2
        prev = 0.0
        for p in (0, 1, 2, 5, 9):
            ref = np.sum(c2 * lam ** (2 * p + 1)) / np.sum(c2 * lam ** (2 * p))
            got = spectral.local_rayleigh(small, j, p)
            assert abs(got / ref - 1) < 1e-10, (j, p, got, ref)
            assert got <= lam[-1] * (1 + 1e-12)
            assert got >= prev * (1 - 1e-12)
            prev = got


def test_local_rayleigh_p0_equilateral_closed_form():
    """p = 0 gives K_jj; for an equilateral triangle of side a with three interior edges,
    |e|/d = sqrt(3) (d = 2 * inradius = a / sqrt(3)) and S = sqrt(3) a^2 / 4, so K_jj = 12/a^2."""
    a = 0.1
    ops = _ops(meshgen.equilateral_lattice(8, a))
    counts = np.bincount(ops.L_B.tocoo().col, minlength=ops.n_t)   # interior edges per triangle
    inner = np.where(counts == 3)[0]
    assert inner.size > 10
    for j in inner[:: max(1, inner.size // 7)]:
        assert abs(spectral.local_rayleigh(ops, int(j), 0) * a * a / 12.0 - 1) < 1e-12


def test_omegas_are_real_and_zero_modes_exist(small):
    """Section 2: w real (K PSD), and a static subspace (uniform B) of zero eigenvalues."""
    lam = np.linalg.eigvalsh(spectral.symmetric_K(small))
    assert lam.min() > -1e-9 * lam.max()
    assert np.sum(np.abs(lam) < 1e-9 * lam.max()) >= 1


def test_stability_bound_brute_force(small):
    """Eq. 20: leap-frog is bounded at dt = 0.99 * 2/rho and grows at 1.01 * 2/rho."""
    rho = spectral.dense_rho(small)
    rng = np.random.default_rng(0)
    res = {}
    for f in (0.99, 1.01):
        st = lf.State(rng.standard_normal(small.n_ei), rng.standard_normal(small.n_t),
                      np.zeros(small.n_ei), 0)
        w0 = lf.energy_W(small, st.E, st.B)
        with np.errstate(all="ignore"):
            st = lf.run(small, st, f * 2.0 / rho, 3000)
            res[f] = lf.energy_W(small, st.E, st.B) / w0
    assert res[0.99] < 1e3
    assert not np.isfinite(res[1.01]) or res[1.01] > 1e6


def test_yee_limit_on_merged_right_split_lattice():
    """Cocircular pairs merged: the right-split lattice is Yee's mesh; all modes match
    w^2 = (4/hx^2) sin^2(m pi hx / 2a) + (4/hy^2) sin^2(n pi hy / 2b)."""
    nx, ny, a, b = 13, 8, 1.2, 0.7
    ms = meshgen.right_split_lattice(nx, ny, a, b)
    m = om.canonicalize(ms.xy, ms.tris)
    mo = operators.MergedOperators(m)
    assert mo.n_c == (nx - 1) * (ny - 1)
    LB = mo.L_B.toarray()
    G = LB.T @ (mo.w_E[:, None] * LB)
    s = 1 / np.sqrt(mo.w_B)
    lam = np.sort(np.linalg.eigvalsh(s[:, None] * G * s[None, :]))
    hx, hy = a / (nx - 1), b / (ny - 1)
    M, N = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    yee = np.sort(((4 / hx ** 2) * np.sin(M * np.pi * hx / (2 * a)) ** 2
                   + (4 / hy ** 2) * np.sin(N * np.pi * hy / (2 * b)) ** 2).ravel())
    np.testing.assert_allclose(lam, yee, rtol=1e-10, atol=1e-9 * yee.max())


def _mode_series(ops, v, w, dt, nsteps):
    st = lf.State(np.zeros(ops.n_ei), v.copy(), np.zeros(ops.n_ei), 0)
    amp = []
    lf.run(ops, st, dt, nsteps, record=lambda s: amp.append(np.dot(ops.w_B * s.B, v)))
    return np.array(amp)


def test_leapfrog_dispersion_relation(small):
    """Eqs. 18-19: a mode of frequency w steps with sin(W dt/2) = w dt/2; the mode amplitude
    obeys b_{n+1} + b_{n-1} = 2 cos(W dt) b_n exactly."""
    lam, V = np.linalg.eigh(spectral.symmetric_K(small))
    rho = math.sqrt(lam[-1])
    for k in (len(lam) // 3, len(lam) - 1):
        w = math.sqrt(lam[k])
        v = V[:, k] / np.sqrt(small.w_B)        # back from the symmetric form
        v /= math.sqrt(np.dot(small.w_B * v, v))
        dt = 0.9 * 2 / rho
        b = _mode_series(small, v, w, dt, 60)
        Wdt = 2 * math.asin(w * dt / 2)
        np.testing.assert_allclose(b[2:] + b[:-2], 2 * math.cos(Wdt) * b[1:-1], atol=1e-9)


def _fit_frequency(t, a):
    a = a - a.mean()
    spec = np.abs(np.fft.rfft(a * np.hanning(a.size)))
    f0 = np.argmax(spec[1:]) + 1
    w0 = 2 * np.pi * f0 / (t[-1] - t[0]) * (a.size - 1) / a.size

    def resid(w):
        X = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
        c, *_ = np.linalg.lstsq(X, a, rcond=None)
        return np.sum((X @ c - a) ** 2)

    r = minimize_scalar(resid, bracket=(0.9 * w0, w0, 1.1 * w0), tol=1e-12)
    return r.x


@pytest.mark.parametrize("m,n", [(1, 1), (2, 1)])
def test_cavity_TE_frequency_converges(m, n):
    """North-star check (c): measured TE(m,n) frequency -> pi sqrt((m/a)^2 + (n/b)^2)."""
    a, b = 1.0, 0.5
    exact = math.pi * math.sqrt((m / a) ** 2 + (n / b) ** 2)
    errs = []
    for k in (16, 32, 64):
        ms = meshgen.cavity_lattice(k + 1, k // 2 + 1, a, b, seed=1001 + k)
        ops = _ops(ms)
        rho, _ = spectral.power_iteration(ops, 200)
        dt = 1.0 / rho
        B0 = meshgen.te_mode_b(ops.geom.O, m, n, a, b)
        T = 6 * 2 * math.pi / exact
        nsteps = int(T / dt)
        amp = []
        st = lf.State(np.zeros(ops.n_ei), B0.copy(), np.zeros(ops.n_ei), 0)
        lf.run(ops, st, dt, nsteps, record=lambda s: amp.append(np.dot(ops.w_B * s.B, B0)))
        t = (np.arange(nsteps) + 1.5) * dt
        W = _fit_frequency(t, np.array(amp))
        w = 2 / dt * math.sin(W * dt / 2)          # undo the leap-frog dispersion (eq. 19)
        errs.append(abs(w - exact) / exact)
    assert errs[0] < 0.02
    assert errs[2] < errs[0] / 3


def test_splitmix64_published_sequence():
    """SplitMix64 as in S. Vigna's reference generator splitmix64.c (the SplitMix scheme of
    Steele, Lea and Flood, OOPSLA 2014, with D. Stafford's Mix13 finaliser) from state 0 gives
    the published outputs 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f, 0xf88bb8a8724c81ec; the
    state advances by the golden-ratio increment between outputs.  The vectorised start vector
    draws the same numbers (entry k of seed s is the output for state s * 2^32 + k)."""
    golden, m64 = 0x9E3779B97F4A7C15, (1 << 64) - 1
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    x = 0
    for w in want:
        assert spectral.splitmix64(x) == w
        x = (x + golden) & m64
    seed, n = 7, 64
    v = spectral.start_vector(n, seed)
    ref = np.array([(spectral.splitmix64((seed << 32) + k) >> 11) * 2.0 ** -53 * 2.0 - 1.0 for k in range(n)])
    assert np.array_equal(v, ref)
