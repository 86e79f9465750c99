"""Highest eigenmodes on the GPU (ue_modes, the complex-time method with deflation of Section 2)
against the FP64 oracle's one-mode-at-a-time deflation and a dense eigendecomposition."""
import numpy as np
import pytest

import meshgen
from oracle import mesh as om, operators, spectral

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


def _dense_pairs(ops):
    """All omegas (descending) and S-normalised modes (columns) from eigh of S^(1/2) K S^(-1/2)."""
    lam, phi = np.linalg.eigh(spectral.symmetric_K(ops))
    order = np.argsort(lam)[::-1]
    return np.sqrt(np.clip(lam[order], 0.0, None)), phi[:, order] / np.sqrt(ops.w_B)[:, None]


@pytest.mark.parametrize("which,n_modes,iters", [("lattice256", 6, 2000), ("cavity1024", 8, 3000)])
def test_modes_match_dense_eigenpairs(ue, which, n_modes, iters):
    """omega_i to 1e-10 of a dense eigendecomposition; each mode S-normalised, an eigenvector
    of K (residual through the oracle's operator), and the dense mode wherever the eigenvalue
    is isolated."""
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7) if which == "lattice256" else meshgen.cavity_te11_mesh()
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    dense, phi = _dense_pairs(ops)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-4)
    w, B = m.modes(n_modes, iters=iters, seed=3, vectors=True)
    m.close()
    assert np.all(np.diff(w) <= 0)
    assert np.abs(w / dense[:n_modes] - 1).max() < 1e-10
    S = ops.w_B
    for i in range(n_modes):
        b = B[i]
        assert abs(np.dot(S * b, b) - 1) < 1e-10
        r = spectral.apply_K(ops, b) - w[i] ** 2 * b
        assert np.sqrt(np.dot(S * r, r)) < 1e-6 * w[i] ** 2
        gap = min(dense[i] - dense[i + 1], dense[i - 1] - dense[i] if i > 0 else np.inf)
        if gap > 1e-3 * dense[i]:
            assert abs(abs(np.dot(S * b, phi[:, i])) - 1) < 1e-8


def test_modes_match_oracle_deflation(ue):
    """The block form and the oracle's one-mode-at-a-time deflation reach the same 6 highest
    omegas and modes on a mesh where both converge."""
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    w_o, V_o = spectral.complex_time_modes(ops, 6, 2000, seed=1)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-4)
    w, B = m.modes(6, iters=2000, seed=5, vectors=True)
    m.close()
    assert np.abs(w / w_o - 1).max() < 1e-10
    S = ops.w_B
    for i in range(6):
        assert abs(abs(np.dot(S * B[i], V_o[:, i])) - 1) < 1e-8


def test_modes_rejects_bad_arguments(ue):
    ms = meshgen.cavity_lattice(9, 5, 1.0, 0.5, seed=7)
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-4)
    for n in (0, 25):
        with pytest.raises(ue.UEError):
            m.modes(n, iters=10)
    with pytest.raises(ue.UEError):
        m.modes(4, iters=0)
    m.close()


def _analytic_te(a, b, count):
    """omega of the PEC rectangle's TE(m, n) modes, pi sqrt((m/a)^2 + (n/b)^2), (m, n) != (0, 0),
    ascending (c = 1)."""
    w = sorted(np.pi * np.hypot(mm / a, nn / b) for mm in range(12) for nn in range(12) if mm or nn)
    return np.array(w[:count])


@pytest.mark.parametrize("which", ["cavity1024", "cavity4k"])
def test_lowest_modes_match_dense_and_the_resonator(ue, which):
    """ue_modes_low: the 10 lowest omegas equal a dense eigendecomposition to 1e-9 (omega_0 = 0,
    the static field); the modes are S-normalised eigenvectors; and the nonzero omegas approach
    the rectangle's TE(m, n) frequencies pi sqrt((m/a)^2 + (n/b)^2) (Fig. 4's analytic curve),
    closer on the finer mesh."""
    ms = meshgen.cavity_te11_mesh() if which == "cavity1024" else meshgen.cavity_lattice(65, 33, 1.0, 0.5, seed=11)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    lam, phi = np.linalg.eigh(spectral.symmetric_K(ops))
    dense = np.sqrt(np.clip(lam, 0.0, None))                      # ascending
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-4)
    w, B = m.modes_low(10, iters=300, degree=24, seed=4, vectors=True)
    m.close()
    assert np.all(np.diff(w) >= -1e-9 * w[-1])
    assert w[0] < 1e-4 * w[1]                                     # the static field, omega^2 ~ rounding
    assert np.abs(w[1:] / dense[1:10] - 1).max() < 1e-9
    S = ops.w_B
    for i in range(10):
        b = B[i]
        assert abs(np.dot(S * b, b) - 1) < 1e-9
        r = spectral.apply_K(ops, b) - w[i] ** 2 * b
        assert np.sqrt(np.dot(S * r, r)) < 1e-5 * w[-1] ** 2
    exact = _analytic_te(1.0, 0.5, 9)
    err = np.abs(w[1:] / exact - 1)
    print(f"{which}: lowest omegas {np.round(w[1:6], 4)}, analytic {np.round(exact[:5], 4)}, max rel err {err.max():.2e}")
    assert err.max() < (0.01 if which == "cavity1024" else 0.003)


def test_lowest_modes_on_a_holed_graded_mesh(ue):
    """ue_modes_low away from the rectangle: a graded square with a PEC hole (no analytic
    spectrum), the 8 lowest omegas against a dense eigendecomposition to 1e-9, each mode an
    S-normalised eigenvector, and omega_0 the static field."""
    ms = meshgen.graded_square(0.03, 0.06, grade=0.3, seed=21,
                               holes=[meshgen.polygon_triangle((0.5, 0.5), 0.25)])
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    lam = np.linalg.eigvalsh(spectral.symmetric_K(ops))
    dense = np.sqrt(np.clip(lam, 0.0, None))
    m = ue.Mesh(ms.xy, ms.tris)
    m.geometry_build(dt_mode=ue.UE_DT_GIVEN, dt=1e-4)
    w, B = m.modes_low(8, iters=300, degree=24, seed=9, vectors=True)
    m.close()
    assert w[0] < 1e-4 * w[1]
    assert np.abs(w[1:] / dense[1:8] - 1).max() < 1e-9
    S = ops.w_B
    for i in range(8):
        assert abs(np.dot(S * B[i], B[i]) - 1) < 1e-9
        r = spectral.apply_K(ops, B[i]) - w[i] ** 2 * B[i]
        # two pairs of modes lie within 0.5% of each other here: their residuals converge
        # more slowly than their frequencies
        assert np.sqrt(np.dot(S * r, r)) < 1e-4 * w[-1] ** 2
