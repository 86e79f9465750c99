"""Spectrum of M, power iteration for rho(M) and the leap-frog stability bound (oracle).

Test infrastructure only.  Section 2: the semi-discrete system dV/dt = M V conserves the eq. 7
energy, so M's eigenvalues are i*w with w real, and the eigenvectors are orthogonal in the eq. 7
metric.  Eliminating E, the B part of a mode solves K B = w^2 B with K = -L_E L_B, which is
self-adjoint and positive semi-definite in the S-weighted product (W_B K = L_B^T W_E L_B).
Hence rho(M) = sqrt(lambda_max(K)).

* ``power_iteration``: the "complex time" method: with t -> i t the modes grow like exp(w t),
  so repeated application of K to a random start vector, renormalised each step, converges to
  the top mode; lambda is read from the S-weighted Rayleigh quotient.  It approaches lambda_max
  from below, so it is a lower bound.
* ``certified_bracket``: max_j K_jj <= lambda_max (Rayleigh quotient of a unit vector) and
  Gershgorin on the symmetric S^{1/2} K S^{-1/2}: lambda_max <= max_j (K_jj + sum_q |e_q| /
  (d_q sqrt(S_j S_j'))).
* ``local_rayleigh``: the S-weighted Rayleigh quotient of K^p delta_j (p power steps of the
  same iteration, started at one triangle).  Like any Rayleigh quotient of K it is a lower
  bound of lambda_max; the learned-dt bracket takes it at the predicted argmax triangle.
* ``complex_time_modes``: the m highest modes by the same method with deflation: each next mode
  is iterated while the components along the modes already found are removed at every step,
  so that they cannot grow back from round-off; omega_i = sqrt of its Rayleigh quotient.
* ``stable_dt``: eq. 20: the leap-frog step is stable for w dt < 2 for every mode, so
  dt = safety * 2 / rho.  With a plasma density the current adds up to max(nbar) to w^2.
* ``start_vector``: the start vector of the power iteration, drawn per caller triangle id from
  the SplitMix64 counter-based generator (Steele, Lea, Flood 2014, constants as published) so
  that any implementation can reproduce it without sharing code.

Parity: pinned by tests/test_oracle_spectral.py (dense eigenvalues on small meshes, bracket
containment, Yee closed form on the merged right-split lattice, stability at 0.99 / 1.01 of
the bound, dispersion relation; the highest modes by deflation against a dense
eigendecomposition; the local Rayleigh quotient against its spectral form
sum c_i^2 lambda_i^(2p+1) / sum c_i^2 lambda_i^2p from a dense eigendecomposition, and K_jj =
12/a^2 on an equilateral lattice at p = 0).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of SplitMix64 for state x (the published mixing function)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def start_vector(n: int, seed: int) -> np.ndarray:
    """Entry k = uniform in [-1, 1): top 53 bits of splitmix64(seed * 2^32 + k), scaled.

    Vectorised copy of ``splitmix64`` (uint64 arithmetic wraps modulo 2^64 as required).
    """
    x = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def apply_K(ops, v: np.ndarray) -> np.ndarray:
    return -(ops.L_E @ (ops.L_B @ v))


def power_iteration(ops, iters: int = 200, v0: np.ndarray | None = None, seed: int = 0):
    """Return (rho, lambda history).  S-normalised power iteration on K."""
    v = np.array(v0, np.float64) if v0 is not None else start_vector(ops.L_B.shape[1], seed)
    S = ops.w_B
    v = v / np.sqrt(np.dot(S * v, v))
    lam = 0.0
    hist = []
    for _ in range(iters):
        w = apply_K(ops, v)
        lam = float(np.dot(S * v, w))           # Rayleigh quotient, v is S-normalised
        hist.append(lam)
        v = w / np.sqrt(np.dot(S * w, w))
    return float(np.sqrt(lam)), np.asarray(hist)


def local_rayleigh(ops, j0: int, p: int = 5) -> float:
    """<v, K v>_S / <v, v>_S for v = K^p delta_j0."""
    v = np.zeros(ops.L_B.shape[1])
    v[j0] = 1.0
    for _ in range(p):
        v = apply_K(ops, v)
    Kv = apply_K(ops, v)
    S = ops.w_B
    return float(np.dot(S * v, Kv) / np.dot(S * v, v))


def complex_time_modes(ops, m: int, iters: int = 2000, seed: int = 0):
    """(omegas in descending order, modes as S-normalised columns) of the m highest modes."""
    S = ops.w_B
    n = ops.L_B.shape[1]
    found, lams = [], []

    def deflate(v):
        for phi in found:
            v = v - np.dot(S * phi, v) * phi
        return v

    for i in range(m):
        v = deflate(start_vector(n, seed + i))
        v = v / np.sqrt(np.dot(S * v, v))
        lam = 0.0
        for _ in range(iters):
            w = deflate(apply_K(ops, v))
            lam = float(np.dot(S * v, w))
            v = w / np.sqrt(np.dot(S * w, w))
        found.append(v)
        lams.append(lam)
    return np.sqrt(np.clip(np.array(lams), 0.0, None)), np.stack(found, axis=1)


def diag_K(ops) -> np.ndarray:
    """K_jj = (1/S_j) sum over the interior edges q of j of |e_q| / d_q."""
    Kd = np.asarray((ops.L_B.multiply(ops.L_B)).T @ ops.w_E).ravel()
    return Kd / ops.w_B


def certified_bracket(ops):
    """(rho_lo, rho_hi) with rho_lo <= rho(M) <= rho_hi."""
    Kd = diag_K(ops)
    # off-diagonal magnitudes of S^{1/2} K S^{-1/2}: |e_q| / (d_q sqrt(S_j S_j'))
    A = ops.L_B.tocoo()
    rows_R = np.zeros(ops.n_ei, np.int64)
    rows_L = np.zeros(ops.n_ei, np.int64)
    pos = A.data > 0
    rows_R[A.row[pos]] = A.col[pos]
    rows_L[A.row[~pos]] = A.col[~pos]
    S = ops.w_B
    off = ops.elen / ops.d / np.sqrt(S[rows_R] * S[rows_L])
    row_sum = np.zeros(S.size)
    np.add.at(row_sum, rows_R, off)
    np.add.at(row_sum, rows_L, off)
    return float(np.sqrt(Kd.max())), float(np.sqrt((Kd + row_sum).max()))


def symmetric_K(ops) -> np.ndarray:
    """Dense S^{1/2} K S^{-1/2} = S^{-1/2} L_B^T W_E L_B S^{-1/2} (small meshes only)."""
    LB = ops.L_B.toarray()
    G = LB.T @ (ops.w_E[:, None] * LB)
    s = 1.0 / np.sqrt(ops.w_B)
    return s[:, None] * G * s[None, :]


def dense_omegas(ops) -> np.ndarray:
    """All mode frequencies w >= 0 (sqrt of the eigenvalues of K), ascending."""
    lam = sla.eigh(symmetric_K(ops), eigvals_only=True)
    return np.sqrt(np.clip(lam, 0.0, None))


def dense_rho(ops) -> float:
    return float(dense_omegas(ops)[-1])


def stable_dt(rho: float, safety: float = 0.5, nbar_max: float = 0.0) -> float:
    return safety * 2.0 / np.sqrt(rho * rho + nbar_max)
