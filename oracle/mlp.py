"""Learned spectral-radius predictor: features, MLP 12-64-64-1, max aggregation (oracle).

Test infrastructure only.  The paper sets dt from the highest mode (eq. 20) and finds it with
the "complex time" power iteration (Section 2); this predictor replaces that iteration for a new
mesh by a per-triangle network, checked against a certified bracket.

Features of triangle j (stored order, vertices rotated to start at the smallest caller node id,
edge q = (v_q, v_q+1); lengths are divided by sqrt(S_j) so that the features are scale free, and
ratios enter as logarithms, since the highest mode is set by ratios |e|/d spanning decades):
  x[0:3]  angle opposite edge q (at vertex v_q+2), radians
  x[3:6]  log(|e_q| / sqrt(S_j))
  x[6:9]  log(d_q / sqrt(S_j))  (|O_R O_L| of eq. 3; BOUNDARY_LOG_D for a boundary edge, i.e. a
          dual so long that the edge adds nothing to K)
  x[9:12] log(S_neighbour(q) / S_j)  (0 for a boundary edge)
Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3 (5,057 parameters).
Prediction: log rho_hat = max_j (z_j + base_j), base_j = log(K_jj) / 2 with
K_jj = (1/S_j) sum_q |e_q|/d_q the diagonal of K = -L_E L_B (interior edges only).  base_j is a
parameter-free function of the same geometry (max_j K_jj is a certified lower bound of rho^2),
so the network learns a bounded correction instead of the whole 1/d dependence; rho_hat =
max_j exp(z_j) sqrt(K_jj).
Loss per mesh: (log rho_hat - log rho_PI)^2; its gradient reaches only the argmax triangle.

Parameter vector layout (float): W1 [64x12] row-major, b1 [64], W2 [64x64] row-major, b2 [64],
w3 [64], b3 [1].

Parity: pinned by tests/test_oracle_mlp.py (closed-form features of equilateral meshes,
forward on hand-set weights, central finite differences of the analytic backward).
"""
from __future__ import annotations

import numpy as np

H = 64
D = 12
BOUNDARY_LOG_D = 4.0
N_PARAMS = H * D + H + H * H + H + H + 1

_OFF = {}
_o = 0
for _name, _n in (("W1", H * D), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)):
    _OFF[_name] = (_o, _o + _n)
    _o += _n


def unpack(p: np.ndarray):
    g = {k: p[a:b] for k, (a, b) in _OFF.items()}
    return (g["W1"].reshape(H, D), g["b1"], g["W2"].reshape(H, H), g["b2"], g["w3"], g["b3"][0])


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation from a seeded normal stream; b3 starts at log(1.25), a typical
    value of log(rho / sqrt(max K_jj))."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, D)) * np.sqrt(2.0 / D)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * np.sqrt(1.0 / H) * 0.01
    return pack(W1, np.zeros(H), W2, np.zeros(H), w3, np.log(1.25))


def features(xy: np.ndarray, tri_nodes: np.ndarray, tri_code: np.ndarray, n_ei: int,
             edge_tri: np.ndarray, d_stored: np.ndarray) -> np.ndarray:
    """(features, S, base) in the stored order.  tri_nodes / tri_code / edge_tri come from the
    device tables (see oracle.rcm.device_tables); d_stored[k] = |O_R O_L| of stored edge k."""
    t = tri_nodes
    p = [xy[t[:, q]] for q in range(3)]
    e = [p[(q + 1) % 3] - p[q] for q in range(3)]                  # edge q vector
    S = 0.5 * (e[0][:, 0] * (p[2] - p[0])[:, 1] - e[0][:, 1] * (p[2] - p[0])[:, 0])
    rs = 1.0 / np.sqrt(S)
    X = np.zeros((t.shape[0], D))
    kd = np.zeros(t.shape[0])
    for q in range(3):
        o = p[(q + 2) % 3]
        u = p[q] - o
        v = p[(q + 1) % 3] - o
        X[:, q] = np.arctan2(np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]), (u * v).sum(1))
        X[:, 3 + q] = np.log(np.hypot(e[q][:, 0], e[q][:, 1]) * rs)
        k = tri_code[:, q] >> 1
        inner = k < n_ei
        kk = np.where(inner, k, 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            X[:, 6 + q] = np.where(inner, np.log(d_stored[kk] * rs), BOUNDARY_LOG_D)
        other = np.where(edge_tri[kk, 0] == np.arange(t.shape[0]), edge_tri[kk, 1], edge_tri[kk, 0])
        X[:, 9 + q] = np.where(inner, np.log(S[other] / S), 0.0)
        kd += np.where(inner, np.hypot(e[q][:, 0], e[q][:, 1]) / d_stored[kk], 0.0)
    with np.errstate(divide="ignore"):
        base = 0.5 * np.log(kd / S)
    return X, S, base


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even) and back to float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p: np.ndarray, X: np.ndarray, round_bf16: bool = False):
    """z for every row of X, plus the activations needed by backward."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    if round_bf16:
        X, W1, W2 = bf16(X), bf16(W1), bf16(W2)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    if round_bf16:
        h1 = bf16(h1)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    return z, (X, a1, h1, a2, h2)


def backward(p: np.ndarray, cache, dz: np.ndarray) -> np.ndarray:
    """Gradient of sum_i dz_i z_i with respect to the parameter vector."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X, a1, h1, a2, h2 = cache
    g_w3 = h2.T @ dz
    g_b3 = dz.sum()
    d2 = np.outer(dz, w3) * (a2 > 0)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)
    g_W1 = d1.T @ X
    g_b1 = d1.sum(0)
    return pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def predict_log_rho(p: np.ndarray, X: np.ndarray, base: np.ndarray, round_bf16: bool = False):
    """(log rho_hat, argmax triangle)."""
    z, _ = forward(p, X, round_bf16)
    s = z + base
    j = int(np.argmax(s))
    return float(s[j]), j


def mesh_loss_grad(p, X, base, log_rho_pi, round_bf16=False):
    """Loss (log rho_hat - log rho_PI)^2 of one mesh and its parameter gradient (argmax row)."""
    lr, j = predict_log_rho(p, X, base, round_bf16)
    r = lr - log_rho_pi
    _, cache = forward(p, X[j:j + 1], round_bf16)
    g = backward(p, cache, np.array([2.0 * r]))
    return r * r, g


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
