"""Pins of the oracle's learned-rho pieces: features, forward, backward, Adam."""
import math

import numpy as np

import meshgen
from oracle import geometry, mesh as om, mlp, rcm


def _stored(ms):
    m = om.canonicalize(ms.xy, ms.tris)
    g = geometry.Geometry(m)
    t = rcm.device_tables(m, np.arange(m.n_tris))
    d = g.d[t["edge_caller"]]
    X, S, base = mlp.features(ms.xy, t["tri_nodes"], t["tri_code"], t["n_ei"], t["edge_tri"], d)
    return X, S, t, base


def test_equilateral_features_closed_form():
    ms = meshgen.equilateral_lattice(6, h=0.3)
    X, S, t, base = _stored(ms)
    np.testing.assert_allclose(X[:, 0:3], math.pi / 3, rtol=1e-12)
    e_over = math.sqrt(4 / math.sqrt(3))                 # |e| / sqrt(sqrt(3)/4 |e|^2)
    np.testing.assert_allclose(X[:, 3:6], math.log(e_over), rtol=1e-12)
    np.testing.assert_allclose(S, math.sqrt(3) / 4 * 0.09, rtol=1e-12)
    inner = (t["tri_code"] >> 1) < t["n_ei"]
    np.testing.assert_allclose(X[:, 6:9][inner], math.log(e_over / math.sqrt(3)), rtol=1e-11)
    assert np.all(X[:, 6:9][~inner] == mlp.BOUNDARY_LOG_D)
    np.testing.assert_allclose(X[:, 9:12], 0.0, atol=1e-12)
    # K_jj = (1/S) sum over interior edges of |e|/d = n_inner sqrt(3) / S
    n_inner = inner.sum(axis=1)
    ok = n_inner > 0
    np.testing.assert_allclose(base[ok], 0.5 * np.log(n_inner[ok] * math.sqrt(3) / S[ok]), rtol=1e-12)


def test_features_are_scale_free_and_angles_sum_to_pi():
    ms = meshgen.cavity_te11_mesh()
    X, S, _, base = _stored(ms)
    ms2 = meshgen.MeshArrays(ms.xy * 7.5, ms.tris, ms.h * 7.5, ms.boundary_node, {})
    X2, S2, _, base2 = _stored(ms2)
    np.testing.assert_allclose(X2, X, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(base2, base - math.log(7.5), rtol=1e-12)   # K scales as 1/L^2
    np.testing.assert_allclose(X[:, 0:3].sum(1), math.pi, rtol=1e-12)


def test_base_term_is_a_certified_lower_bound():
    """max_j exp(2 base_j) = max_j K_jj <= rho(M)^2 (Rayleigh quotient of a unit vector)."""
    from oracle import operators, spectral
    ms = meshgen.cavity_lattice(17, 9, 1.0, 0.5, seed=7)
    X, S, t, base = _stored(ms)
    ops = operators.Operators(om.canonicalize(ms.xy, ms.tris))
    rho = spectral.dense_rho(ops)
    assert math.exp(2 * base.max()) <= rho ** 2 * (1 + 1e-12)
    np.testing.assert_allclose(np.sort(np.exp(2 * base)), np.sort(spectral.diag_K(ops)), rtol=1e-12)


def test_forward_on_hand_set_weights():
    p = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = [np.array(a, copy=True) for a in mlp.unpack(p)]
    W1[0, 0] = 1.0          # h1_0 = relu(x0)
    W1[1, 1] = -1.0         # h1_1 = relu(-x1)
    W2[0, 0] = 2.0          # h2_0 = relu(2 h1_0 + 0.5)
    W2[1, 1] = 3.0          # h2_1 = relu(3 h1_1 - 1)
    b2[0], b2[1] = 0.5, -1.0
    w3[0], w3[1] = 1.0, 10.0
    p = mlp.pack(W1, b1, W2, b2, w3, -0.25)
    X = np.zeros((3, 12))
    X[:, 0] = [1.0, -2.0, 0.5]
    X[:, 1] = [-1.0, 3.0, -0.1]
    z, _ = mlp.forward(p, X)
    exp = []
    for x0, x1 in X[:, :2]:
        h0, h1_ = max(x0, 0), max(-x1, 0)
        exp.append(max(2 * h0 + 0.5, 0) + 10 * max(3 * h1_ - 1, 0) - 0.25)
    np.testing.assert_allclose(z, exp, rtol=1e-15)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(3) + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((7, 12))
    c = rng.standard_normal(7)
    z, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, c)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (np.dot(c, mlp.forward(p + e, X)[0]) - np.dot(c, mlp.forward(p - e, X)[0])) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_mesh_loss_gradient_matches_central_differences():
    ms = meshgen.cavity_te11_mesh()
    X, S, _, base = _stored(ms)
    p = mlp.init_params(5)
    L, g = mlp.mesh_loss_grad(p, X, base, math.log(400.0))
    rng = np.random.default_rng(1)
    h = 1e-6
    for i in rng.choice(mlp.N_PARAMS, 40, replace=False):
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.mesh_loss_grad(p + e, X, base, math.log(400.0))[0] -
              mlp.mesh_loss_grad(p - e, X, base, math.log(400.0))[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_a_signed_step():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = mlp.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=1e-9)


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    r = mlp.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even mantissa
    assert r[2] == 1.0 + 2 ** -7            # above the tie -> up
    assert abs(r[3] - -3.14159) <= 2 ** -8 * 4
    assert abs(r[4] / 1e-3 - 1) <= 2 ** -8
