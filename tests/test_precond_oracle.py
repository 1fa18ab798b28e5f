"""Pins of the learned-preconditioner oracle (CPU, FP64).

* the analytic gradient of the loss equals central finite differences;
* P r through the Woodbury formula equals the explicit matrix
  S (I + V V^T)^{-1} S, which is symmetric positive definite for any outputs;
* outputs that make P the exact inverse of an SPD system give zero loss.
"""
import numpy as np
import pytest

from oracle import precond as lp


def _toy(n=40, K=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, lp.N_FEAT))
    R = rng.standard_normal((n, K))
    E = rng.standard_normal((n, K))
    theta = lp.init_params(seed, out_scale=0.3)
    theta += 0.05 * rng.standard_normal(theta.shape)   # move off exact zeros of the ReLUs' inputs
    return theta, X, R, E


def test_gradient_matches_central_differences():
    theta, X, R, E = _toy()
    L, g = lp.loss_and_grad(theta, X, R, E, learn_diag=True)
    rng = np.random.default_rng(1)
    idx = rng.choice(lp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (lp.loss_and_grad(tp, X, R, E)[0] - lp.loss_and_grad(tm, X, R, E)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_initial_preconditioner_is_the_scaled_identity():
    theta = lp.init_params(7)
    X = np.random.default_rng(8).standard_normal((30, lp.N_FEAT))
    o, _ = lp.mlp_forward(theta, X)
    D, V = lp.outputs_to_DV(o, 5.0)
    np.testing.assert_allclose(D, 5.0, rtol=1e-12)


@pytest.mark.parametrize("scale", [1.0, 37.5])
def test_output_gradient_matches_central_differences(scale):
    rng = np.random.default_rng(2)
    n, K = 25, 2
    o = rng.standard_normal((n, lp.NOUT)) * 0.5
    R, E = rng.standard_normal((n, K)), rng.standard_normal((n, K))
    L, g = lp.loss_and_output_grad(o, R, E, scale, learn_diag=True)
    h = 1e-6
    for _ in range(40):
        i, j = rng.integers(n), rng.integers(lp.NOUT)
        op, om = o.copy(), o.copy()
        op[i, j] += h
        om[i, j] -= h
        fd = (lp.loss_and_output_grad(op, R, E, scale)[0] - lp.loss_and_output_grad(om, R, E, scale)[0]) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(fd))
    # the default (V-only) gradient equals the full one with the o_0 column zeroed
    L2, g2 = lp.loss_and_output_grad(o, R, E, scale)
    assert L2 == L and np.all(g2[:, 0] == 0) and np.array_equal(g2[:, 1:], g[:, 1:])


def test_woodbury_apply_equals_explicit_spd_matrix():
    rng = np.random.default_rng(3)
    n = 30
    o = rng.standard_normal((n, lp.NOUT))
    D, V = lp.outputs_to_DV(o)
    P = lp.P_matrix(D, V)
    r = rng.standard_normal(n)
    np.testing.assert_allclose(lp.apply_P(D, V, r), P @ r, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(P, P.T, atol=1e-12)
    assert np.linalg.eigvalsh(P).min() > 0


def test_exact_inverse_gives_zero_loss():
    """If A = S^-1 (I + V V^T) S^-1 then P = A^-1 and P r_k = e_k for r_k = A e_k."""
    rng = np.random.default_rng(4)
    n, K = 20, 3
    o = rng.standard_normal((n, lp.NOUT)) * 0.3
    D, V = lp.outputs_to_DV(o)
    Sinv = np.diag(1.0 / np.sqrt(D))
    A = Sinv @ (np.eye(n) + V @ V.T) @ Sinv
    E = rng.standard_normal((n, K))
    R = A @ E
    L, _ = lp.loss_and_output_grad(o, R, E)
    assert L < 1e-24


def test_data_scale_fits_corrections():
    rng = np.random.default_rng(5)
    R = rng.standard_normal((50, 4))
    E = 3.0 * R + 0.1 * rng.standard_normal((50, 4))
    c = lp.data_scale(R, E)
    # 1/c is the least-squares fit of r ~ (1/c) e
    ws = np.linspace(1 / c - 0.05, 1 / c + 0.05, 101)
    err = [np.sum((w * E - R) ** 2) for w in ws]
    assert abs(ws[int(np.argmin(err))] - 1 / c) < 0.0011
    # exact for r = A e restricted to one eigen-direction: c = 1 / eigenvalue
    v = rng.standard_normal(50)
    assert abs(lp.data_scale(0.01 * v[:, None], v[:, None]) - 100.0) < 1e-9
    # with o such that D = c (softplus(o0) = 1) and V = 0, P r = c r
    o = np.zeros((50, lp.NOUT))
    o[:, 0] = np.log(np.expm1(1.0))
    D, V = lp.outputs_to_DV(o, c)
    np.testing.assert_allclose(lp.apply_P(D, V, R[:, 0]), c * R[:, 0], rtol=1e-12)


def test_features_and_normalisation():
    d = np.array([0, 0, 2, 1, 0])
    t = np.array([1, 3, 3, 3, 0])
    M = np.diag([2.0, 3.0, 4.0])
    N = np.diag([5.0, 6.0, 7.0, 8.0])
    F = lp.pair_features(M, N, d, t, 3, 4, matvec=lambda v: 2.0 * v)
    np.testing.assert_allclose(F[:, 0], [2, 2, 4, 3, 2])
    np.testing.assert_allclose(F[:, 3], np.log1p([1, 3, 3, 3, 1]))
    np.testing.assert_allclose(F[:, 4], np.log1p(2.0))
    np.testing.assert_allclose(F[:, 5], np.log1p(2.0))   # K (g1 / mean g1) = 2 * 1
    assert lp.slog(-3.0) == -np.log1p(3.0)
    mu, sd = lp.normalisation(F)
    Xn = (F - mu) / sd
    np.testing.assert_allclose(Xn.mean(axis=0), 0, atol=1e-12)
