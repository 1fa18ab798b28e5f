"""Pins of the oracle's MINRES (the solver of Sec. 6) on small SPD systems (CPU, FP64).

* every iterate a_k is the minimiser of ||y - A a|| over the Krylov space
  span{y, A y, ..., A^{k-1} y}, computed independently by least squares on an
  orthonormal basis of that space (the defining property of MINRES);
* the recursively updated residual norm equals the true ||y - A a_k||;
* residual norms never increase, and the converged iterate is the direct solution.
"""
import numpy as np

import oracle as orc


def _system(n=40, seed=0, lam=1e-2):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 5))
    K = np.exp(-0.2 * ((X[:, None] - X[None]) ** 2).sum(-1))
    y = rng.standard_normal(n)
    return K, y, lam


def test_iterates_minimise_the_residual_over_the_krylov_space():
    K, y, lam = _system()
    A = K + lam * np.eye(len(y))
    mv = lambda x: K @ x
    for k in range(1, 9):
        a, it, rel, _ = orc.minres_solve(mv, y, lam, tol=0.0, max_iter=k)
        assert it == k
        B = np.stack([np.linalg.matrix_power(A, j) @ y for j in range(k)], axis=1)
        Q, _ = np.linalg.qr(B)
        c, *_ = np.linalg.lstsq(A @ Q, y, rcond=None)
        a_star = Q @ c
        assert np.max(np.abs(a - a_star)) <= 1e-8 * max(1.0, np.max(np.abs(a_star))), k
        true = np.linalg.norm(y - A @ a) / np.linalg.norm(y)
        assert abs(rel - true) <= 1e-10 + 1e-8 * true, k


def test_residuals_decrease_and_the_limit_is_the_direct_solution():
    K, y, lam = _system(n=60, seed=1, lam=1e-1)
    A = K + lam * np.eye(len(y))
    mv = lambda x: K @ x
    _, _, _, recs = orc.minres_solve(mv, y, lam, tol=0.0, max_iter=40, record_every=1)
    res = [np.linalg.norm(y - A @ r) for r in recs]
    assert all(b <= a * (1 + 1e-12) + 1e-14 for a, b in zip(res, res[1:]))
    a, it, rel, _ = orc.minres_solve(mv, y, lam, tol=1e-12, max_iter=1000)
    assert rel <= 1e-12
    np.testing.assert_allclose(a, np.linalg.solve(A, y), rtol=1e-9, atol=1e-9)


def test_minres_and_cg_agree_on_the_solution():
    K, y, lam = _system(n=50, seed=2)
    mv = lambda x: K @ x
    a1, *_ = orc.minres_solve(mv, y, lam, tol=1e-12)
    a2, *_ = orc.cg_solve(mv, y, lam, tol=1e-12)
    np.testing.assert_allclose(a1, a2, rtol=1e-8, atol=1e-8)
