"""Pins of the oracle's multi-shift CG (one Krylov space for every lambda of a sweep), CPU FP64.

* after k steps, the iterate of every shift equals k steps of plain CG on that shifted system
  (shift invariance of the Krylov space; the collinear-residual recurrences must reproduce it);
* converged iterates equal the direct solutions, and the residual estimates the true residuals.
"""
import numpy as np

import oracle as orc


def _system(n=50, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 4))
    K = np.exp(-0.25 * ((X[:, None] - X[None]) ** 2).sum(-1))
    return K, rng.standard_normal(n)


def test_iterates_equal_plain_cg_on_each_shift():
    K, y = _system()
    mv = lambda x: K @ x
    lams = [1e-2, 3e-1, 1.0, 2e-2]
    for k in range(1, 7):
        X, it, _ = orc.cg_multishift(mv, y, lams, tol=0.0, max_iter=k)
        assert it == k
        for s, lam in enumerate(lams):
            a, its, _ = orc.cg_solve(mv, y, lam, tol=0.0, max_iter=k)
            assert its == k
            assert np.max(np.abs(X[:, s] - a)) <= 1e-9 * max(1.0, np.max(np.abs(a))), (k, s)


def test_converged_shifts_are_the_direct_solutions():
    K, y = _system(n=70, seed=1)
    mv = lambda x: K @ x
    lams = [1e-3, 1e-2, 1e-1, 1.0]
    X, it, res = orc.cg_multishift(mv, y, lams, tol=1e-10, max_iter=5000)
    for s, lam in enumerate(lams):
        A = K + lam * np.eye(len(y))
        np.testing.assert_allclose(X[:, s], np.linalg.solve(A, y), rtol=1e-6, atol=1e-7 / lam)
        true = np.linalg.norm(y - A @ X[:, s]) / np.linalg.norm(y)
        assert res[s] <= 1e-10 and true <= 1e-8, (s, res[s], true)
