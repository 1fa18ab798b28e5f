"""Pins of the oracle's squared-hinge SVM by Newton's method over active sets (CPU, FP64).

* the returned coefficients satisfy the optimality conditions: a = 0 outside the active set
  S = {i : y_i f_i < 1} (f = K a), and (K_SS + lam I) a_S = y_S on it, against a dense solve;
* an independent minimiser of the same objective (scipy's L-BFGS on J with its gradient
  2 K (lam a + [y f < 1] (f - y))) reaches the same objective value and the same f;
* when every pair stays active (large lam) the solution is the kernel ridge regression solution
  (K + lam I)^-1 y of Eq. 1;
* flipping every label flips the solution (y -> -y gives a -> -a), and the objective never
  increases from one Newton iterate to the next.

The hinge-loss SVM by sub-gradients (Pegasos in the coefficients): its first step is y / (lam n)
in closed form, it flips with the labels, and its objective approaches, from above, the optimum
computed independently from the dual quadratic program (scipy's bounded L-BFGS).
"""
import numpy as np
import pytest

import oracle as orc


def _problem(n=70, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 3))
    K = np.exp(-0.5 * ((X[:, None] - X[None]) ** 2).sum(-1))
    y = np.sign(X[:, 0] + 0.4 * rng.standard_normal(n))
    y[y == 0] = 1.0
    return K, y


def test_optimality_conditions_at_the_solution():
    K, y = _problem()
    lam = 0.1
    a, it, cg, ok = orc.svm_newton(lambda x: K @ x, y, lam)
    assert ok and it < 30
    f = K @ a
    S = y * f < 1.0
    assert 0 < S.sum() < len(y)                     # some pairs are inside the margin, some not
    assert np.all(a[~S] == 0.0)
    want = np.linalg.solve(K[np.ix_(S, S)] + lam * np.eye(S.sum()), y[S])
    np.testing.assert_allclose(a[S], want, rtol=1e-9, atol=1e-11)


def test_independent_minimiser_reaches_the_same_objective():
    scipy_opt = pytest.importorskip("scipy.optimize")
    K, y = _problem(n=50, seed=1)
    lam = 0.05
    a, _, _, ok = orc.svm_newton(lambda x: K @ x, y, lam)
    assert ok

    def J(b):
        f = K @ b
        return lam * b @ f + np.sum(np.maximum(0.0, 1.0 - y * f) ** 2)

    def grad(b):
        f = K @ b
        act = (y * f < 1.0).astype(float)
        return 2.0 * K @ (lam * b + act * (f - y))

    res = scipy_opt.minimize(J, np.zeros_like(y), jac=grad, method="L-BFGS-B",
                             options={"maxiter": 20000, "gtol": 1e-12, "ftol": 1e-15})
    assert abs(J(a) - res.fun) <= 1e-8 * max(1.0, abs(res.fun))
    assert J(a) <= res.fun + 1e-10
    np.testing.assert_allclose(K @ a, K @ res.x, rtol=0, atol=1e-4)
    assert abs(orc.svm_objective(K @ a, a, y, lam) - J(a)) <= 1e-12 * J(a)


def test_all_active_reduces_to_kernel_ridge_regression():
    K, y = _problem(n=40, seed=2)
    lam = 50.0                                      # f = K a stays small: every y_i f_i < 1
    a, it, _, ok = orc.svm_newton(lambda x: K @ x, y, lam)
    assert ok
    assert np.all(y * (K @ a) < 1.0)
    np.testing.assert_allclose(a, np.linalg.solve(K + lam * np.eye(len(y)), y), rtol=1e-10, atol=1e-13)


def test_label_flip_and_monotone_objective():
    K, y = _problem(n=60, seed=3)
    lam = 0.2
    mv = lambda x: K @ x
    a, _, _, _ = orc.svm_newton(mv, y, lam)
    b, _, _, _ = orc.svm_newton(mv, -y, lam)
    np.testing.assert_allclose(b, -a, rtol=1e-10, atol=1e-12)
    prev = np.inf
    for k in range(1, 8):
        ak, _, _, _ = orc.svm_newton(mv, y, lam, newton_iters=k)
        Jk = orc.svm_objective(K @ ak, ak, y, lam)
        assert Jk <= prev + 1e-12
        prev = Jk


# ---------------------------------------------------------------- hinge loss, sub-gradients
def _dual_optimum(K, y, lam):
    """The hinge SVM optimum from its dual, a box-constrained QP solved by scipy's L-BFGS-B:
    max_alpha sum(alpha) / n - (1 / (2 lam n^2)) alpha^T (yy^T o K) alpha, 0 <= alpha <= 1, and
    a* = alpha * y / (lam n)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    n = len(y)
    Q = (y[:, None] * y[None, :]) * K / (lam * n * n)
    fun = lambda al: 0.5 * al @ Q @ al - al.sum() / n
    jac = lambda al: Q @ al - 1.0 / n
    res = scipy_opt.minimize(fun, np.full(n, 0.5), jac=jac, method="L-BFGS-B", bounds=[(0.0, 1.0)] * n,
                             options={"maxiter": 50000, "gtol": 1e-14, "ftol": 1e-16})
    return res.x * y / (lam * n)


def test_hinge_subgradient_first_step_and_label_flip():
    K, y = _problem(n=30, seed=4)
    lam = 0.1
    mv = lambda x: K @ x
    a1, f1, _ = orc.hinge_svm_subgradient(mv, y, lam, 1)
    np.testing.assert_allclose(a1, y / (lam * len(y)), rtol=0, atol=0)   # f = 0: every pair active
    np.testing.assert_allclose(f1, K @ a1, rtol=1e-14, atol=1e-15)
    a, _, _ = orc.hinge_svm_subgradient(mv, y, lam, 50)
    b, _, _ = orc.hinge_svm_subgradient(mv, -y, lam, 50)
    np.testing.assert_allclose(b, -a, rtol=0, atol=1e-15)


def test_hinge_subgradient_approaches_the_dual_optimum():
    K, y = _problem(n=40, seed=5)
    lam = 0.1
    mv = lambda x: K @ x
    a_star = _dual_optimum(K, y, lam)
    J_star = orc.hinge_svm_objective(K @ a_star, a_star, y, lam)
    gaps = []
    for T in (100, 1000, 10000):
        a, f, J = orc.hinge_svm_subgradient(mv, y, lam, T)
        assert J >= J_star - 1e-9                       # the dual optimum is a lower bound
        gaps.append(J - J_star)
    assert gaps[2] < gaps[0] and gaps[2] <= 2e-3 * J_star
