"""Pins of the oracle's kernel logistic regression by Newton's method (CPU, FP64).

* at the returned coefficients the optimality condition of the dual objective holds:
  lam a_i = y_i sigmoid(-y_i f_i) for every i (f = K a), checked directly;
* the Newton step solves the Newton system: K (W K + lam I) d = -K (g + lam a), against the
  explicit Hessian;
* the objective decreases every iteration and the solution does not depend on the scale of
  the labels' sign convention (y -> -y gives a -> -a).
"""
import numpy as np

import oracle as orc


def _problem(n=60, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 3))
    K = np.exp(-0.5 * ((X[:, None] - X[None]) ** 2).sum(-1))
    y = np.sign(X[:, 0] + 0.3 * rng.standard_normal(n))
    y[y == 0] = 1.0
    return K, y


def test_optimality_condition_at_the_solution():
    K, y = _problem()
    lam = 0.1
    a, it, rel = orc.klr_newton(lambda x: K @ x, y, lam)
    f = K @ a
    sig = 1.0 / (1.0 + np.exp(y * f))               # sigmoid(-y f)
    np.testing.assert_allclose(lam * a, y * sig, rtol=1e-8, atol=1e-10)
    assert rel <= 1e-10 and it < 30


def test_newton_step_solves_the_newton_system():
    K, y = _problem(n=40, seed=1)
    lam = 0.05
    mv = lambda x: K @ x
    a, _, _ = orc.klr_newton(mv, y, lam, newton_iters=1)   # one step from zero (full step accepted)
    f0 = np.zeros_like(y)
    s = 0.5 * (1.0 + np.tanh(0.5 * y * f0))
    g = -y * (1.0 - s)
    W = np.diag(s * (1.0 - s))
    H = K @ W @ K + lam * K
    d_ref = np.linalg.solve(H, -K @ g)
    np.testing.assert_allclose(a, d_ref, rtol=1e-7, atol=1e-9)


def test_objective_decreases_and_label_sign_symmetry():
    K, y = _problem(n=50, seed=2)
    lam = 0.2
    mv = lambda x: K @ x
    Js = []
    for k in range(1, 6):
        a, _, _ = orc.klr_newton(mv, y, lam, newton_iters=k)
        Js.append(orc.klr_objective(K @ a, a, y, lam))
    assert all(b <= a_ + 1e-12 for a_, b in zip(Js, Js[1:]))
    a1, _, _ = orc.klr_newton(mv, y, lam)
    a2, _, _ = orc.klr_newton(mv, -y, lam)
    np.testing.assert_allclose(a1, -a2, rtol=1e-9, atol=1e-12)
