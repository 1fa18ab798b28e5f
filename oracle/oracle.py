"""Plain FP64 CPU oracle: definitions from the paper, written out slowly.

TEST INFRASTRUCTURE ONLY.  Loaded by the tests, the smoke check and the CPU
baseline of the benchmark; never by the product path.  Shares no code with
the CUDA library.

Contents (each function cites the passage it follows):
  * kernel kinds of Table 4b and the pairwise kernel value / matrix / matvec
    (C, ``gvt_oracle.c``): the explicit O(n * nhat) product, Sec. 4.9 approach 1;
  * Gaussian base kernel (C), Sec. 5.2 with the squared norm;
  * explicit operators of Definition 1 (commutation P, unification Q, PQ) and
    the sampling operator R of Sec. 3, as dense 0/1 matrices;
  * kernel ridge regression, Eq. 1: dense Cholesky solve and plain CG;
  * the complete-data closed form through eigendecompositions (Sec. 1).

Every function here is pinned by ``tests/test_oracle_pins.py`` against values
the paper prints, closed forms, invariants or brute force.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

KINDS = ["kronecker", "gaussian", "linear", "poly2d", "cartesian",
         "symmetric", "antisymmetric", "ranking", "mlpk"]
HOMOGENEOUS = {"symmetric", "antisymmetric", "ranking", "mlpk"}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        p = ctypes.c_void_p
        lib.orc_kernel_value.argtypes = [i32, p, i64, p, i64, i64, i64, i64, i64, p]
        lib.orc_kernel_value.restype = i32
        lib.orc_kernel_matrix.argtypes = [i32, p, i64, p, i64, p, p, i64, p, p, i64, p]
        lib.orc_kernel_matrix.restype = i32
        lib.orc_pairwise_matvec.argtypes = [i32, p, i64, p, i64, p, p, i64, p, p, i64,
                                            p, i64, p, i32]
        lib.orc_pairwise_matvec.restype = i32
        lib.orc_gaussian_kernel.argtypes = [p, i64, p, i64, i64, dbl, p, i32]
        lib.orc_gaussian_kernel.restype = i32
        lib.orc_compensated_sum.argtypes = [p, i64]
        lib.orc_compensated_sum.restype = dbl
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = i32
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def kind_id(kind):
    return KINDS.index(kind)


def num_threads():
    """Threads the C oracle uses by default (OpenMP)."""
    return int(_load().orc_num_threads())


def _mats(kind, M, N):
    M = _f64(M)
    N = M if (kind in HOMOGENEOUS or N is None) else _f64(N)
    return M, N


def kernel_value(kind, M, N, a, b, c, e):
    """k((a,b),(c,e)) from Table 4b."""
    M, N = _mats(kind, M, N)
    out = np.zeros(1)
    rc = _load().orc_kernel_value(kind_id(kind), _ptr(M), M.shape[1], _ptr(N), N.shape[1],
                                  int(a), int(b), int(c), int(e), _ptr(out))
    assert rc == 0
    return float(out[0])


def kernel_matrix(kind, M, N, d_out, t_out, d_in, t_in):
    """Explicit block R(dhat,that) K_op R(d,t)^T with entries from Table 4b."""
    M, N = _mats(kind, M, N)
    d_out, t_out, d_in, t_in = map(_i32, (d_out, t_out, d_in, t_in))
    K = np.zeros((len(d_out), len(d_in)))
    rc = _load().orc_kernel_matrix(kind_id(kind), _ptr(M), M.shape[1], _ptr(N), N.shape[1],
                                   _ptr(d_out), _ptr(t_out), len(d_out),
                                   _ptr(d_in), _ptr(t_in), len(d_in), _ptr(K))
    assert rc == 0
    return K


def pairwise_matvec(kind, M, N, d_out, t_out, d_in, t_in, v, nthreads=0):
    """u = R(dhat,that) K_op R(d,t)^T v, as the plain double sum (Sec. 4.9, approach 1).

    ``v`` is (n_in,) or (n_in, k); the result has the matching shape.
    Compensated FP64 sums; O(n_in * n_out * k) kernel evaluations.
    """
    M, N = _mats(kind, M, N)
    d_out, t_out, d_in, t_in = map(_i32, (d_out, t_out, d_in, t_in))
    v = np.asarray(v, dtype=np.float64)
    vec = v.ndim == 1
    V = v.reshape(len(d_in), -1)
    k = V.shape[1]
    Vc = np.asfortranarray(V)
    U = np.zeros((len(d_out), k), order="F")
    rc = _load().orc_pairwise_matvec(kind_id(kind), _ptr(M), M.shape[1], _ptr(N), N.shape[1],
                                     _ptr(d_out), _ptr(t_out), len(d_out),
                                     _ptr(d_in), _ptr(t_in), len(d_in),
                                     _ptr(Vc), k, _ptr(U), int(nthreads))
    assert rc == 0
    U = np.ascontiguousarray(U)
    return U[:, 0] if vec else U


def gaussian_kernel(X, Y=None, gamma=1.0, nthreads=0):
    """K[a,b] = exp(-gamma ||X_a - Y_b||^2), Sec. 5.2 (squared norm reading)."""
    X = _f64(X)
    Y = X if Y is None else _f64(Y)
    assert X.shape[1] == Y.shape[1]
    K = np.zeros((X.shape[0], Y.shape[0]))
    _load().orc_gaussian_kernel(_ptr(X), X.shape[0], _ptr(Y), Y.shape[0], X.shape[1],
                                float(gamma), _ptr(K), int(nthreads))
    return K


def tanimoto_kernel(Xb, Yb=None):
    """Tanimoto (MinMax) kernel of binary vectors, Sec. 5:
    K[a,b] = sum_i min(x_ai, y_bi) / sum_i max(x_ai, y_bi); 1 when both vectors are zero."""
    X = np.asarray(Xb, dtype=np.float64)
    Y = X if Yb is None else np.asarray(Yb, dtype=np.float64)
    K = np.ones((X.shape[0], Y.shape[0]))
    for a in range(X.shape[0]):
        mn = np.minimum(X[a][None, :], Y).sum(axis=1)
        mx = np.maximum(X[a][None, :], Y).sum(axis=1)
        nz = mx > 0
        K[a, nz] = mn[nz] / mx[nz]
    return K


def auc(scores, labels):
    """Area under the ROC curve, the paper's evaluation measure (Sec. 6): the fraction of
    (positive, negative) pairs whose positive scores higher, ties counting one half.  Computed
    from average ranks (the Mann-Whitney statistic)."""
    s = np.asarray(scores, dtype=np.float64)
    yb = np.asarray(labels).astype(bool)
    n_pos, n_neg = int(yb.sum()), int((~yb).sum())
    assert n_pos > 0 and n_neg > 0
    order = np.argsort(s, kind="mergesort")
    ranks = np.empty(len(s))
    ss = s[order]
    i = 0
    while i < len(s):          # average rank (1-based) over each run of equal scores
        j = i
        while j + 1 < len(s) and ss[j + 1] == ss[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1.0
        i = j + 1
    return float((ranks[yb].sum() - n_pos * (n_pos + 1) / 2.0) / (n_pos * n_neg))


def linear_kernel(X, Y=None):
    """Linear base kernel K[a,b] = <X_a, Y_b> (Sec. 5, the Metz data: rows of a similarity matrix
    used as feature vectors).  A plain matrix product in FP64."""
    X = _f64(X)
    Y = X if Y is None else _f64(Y)
    assert X.shape[1] == Y.shape[1]
    return X @ Y.T


def compensated_sum(x):
    x = _f64(x)
    return float(_load().orc_compensated_sum(_ptr(x), len(x)))


# --------------------------------------------------------------------------
# Operators of Definition 1 and the sampling operator of Sec. 3, as matrices.
# Pairs are numbered in the natural (lexicographic) order: (x, y) -> x*|Y| + y.
# --------------------------------------------------------------------------

def commutation_P(nD, nT):
    """P in R^{(T x D) x (D x T)}: P[(t,d),(dbar,tbar)] = 1 iff d=dbar and t=tbar."""
    P = np.zeros((nT * nD, nD * nT))
    for t in range(nT):
        for d in range(nD):
            P[t * nD + d, d * nT + t] = 1.0
    return P


def unification_Q(nD, nT):
    """Q in R^{(D x T) x (D x D)}: Q[(d,t),(dbar,dbar')] = 1 iff d = dbar = dbar'."""
    Q = np.zeros((nD * nT, nD * nD))
    for d in range(nD):
        for t in range(nT):
            Q[d * nT + t, d * nD + d] = 1.0
    return Q


def sampling_R(d, t, nD, nT):
    """R(d,t) in R^{n x (D x T)}: row i selects the pair (d_i, t_i) (Sec. 3)."""
    R = np.zeros((len(d), nD * nT))
    for i, (a, b) in enumerate(zip(d, t)):
        R[i, int(a) * nT + int(b)] = 1.0
    return R


# --------------------------------------------------------------------------
# Kernel ridge regression, Eq. 1: (K + lambda I) a = y.
# --------------------------------------------------------------------------

def krr_solve_dense(K, y, lam):
    """Solve (K + lam I) a = y by a dense Cholesky factorisation (library primitive)."""
    from scipy.linalg import cho_factor, cho_solve
    A = np.array(K, dtype=np.float64) + lam * np.eye(K.shape[0])
    return cho_solve(cho_factor(A, lower=True), np.asarray(y, dtype=np.float64))


def krr_complete_closed_form(M, N, Y, lam):
    """Complete data (every (d,t) pair present, natural order): solve
    (M kron N + lam I) vec(A) = vec(Y) through the eigendecompositions
    M = U diag(s) U^T, N = V diag(w) V^T (the closed form for complete data
    that Sec. 1 cites).  Y is q x m with Y[t, d] = y_(d,t); returns A, q x m.
    """
    s, U = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    w, V = np.linalg.eigh(np.asarray(N, dtype=np.float64))
    C = V.T @ Y @ U                      # coordinates in the eigenbasis
    C = C / (np.outer(w, s) + lam)       # (M kron N + lam I) is diagonal there
    return V @ C @ U.T


def cg_solve(matvec, y, lam, tol=1e-6, max_iter=10000, x0=None):
    """Plain conjugate gradients for (K + lam I) a = y (K symmetric PSD).

    ``matvec(p)`` returns K p.  Stops when ||y - (K+lam I)a||_2 / ||y||_2 <= tol
    for the recursively updated residual.  Returns (a, iterations, rel_res).
    """
    y = np.asarray(y, dtype=np.float64)
    a = np.zeros_like(y) if x0 is None else np.array(x0, dtype=np.float64)
    r = y - (matvec(a) + lam * a) if x0 is not None else y.copy()
    p = r.copy()
    rr = float(r @ r)
    ynorm = float(np.sqrt(y @ y))
    if ynorm == 0.0:
        return a, 0, 0.0
    it = 0
    while np.sqrt(rr) / ynorm > tol and it < max_iter:
        w = matvec(p) + lam * p
        alpha = rr / float(p @ w)
        a += alpha * p
        r -= alpha * w
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return a, it, float(np.sqrt(rr) / ynorm)


def cg_multishift(matvec, y, lams, tol=1e-6, max_iter=10000):
    """Multi-shift CG: (K + lam_s I) a_s = y for every lam_s from one Krylov space.

    CG runs on the base system A = K + lam_0 I, lam_0 = min(lams); for the shift
    sigma = lam_s - lam_0 the residual stays collinear, r_s = zeta r, with
        zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
                     (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + sigma alpha_k)),
        alpha^s_k = alpha_k zeta_{k+1} / zeta_k,   beta^s_k = (zeta_{k+1} / zeta_k)^2 beta_k,
        a_s += alpha^s_k p_s,   p_s = zeta_{k+1} r_{k+1} + beta^s_k p_s,
    starting from alpha_{-1} = 1, beta_{-1} = 0, zeta_{-1} = zeta_0 = 1, p_s = y.
    A shift stops updating once |zeta| ||r|| <= tol ||y||.  Returns (A: n x S, iterations,
    relative residual estimates |zeta_s| ||r|| / ||y|| per shift, taken when it stopped).
    """
    y = np.asarray(y, dtype=np.float64)
    lams = np.asarray(lams, dtype=np.float64)
    S, n = len(lams), len(y)
    lam0 = float(lams.min())
    sig = lams - lam0
    X = np.zeros((n, S))
    P = np.tile(y[:, None], (1, S))
    r = y.copy()
    p = y.copy()
    rr = float(r @ r)
    ynorm = np.sqrt(rr)
    if ynorm == 0.0:
        return X, 0, np.zeros(S)
    z_prev, z = np.ones(S), np.ones(S)
    alpha_prev, beta_prev = 1.0, 0.0
    done = np.zeros(S, bool)
    res_final = np.zeros(S)
    it = 0
    while True:
        res = np.abs(z) * np.sqrt(rr) / ynorm
        newly = ~done & ((res <= tol) | (it >= max_iter))
        res_final[newly] = res[newly]
        done |= newly
        if done.all():
            break
        w = matvec(p) + lam0 * p
        alpha = rr / float(p @ w)
        r_new = r - alpha * w
        rr_new = float(r_new @ r_new)
        beta = rr_new / rr
        z_next = z * z_prev * alpha_prev / (alpha * beta_prev * (z_prev - z) + z_prev * alpha_prev * (1.0 + sig * alpha))
        alpha_s = alpha * z_next / z
        beta_s = (z_next / z) ** 2 * beta
        for s in range(S):
            if not done[s]:
                X[:, s] += alpha_s[s] * P[:, s]
                P[:, s] = z_next[s] * r_new + beta_s[s] * P[:, s]
        p = r_new + beta * p
        r, rr = r_new, rr_new
        z_prev, z = np.where(done, z_prev, z), np.where(done, z, z_next)
        alpha_prev, beta_prev = alpha, beta
        it += 1
    return X, it, res_final


def klr_objective(f, a, y, lam):
    """J = sum_i log(1 + exp(-y_i f_i)) + (lam / 2) a^T f  with f = K a (kernel logistic regression)."""
    return float(np.sum(np.logaddexp(0.0, -y * f)) + 0.5 * lam * float(a @ f))


def klr_newton(matvec, y, lam, newton_iters=30, cg_tol=1e-10, grad_tol=1e-10):
    """Kernel logistic regression by Newton's method on the dual coefficients a (f = K a).

    Gradient K (g + lam a) with g_i = -y_i sigmoid(-y_i f_i); Hessian K (W K + lam I), W_ii =
    s_i (1 - s_i).  The Newton step solves (W K + lam I) d = b, b = -(g + lam a), through the SPD
    system (W^1/2 K W^1/2 + lam I) c = W^1/2 K b and d = (b - W^1/2 c) / lam; a backtracking
    line search halves the step until J decreases.  Stops when ||g + lam a|| <= grad_tol ||y||.
    Returns (a, newton iterations, ||g + lam a|| / ||y||)."""
    y = np.asarray(y, dtype=np.float64)
    a = np.zeros_like(y)
    f = np.zeros_like(y)
    it = 0
    rel = np.inf
    while it < newton_iters:
        s = 0.5 * (1.0 + np.tanh(0.5 * y * f))       # sigmoid(y f)
        g = -y * (1.0 - s)                            # d/df log(1 + exp(-y f))
        b = -(g + lam * a)
        rel = float(np.linalg.norm(b) / np.linalg.norm(y))
        if rel <= grad_tol:
            break
        w = s * (1.0 - s)
        sw = np.sqrt(w)
        Kb = matvec(b)
        c, _, _ = cg_solve(lambda x: sw * matvec(sw * x), sw * Kb, lam, tol=cg_tol, max_iter=100000)
        d = (b - sw * c) / lam
        Kd = matvec(d)
        J0 = klr_objective(f, a, y, lam)
        step = 1.0
        while step > 1e-12:
            if klr_objective(f + step * Kd, a + step * d, y, lam) <= J0:
                break
            step *= 0.5
        a = a + step * d
        f = f + step * Kd
        it += 1
    return a, it, rel


def svm_objective(f, a, y, lam):
    """J = lam a^T f + sum_i max(0, 1 - y_i f_i)^2 with f = K a: the support vector machine with
    the squared hinge loss, in the coefficients a of the representer theorem (a regularised kernel
    method driven by the same product, Sec. 7)."""
    return float(lam * float(a @ f) + np.sum(np.maximum(0.0, 1.0 - y * f) ** 2))


def svm_newton(matvec, y, lam, newton_iters=50, cg_tol=1e-12):
    """Squared-hinge SVM by Newton's method over active sets (Chapelle, "Training a support vector
    machine in the primal", 2007).  With S = {i : y_i f_i < 1} the Newton point a+ solves
    (K_SS + lam I) a+_S = y_S with a+ = 0 outside S (on S the loss is (y_i - f_i)^2).  A
    backtracking line search halves the step from a toward a+ until J does not increase.  The
    solution is found when a full step leaves S unchanged: then a is zero outside S, solves the
    system on S, and S is exactly the set with y_i f_i < 1.
    Returns (a, newton iterations, total CG iterations, converged)."""
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    a = np.zeros(n)
    f = np.zeros(n)
    S_prev, full_prev, cg_total = None, False, 0
    for it in range(newton_iters + 1):
        S = y * f < 1.0
        if S_prev is not None and full_prev and np.array_equal(S, S_prev):
            return a, it, cg_total, True
        if it == newton_iters:
            break
        idx = np.flatnonzero(S)

        def sub(x):                          # K_SS x through the full product
            z = np.zeros(n)
            z[idx] = x
            return matvec(z)[idx]

        a_plus = np.zeros(n)
        if len(idx):
            b, k, _ = cg_solve(sub, y[idx], lam, tol=cg_tol, max_iter=100000)
            a_plus[idx] = b
            cg_total += k
        f_plus = matvec(a_plus)
        J0 = svm_objective(f, a, y, lam)
        t = 1.0
        while t > 1e-12:
            if svm_objective(f + t * (f_plus - f), a + t * (a_plus - a), y, lam) <= J0:
                break
            t *= 0.5
        a = a + t * (a_plus - a)
        f = f + t * (f_plus - f)
        S_prev, full_prev = S, t == 1.0
    return a, newton_iters, cg_total, False


def hinge_svm_objective(f, a, y, lam):
    """J = (lam / 2) a^T f + (1 / n) sum_i max(0, 1 - y_i f_i) with f = K a: the hinge-loss SVM in
    the coefficients of the representer theorem."""
    return float(0.5 * lam * float(a @ f) + np.mean(np.maximum(0.0, 1.0 - y * f)))


def hinge_svm_subgradient(matvec, y, lam, iters):
    """Hinge-loss SVM by the stochastic-free kernelised sub-gradient method of Pegasos
    (Shalev-Shwartz et al., 2011): with step 1 / (lam t), the sub-gradient step in the RKHS is
        a <- (1 - 1/t) a + (1 / (lam t n)) y * [y f < 1],   f = K a,   t = 1, 2, ...
    Returns (a, f, the objective at the returned a)."""
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    a = np.zeros(n)
    f = np.zeros(n)
    for t in range(1, iters + 1):
        act = (y * f < 1.0).astype(np.float64)
        a = (1.0 - 1.0 / t) * a + (1.0 / (lam * t * n)) * y * act
        f = matvec(a)
    return a, f, hinge_svm_objective(f, a, y, lam)


def minres_solve(matvec, y, lam, tol=1e-6, max_iter=10000, record_every=0):
    """MINRES (Paige and Saunders) for (K + lam I) a = y, the solver of Sec. 6.

    Lanczos vectors v_k of A = K + lam I started from y; the tridiagonal T_k is reduced by
    Givens rotations, so that a_k minimises ||y - A a|| over the Krylov space K_k(A, y).
    Column k of T_k holds beta_k (row k-1), alpha_k (row k) and beta_{k+1} (row k+1); after
    the rotations k-2 and k-1 it becomes (eps_k, delta_k, gammabar_k) and rotation k removes
    beta_{k+1}.  The right-hand side beta_1 e_1 turns into tau_k, and |phibar_k| = ||r_k||.
    Directions d_k = (v_k - delta_k d_{k-1} - eps_k d_{k-2}) / gamma_k, a_k = a_{k-1} + tau_k d_k.
    Stops when |phibar_k| / ||y|| <= tol.  Returns (a, iterations, |phibar|/||y||, records)
    with records[j] = a_k for k = record_every * (j + 1).
    """
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    a = np.zeros(n)
    beta1 = float(np.sqrt(y @ y))
    if beta1 == 0.0:
        return a, 0, 0.0, []
    v_prev, v = np.zeros(n), y / beta1
    beta = 0.0                      # beta_k (T[k-1, k]); zero for k = 1
    c2, s2, c1, s1 = 1.0, 0.0, 1.0, 0.0   # rotations k-2 and k-1
    d2, d1 = np.zeros(n), np.zeros(n)   # d_{k-2}, d_{k-1}
    phibar = beta1
    records = []
    k = 0
    while k < max_iter and abs(phibar) / beta1 > tol:
        k += 1
        w = matvec(v) + lam * v - beta * v_prev
        alpha = float(v @ w)
        w -= alpha * v
        beta_next = float(np.sqrt(w @ w))
        eps = s2 * beta
        dprime = c2 * beta
        delta = c1 * dprime + s1 * alpha
        gbar = -s1 * dprime + c1 * alpha
        gamma = float(np.hypot(gbar, beta_next))
        c, s = gbar / gamma, beta_next / gamma
        tau = c * phibar
        phibar = -s * phibar
        d = (v - delta * d1 - eps * d2) / gamma
        a = a + tau * d
        if record_every > 0 and k % record_every == 0:
            records.append(a.copy())
        d2, d1 = d1, d
        c2, s2, c1, s1 = c1, s1, c, s
        if beta_next == 0.0:
            break
        v_prev, v = v, w / beta_next
        beta = beta_next
    return a, k, abs(phibar) / beta1, records


def relative_residual(matvec, a, y, lam):
    """||y - (K + lam I) a||_2 / ||y||_2 with the oracle's own matvec."""
    r = np.asarray(y, dtype=np.float64) - (matvec(a) + lam * np.asarray(a))
    return float(np.linalg.norm(r) / np.linalg.norm(y))
