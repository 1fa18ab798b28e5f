"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares the
oracle with an independent derivation (the printed worked example, the
operator identities of Theorem 2, the sum-of-Kronecker forms of Corollary 1,
the feature maps of Table 4a, Roth's column lemma, the ranking incidence
form, PSD-ness, library routines, brute force).  Runs without a GPU.
"""
import numpy as np
import pytest

import oracle as orc
from conftest import read_golden_matrices
from paper_2009_01054_gb300 import synth

KINDS = orc.KINDS
HETERO = ["kronecker", "gaussian", "linear", "poly2d", "cartesian"]
HOMO = ["symmetric", "antisymmetric", "ranking", "mlpk"]


def _rng(seed=0):
    return np.random.default_rng(seed)


def _gauss(rng, n, dim=3, gamma=0.5):
    X = rng.standard_normal((n, dim))
    return orc.gaussian_kernel(X, gamma=gamma), X


def _all_pairs(nD, nT):
    d, t = np.divmod(np.arange(nD * nT), nT)
    return d.astype(np.int32), t.astype(np.int32)


# ---------------------------------------------------------------- Definition 1

def test_worked_example_P_Q_match_printed_matrices():
    g = read_golden_matrices("operators_3x2.txt")
    np.testing.assert_array_equal(orc.commutation_P(3, 2), g["P"])
    np.testing.assert_array_equal(orc.unification_Q(3, 2), g["Q"])


@pytest.mark.parametrize("nD,nT", [(3, 2), (4, 5), (2, 2)])
def test_operator_identities_theorem2(nD, nT):
    rng = _rng(1)
    D, _ = _gauss(rng, nD)
    T, _ = _gauss(rng, nT)
    P = orc.commutation_P(nD, nT)
    I = np.eye(nD * nT)
    np.testing.assert_array_equal(P @ P.T, I)
    np.testing.assert_array_equal(P.T @ P, I)
    np.testing.assert_allclose(P @ np.kron(D, T), np.kron(T, D) @ P, atol=1e-15)
    np.testing.assert_allclose(P @ np.kron(D, T) @ P.T, np.kron(T, D), atol=1e-15)
    # homogeneous P is symmetric and commutes with D kron D
    Ph = orc.commutation_P(nD, nD)
    np.testing.assert_array_equal(Ph, Ph.T)
    np.testing.assert_allclose(Ph @ np.kron(D, D), np.kron(D, D) @ Ph, atol=1e-15)
    np.testing.assert_allclose(Ph @ np.kron(D, D) @ Ph, np.kron(D, D), atol=1e-15)
    # unification: Q (D kron D) Q^T = D^{o2} kron 1  (Q in (D x T) x (D x D))
    Q = orc.unification_Q(nD, nT)
    np.testing.assert_allclose(Q @ np.kron(D, D) @ Q.T, np.kron(D * D, np.ones((nT, nT))),
                               atol=1e-15)
    # and the target-side analogue P Q (T kron T) Q^T P^T = 1 kron T^{o2}
    Qt = orc.unification_Q(nT, nD)          # (T x D) x (T x T)
    Pt = orc.commutation_P(nT, nD)          # (D x T) x (T x D)
    np.testing.assert_allclose(Pt @ Qt @ np.kron(T, T) @ Qt.T @ Pt.T,
                               np.kron(np.ones((nD, nD)), T * T), atol=1e-15)


def test_index_remap_rules():
    """R(d,t)P = R(t,d) and R(d,t)Q = R(d,d) on a homogeneous domain (Sec. 4.9 proof)."""
    rng = _rng(2)
    nD = 5
    d, t = synth.random_pairs(rng, 17, nD, nD)
    R = orc.sampling_R(d, t, nD, nD)
    P = orc.commutation_P(nD, nD)
    Q = orc.unification_Q(nD, nD)
    np.testing.assert_array_equal(R @ P, orc.sampling_R(t, d, nD, nD))
    np.testing.assert_array_equal(R @ Q, orc.sampling_R(d, d, nD, nD))
    # heterogeneous: R(d,t) P^T selects (t, d) in T x D
    nT = 3
    d2, t2 = synth.random_pairs(rng, 11, nD, nT)
    R2 = orc.sampling_R(d2, t2, nD, nT)
    np.testing.assert_array_equal(R2 @ orc.commutation_P(nD, nT).T,
                                  orc.sampling_R(t2, d2, nT, nD))


# ------------------------------------------- Table 4b versus Corollary 1 forms

def _corollary_operator(kind, D, T):
    """K_op of Corollary 1, built from explicit operators (readings in the oracle header)."""
    nD, nT = D.shape[0], T.shape[0]
    if kind in ("kronecker", "gaussian"):
        return np.kron(D, T)
    if kind == "linear":
        return np.kron(D, np.ones((nT, nT))) + np.kron(np.ones((nD, nD)), T)
    if kind == "poly2d":
        Q = orc.unification_Q(nD, nT)
        Qt = orc.unification_Q(nT, nD)
        Pt = orc.commutation_P(nT, nD)
        return (Q @ np.kron(D, D) @ Q.T + 2 * np.kron(D, T)
                + Pt @ Qt @ np.kron(T, T) @ Qt.T @ Pt.T)
    if kind == "cartesian":
        return np.kron(D, np.eye(nT)) + np.kron(np.eye(nD), T)
    P = orc.commutation_P(nD, nD)
    I = np.eye(nD * nD)
    DD = np.kron(D, D)
    if kind == "symmetric":
        return (P + I) @ DD
    if kind == "antisymmetric":
        return (I - P) @ DD            # Table 4b sign; Corollary 1 prints (P - I)
    if kind == "ranking":
        return (I - P) @ np.kron(D, np.ones((nD, nD))) @ (I - P)
    if kind == "mlpk":
        Q = orc.unification_Q(nD, nD)
        return (I + P) @ (I - Q) @ DD @ (I - Q).T @ (I + P)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", KINDS)
def test_table4b_equals_corollary_sum_of_kroneckers(kind):
    rng = _rng(3)
    nD = 4
    nT = 4 if kind in HOMO else 3
    D, _ = _gauss(rng, nD)
    T, _ = _gauss(rng, nT)
    d_in, t_in = synth.random_pairs(rng, 9, nD, nT)
    d_out, t_out = synth.random_pairs(rng, 7, nD, nT)
    K = orc.kernel_matrix(kind, D, T, d_out, t_out, d_in, t_in)
    Kop = _corollary_operator(kind, D, T if kind not in HOMO else D)
    Rb = orc.sampling_R(d_out, t_out, nD, nT)
    R = orc.sampling_R(d_in, t_in, nD, nT)
    np.testing.assert_allclose(K, Rb @ Kop @ R.T, rtol=1e-13, atol=1e-14)


def test_mlpk_has_ten_kronecker_terms():
    """The 10-term expansion of the MLPK operator (proof of Corollary 1) equals the factored form."""
    rng = _rng(4)
    nD = 3
    D, _ = _gauss(rng, nD)
    P = orc.commutation_P(nD, nD)
    Q = orc.unification_Q(nD, nD)
    DD = np.kron(D, D)
    terms = [Q @ DD @ Q.T, P @ Q @ DD @ Q.T, Q @ DD @ Q.T @ P, P @ Q @ DD @ Q.T @ P,
             2 * DD, 2 * P @ DD, -2 * Q @ DD, -2 * P @ Q @ DD, -2 * DD @ Q.T,
             -2 * DD @ Q.T @ P]
    assert len(terms) == 10
    np.testing.assert_allclose(sum(terms), _corollary_operator("mlpk", D, D), atol=1e-14)


def test_antisymmetric_sign_reading_is_the_psd_one():
    """Table 4b's (I - P)(D kron D) is PSD; the Corollary's printed (P - I) is not."""
    rng = _rng(5)
    D, _ = _gauss(rng, 4)
    P = orc.commutation_P(4, 4)
    DD = np.kron(D, D)
    ev_tab = np.linalg.eigvalsh(((np.eye(16) - P) @ DD + ((np.eye(16) - P) @ DD).T) / 2)
    ev_cor = np.linalg.eigvalsh(((P - np.eye(16)) @ DD + ((P - np.eye(16)) @ DD).T) / 2)
    assert ev_tab.min() > -1e-12 and ev_tab.max() > 1e-3
    assert ev_cor.min() < -1e-3


# ------------------------------------------------------------ Table 4a features

def _feature_map(kind, xd, xt, nD, nT, d, t):
    if kind == "linear":
        return np.concatenate([xd, xt])
    if kind == "poly2d":
        z = np.concatenate([xd, xt])
        return np.kron(z, z)
    if kind == "kronecker":
        return np.kron(xd, xt)
    if kind == "cartesian":
        return np.concatenate([np.kron(xd, np.eye(nT)[t]), np.kron(np.eye(nD)[d], xt)])
    if kind == "symmetric":
        return np.sqrt(0.5) * (np.kron(xd, xt) + np.kron(xt, xd))
    if kind == "antisymmetric":
        return np.sqrt(0.5) * (np.kron(xd, xt) - np.kron(xt, xd))
    if kind == "ranking":
        return xd - xt
    if kind == "mlpk":
        return np.kron(xd - xt, xd - xt)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", [k for k in KINDS if k != "gaussian"])
def test_feature_map_gram_table4a(kind):
    """With linear base kernels D = X X^T the pairwise kernel is the Gram of the Table 4a map."""
    rng = _rng(6)
    nD, nT, r = 5, (5 if kind in HOMO else 4), 3
    Xd = rng.standard_normal((nD, r))
    Xt = Xd if kind in HOMO else rng.standard_normal((nT, r + 1))
    D, T = Xd @ Xd.T, Xt @ Xt.T
    d, t = synth.random_pairs(rng, 12, nD, nT)
    Phi = np.array([_feature_map(kind, Xd[a], Xt[b], nD, nT, a, b) for a, b in zip(d, t)])
    K = orc.kernel_matrix(kind, D, T, d, t, d, t)
    np.testing.assert_allclose(K, Phi @ Phi.T, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- other closed forms

def test_roth_column_lemma_on_complete_data():
    """All m*q pairs present: (M kron N) vec(X) = vec(N X M^T) (Sec. 3, vec trick)."""
    rng = _rng(7)
    m, q = 6, 5
    M, _ = _gauss(rng, m)
    N, _ = _gauss(rng, q)
    d, t = _all_pairs(m, q)
    v = rng.standard_normal(m * q)
    u = orc.pairwise_matvec("kronecker", M, N, d, t, d, t, v)
    X = v.reshape(m, q).T                      # X[t, d] = v[d*q + t]
    np.testing.assert_allclose(u, (N @ X @ M.T).T.reshape(-1), rtol=1e-13, atol=1e-13)


def test_ranking_incidence_form():
    """Ranking kernel = M_inc^T D M_inc with the oriented incidence operator (Sec. 4.5)."""
    rng = _rng(8)
    nD, n = 6, 14
    D, _ = _gauss(rng, nD)
    cells = rng.choice(nD * (nD - 1), n, replace=False)
    a, r = np.divmod(cells, nD - 1)
    b = r + (r >= a)
    Minc = np.zeros((nD, n))
    Minc[a, np.arange(n)] = 1.0
    Minc[b, np.arange(n)] = -1.0
    K = orc.kernel_matrix("ranking", D, None, a, b, a, b)
    np.testing.assert_allclose(K, Minc.T @ D @ Minc, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("kind", ["symmetric", "antisymmetric", "ranking", "mlpk"])
def test_swap_symmetry(kind):
    """Symmetric / MLPK rows are invariant under swapping the output pair; anti-symmetric and
    ranking rows change sign (Sec. 4.4, 4.5)."""
    rng = _rng(9)
    m = 7
    M, _ = _gauss(rng, m)
    d, t = synth.random_pairs(rng, 30, m, m)
    do, to = synth.random_pairs(rng, 10, m, m)
    v = rng.standard_normal(30)
    u = orc.pairwise_matvec(kind, M, None, do, to, d, t, v)
    us = orc.pairwise_matvec(kind, M, None, to, do, d, t, v)
    sign = -1.0 if kind in ("antisymmetric", "ranking") else 1.0
    np.testing.assert_allclose(us, sign * u, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_kernel_matrix_is_psd(kind):
    rng = _rng(10)
    m = 6
    q = m if kind in HOMO else 5
    M, _ = _gauss(rng, m)
    N, _ = _gauss(rng, q)
    d, t = synth.random_pairs(rng, 25, m, q)
    K = orc.kernel_matrix(kind, M, N, d, t, d, t)
    np.testing.assert_allclose(K, K.T, atol=1e-14)
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-12 * np.abs(ev).max()


def test_gaussian_base_kernel_matches_library_distance():
    from scipy.spatial.distance import cdist
    rng = _rng(11)
    X = rng.standard_normal((13, 7))
    Y = rng.standard_normal((9, 7))
    K = orc.gaussian_kernel(X, Y, gamma=0.3)
    np.testing.assert_allclose(K, np.exp(-0.3 * cdist(X, Y, "sqeuclidean")), rtol=1e-13)


def test_gaussian_pairwise_factorises_on_concatenated_features():
    """exp(-g||(xd,xt)-(xd',xt')||^2) = k_D * k_T (Sec. 4.3, squared-norm reading)."""
    rng = _rng(12)
    Xd = rng.standard_normal((5, 3))
    Xt = rng.standard_normal((4, 2))
    g = 0.4
    M = orc.gaussian_kernel(Xd, gamma=g)
    N = orc.gaussian_kernel(Xt, gamma=g)
    d, t = synth.random_pairs(rng, 10, 5, 4)
    Z = np.concatenate([Xd[d], Xt[t]], axis=1)
    np.testing.assert_allclose(orc.kernel_matrix("gaussian", M, N, d, t, d, t),
                               orc.gaussian_kernel(Z, gamma=g), rtol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_matvec_equals_explicit_matrix_product(kind):
    rng = _rng(13)
    m = 9
    q = m if kind in HOMO else 7
    M, _ = _gauss(rng, m)
    N, _ = _gauss(rng, q)
    d, t = synth.random_pairs(rng, 40, m, q)
    do, to = synth.random_pairs(rng, 23, m, q)
    V = rng.standard_normal((40, 3))
    K = orc.kernel_matrix(kind, M, N, do, to, d, t)
    np.testing.assert_allclose(orc.pairwise_matvec(kind, M, N, do, to, d, t, V), K @ V,
                               rtol=1e-12, atol=1e-12)


def test_compensated_sum_recovers_cancelled_term():
    x = np.array([1e16, 1.0, -1e16, 3.0, 0.5])
    assert orc.compensated_sum(x) == 4.5
    naive = 0.0
    for xi in x.tolist():
        naive = naive + xi
    assert naive != 4.5


def test_krr_dense_matches_complete_data_closed_form():
    rng = _rng(14)
    m, q, lam = 5, 4, 0.05
    M, _ = _gauss(rng, m)
    N, _ = _gauss(rng, q)
    d, t = _all_pairs(m, q)
    y = rng.standard_normal(m * q)
    K = orc.kernel_matrix("kronecker", M, N, d, t, d, t)
    a = orc.krr_solve_dense(K, y, lam)
    A = orc.krr_complete_closed_form(M, N, y.reshape(m, q).T, lam)
    np.testing.assert_allclose(a, A.T.reshape(-1), rtol=1e-10, atol=1e-12)


def test_cg_matches_cholesky():
    p = synth.small(0)
    M = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    N = orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    lam = p.lambdas[0]
    K = orc.kernel_matrix("kronecker", M, N, p.d, p.t, p.d, p.t)
    a_ref = orc.krr_solve_dense(K, p.y, lam)
    a, it, rr = orc.cg_solve(lambda x: K @ x, p.y, lam, tol=1e-10)
    assert rr <= 1e-10 and it > 0
    np.testing.assert_allclose(a, a_ref, rtol=1e-7, atol=1e-8)
    mv = lambda x: orc.pairwise_matvec("kronecker", M, N, p.d, p.t, p.d, p.t, x)
    assert orc.relative_residual(mv, a_ref, p.y, lam) < 1e-10


def test_synthetic_shapes_keep_table5_densities():
    rows = [l.split() for l in open(__import__("os").path.join(
        __import__("conftest").ROOT, "tests", "golden", "table5_datasets.txt"))
        if l.strip() and not l.startswith("#")]
    dens = {r[0]: int(r[1]) / (int(r[2]) * int(r[3])) for r in rows}
    assert abs(dens["merget"] - 0.25) < 0.01 and abs(dens["heterodimer"] - 0.0024) < 1e-4
    assert abs(synth.homogeneous(0, m=200, n=2000).n / (200 * 200) - 0.05) < 1e-9
    small = synth.small(0)
    assert len(set(zip(small.d, small.t)) & set(zip(small.d_pred, small.t_pred))) == 0


def test_tanimoto_kernel_is_the_jaccard_index_and_psd():
    """Tanimoto (MinMax) kernel of Sec. 5 on binary vectors: equal to |A & B| / |A | B| of the
    index sets (brute force with Python sets), 1 on the diagonal and for two empty vectors,
    0 for disjoint vectors, symmetric and positive semidefinite."""
    rng = np.random.default_rng(31)
    bits, _ = synth.fingerprints(rng, 25, 70, 0.2)
    bits[3] = 0
    bits[7] = 0                                   # two empty fingerprints
    K = orc.tanimoto_kernel(bits)
    sets = [set(np.flatnonzero(b)) for b in bits]
    for a in range(25):
        for b in range(25):
            u = len(sets[a] | sets[b])
            want = len(sets[a] & sets[b]) / u if u else 1.0
            assert abs(K[a, b] - want) <= 1e-15
    assert np.all(np.diag(K) == 1.0) and K[3, 7] == 1.0 and K[3, 0] == 0.0
    x = np.zeros((2, 8), np.uint8)
    x[0, :4] = 1
    x[1, 4:] = 1
    assert orc.tanimoto_kernel(x)[0, 1] == 0.0
    np.testing.assert_array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() >= -1e-12 * np.abs(K).max()


def test_linear_kernel_on_similarity_rows():
    """Linear base kernel of Sec. 5 (Metz: rows of a similarity matrix as features):
    * entry by entry, a brute-force sum of products;
    * on the rows of a symmetric similarity matrix S it is the matrix square S S;
    * it ties to the Gaussian kernel through ||x - y||^2 = k(x, x) + k(y, y) - 2 k(x, y);
    * the cross kernel of new rows against training rows is the matching block of the kernel of
      the stacked rows;
    * it is symmetric and positive semidefinite."""
    rng = np.random.default_rng(33)
    X = rng.standard_normal((9, 5))
    K = orc.linear_kernel(X)
    for a in range(9):
        for b in range(9):
            want = sum(float(X[a, i]) * float(X[b, i]) for i in range(5))
            assert abs(K[a, b] - want) <= 1e-14 * max(1.0, abs(want))
    A = rng.uniform(0.0, 1.0, (12, 12))
    S = (A + A.T) / 2
    np.fill_diagonal(S, 1.0)
    np.testing.assert_allclose(orc.linear_kernel(S), np.linalg.matrix_power(S, 2), rtol=1e-13, atol=1e-13)
    Y = rng.standard_normal((4, 5))
    d2 = np.diag(K)[:, None] + np.sum(Y * Y, axis=1)[None, :] - 2 * orc.linear_kernel(X, Y)
    np.testing.assert_allclose(np.exp(-0.3 * d2), orc.gaussian_kernel(X, Y, gamma=0.3), rtol=1e-12, atol=1e-14)
    Kall = orc.linear_kernel(np.vstack([X, Y]))
    np.testing.assert_allclose(orc.linear_kernel(Y, X), Kall[9:, :9], rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() >= -1e-12 * np.abs(K).max()


def test_auc_is_the_pairwise_ranking_probability():
    """AUC (the paper's measure): equal to the brute-force fraction of correctly ordered
    (positive, negative) pairs with ties counting 1/2; 1 for a perfect ranking, 0 for the
    reversed one, 1/2 when every score ties; unchanged by a strictly increasing transform."""
    rng = np.random.default_rng(34)
    s = np.round(rng.standard_normal(60), 1)          # rounding creates ties
    y = rng.random(60) < 0.3
    pos, neg = s[y], s[~y]
    want = sum((p > q) + 0.5 * (p == q) for p in pos for q in neg) / (len(pos) * len(neg))
    assert abs(orc.auc(s, y) - want) <= 1e-15
    lab = np.array([0, 0, 1, 1, 0, 1])
    sc = np.array([0.1, 0.2, 0.8, 0.9, 0.3, 0.7])
    assert orc.auc(sc, lab) == 1.0 and orc.auc(-sc, lab) == 0.0
    assert orc.auc(np.zeros(6), lab) == 0.5
    assert abs(orc.auc(np.exp(3 * s) + 2, y) - orc.auc(s, y)) <= 1e-15


def test_fingerprint_packing_round_trip():
    rng = np.random.default_rng(32)
    bits, packed = synth.fingerprints(rng, 9, 77, 0.4)
    assert packed.dtype == np.uint32 and packed.shape == (9, 3)
    unpacked = ((packed[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(9, 96)[:, :77]
    np.testing.assert_array_equal(unpacked, bits)
    assert np.all((packed[:, 2] >> np.uint32(13)) == 0)   # bits past the length are zero


def test_kernel_value_is_the_kernel_matrix_entry():
    """The oracle's single-entry call k((a, b), (c, e)) equals the matching entry of its explicit
    pairwise kernel matrix for all nine kernels (argument order: output pair, then input pair)."""
    rng = np.random.default_rng(35)
    m, q = 7, 5
    A = rng.standard_normal((m, 3))
    B = rng.standard_normal((q, 3))
    M = orc.gaussian_kernel(A, gamma=0.4)
    N = orc.gaussian_kernel(B, gamma=0.7)
    for kind in ["kronecker", "gaussian", "linear", "poly2d", "cartesian", "symmetric", "antisymmetric",
                 "ranking", "mlpk"]:
        homo = kind in ("symmetric", "antisymmetric", "ranking", "mlpk")
        qq = m if homo else q
        d_out, t_out = synth.random_pairs(rng, 6, m, qq)
        d_in, t_in = synth.random_pairs(rng, 5, m, qq)
        Nk = M if homo else N
        K = orc.kernel_matrix(kind, M, Nk, d_out, t_out, d_in, t_in)
        for i in range(6):
            for j in range(5):
                val = orc.kernel_value(kind, M, Nk, d_out[i], t_out[i], d_in[j], t_in[j])
                assert val == K[i, j], (kind, i, j)
