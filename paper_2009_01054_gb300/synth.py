"""Seeded synthetic inputs shaped like the paper's drug-target workloads.

This module holds no arithmetic of the method: it draws features, pair index
sequences, right-hand sides and labels with NumPy's ``default_rng``.  Both the
CUDA path and the oracle build their kernel matrices from these features
themselves.  The paper's data sets (Table 5) are not available, so these
stand in for them:

  small       m=64 drugs, q=48 targets, 16-d features, gamma=1/16; the 3072 grid
              cells are permuted, the first 1000 are training pairs and the
              next 500 (disjoint) are prediction pairs; v, y ~ N(0,1); lambda=1e-2.
  homogeneous m=q=2000 objects, 64-d, gamma=1/64; 200k ordered pairs (d, d'),
              d != d', uniform without replacement (5 % of the off-diagonal
              cells, the shape of the heterodimer / kernel-filling sets).
  merget      m=2000, q=250, 128-d, gamma=1/128; 120k pairs uniform without
              replacement (24 %, the shape of the Merget set);
              y = x_d^T B x_t / sqrt(128*128) + N(0, 0.1^2), B ~ N(0,1).
  batched     256 problems, problem b drawn with seed+b: m, q ~ U{32..512},
              density ~ U[0.05, 0.6], 32-d, gamma=1/32, labels as merget,
              16 lambdas logspace(-4, 0).
  zipf        m=q=20000, 256-d, gamma=1/256, 10M unique pairs with power-law
              degrees: Zipf(1.1) weights on drug and target ids (through a random
              permutation of the ids) and cell (d, t) drawn with probability
              min(1, c w_d w_t) (kernel-filling scale).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class PairProblem:
    name: str
    m: int                      # drugs (rows/cols of M)
    q: int                      # targets (rows/cols of N)
    Xd: np.ndarray              # m x dim drug features
    Xt: np.ndarray              # q x dim target features (same array as Xd when homogeneous)
    gamma: float
    d: np.ndarray               # training pair drug ids (int32)
    t: np.ndarray               # training pair target ids (int32)
    v: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None
    d_pred: Optional[np.ndarray] = None
    t_pred: Optional[np.ndarray] = None
    lambdas: List[float] = field(default_factory=list)
    homogeneous: bool = False

    @property
    def n(self):
        return int(len(self.d))


def _uniform_cells(rng, n_cells, n):
    return rng.choice(n_cells, size=n, replace=False)


def small(seed=0):
    """m=64, q=48, 16-d features, 1000 training + 500 disjoint prediction pairs."""
    rng = np.random.default_rng(seed)
    m, q, dim = 64, 48, 16
    Xd = rng.standard_normal((m, dim))
    Xt = rng.standard_normal((q, dim))
    cells = rng.permutation(m * q)
    tr, pr = cells[:1000], cells[1000:1500]
    v = rng.standard_normal(1000)
    y = rng.standard_normal(1000)
    return PairProblem("small", m, q, Xd, Xt, 1.0 / dim,
                       (tr // q).astype(np.int32), (tr % q).astype(np.int32),
                       v=v, y=y, d_pred=(pr // q).astype(np.int32),
                       t_pred=(pr % q).astype(np.int32), lambdas=[1e-2])


def homogeneous(seed=0, m=2000, dim=64, n=200_000):
    """m=q objects, ordered off-diagonal pairs (d, d'), d != d', uniform w/o replacement."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, dim))
    cells = _uniform_cells(rng, m * (m - 1), n)
    d = cells // (m - 1)
    r = cells % (m - 1)
    t = r + (r >= d)
    v = rng.standard_normal(n)
    y = rng.standard_normal(n)
    return PairProblem("homogeneous", m, m, X, X, 1.0 / dim,
                       d.astype(np.int32), t.astype(np.int32), v=v, y=y,
                       lambdas=[1e-2], homogeneous=True)


def _bilinear_labels(rng, Xd, Xt, d, t, noise=0.1, chunk=1 << 18):
    """y = x_d^T B x_t / sqrt(dim_d dim_t) + noise, B ~ N(0, 1): the drug projections x_d^T B
    once, then the pair products in chunks (10M pairs never materialise their features)."""
    B = rng.standard_normal((Xd.shape[1], Xt.shape[1]))
    P = Xd @ B
    sig = np.empty(len(d))
    for k in range(0, len(d), chunk):
        sig[k:k + chunk] = np.einsum("ij,ij->i", P[d[k:k + chunk]], Xt[t[k:k + chunk]])
    sig /= np.sqrt(Xd.shape[1] * Xt.shape[1])
    return sig + noise * rng.standard_normal(len(d))


def merget(seed=0, m=2000, q=250, dim=128, n=120_000):
    """Heterogeneous drug-target problem shaped like the Merget set (24 % dense)."""
    rng = np.random.default_rng(seed)
    Xd = rng.standard_normal((m, dim))
    Xt = rng.standard_normal((q, dim))
    cells = _uniform_cells(rng, m * q, n)
    d = (cells // q).astype(np.int32)
    t = (cells % q).astype(np.int32)
    y = _bilinear_labels(rng, Xd, Xt, d, t)
    v = rng.standard_normal(n)
    return PairProblem("merget", m, q, Xd, Xt, 1.0 / dim, d, t, v=v, y=y,
                       lambdas=[1e-4, 1e-2, 1.0])


def batched_problem(b, seed=0, dim=32):
    """Problem b of the batched set: m, q ~ U{32..512}, density ~ U[0.05, 0.6]."""
    rng = np.random.default_rng(seed + b)
    m = int(rng.integers(32, 513))
    q = int(rng.integers(32, 513))
    rho = float(rng.uniform(0.05, 0.6))
    n = max(1, int(round(rho * m * q)))
    Xd = rng.standard_normal((m, dim))
    Xt = rng.standard_normal((q, dim))
    cells = _uniform_cells(rng, m * q, n)
    d = (cells // q).astype(np.int32)
    t = (cells % q).astype(np.int32)
    y = _bilinear_labels(rng, Xd, Xt, d, t)
    return PairProblem("batched%d" % b, m, q, Xd, Xt, 1.0 / dim, d, t, y=y,
                       lambdas=list(np.logspace(-4, 0, 16)))


def batched(n_problems=256, seed=0):
    return [batched_problem(b, seed) for b in range(n_problems)]


def _zipf_weights(n_ids, s, perm):
    """Weight rank^-s of every id, ranks assigned through the permutation `perm`."""
    w = np.empty(n_ids)
    w[perm] = np.arange(1, n_ids + 1, dtype=np.float64) ** (-s)
    return w


def _expected_degree_scale(wd, wt, n):
    """c such that sum_{d,t} min(1, c wd wt) = n (bisection; per drug the cells with
    c wd wt >= 1 are counted from the sorted target weights)."""
    ws = np.sort(wt)[::-1]
    pref = np.concatenate([[0.0], np.cumsum(ws)])
    neg = -ws

    def total(c):
        k = np.searchsorted(neg, -1.0 / (c * wd), side="right")   # targets with c wd wt >= 1
        return float(np.sum(k + c * wd * (pref[-1] - pref[k])))

    lo, hi = 0.0, 1.0
    while total(hi) < n:
        hi *= 2.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if total(mid) < n:
            lo = mid
        else:
            hi = mid
    return hi


def zipf(seed=0, m=20000, dim=256, n=10_000_000, s=1.1, labels=False, rows_per_chunk=500):
    """Heterogeneous m x m problem (kernel-filling scale) with power-law degrees.

    Drug and target ids get Zipf(s) weights w (rank^-s over a random permutation of
    the ids).  Cell (d, t) is a pair with probability min(1, c w_d w_t) (an
    expected-degree model: degrees follow the power law, capped at the id range),
    c set so that a little more than n pairs are expected; n of the drawn pairs are
    then kept at random, in drug-major order.  Labels (the bilinear signal) only
    when `labels`, since they cost a pass over all pairs.
    """
    rng = np.random.default_rng(seed)
    Xd = rng.standard_normal((m, dim))
    Xt = rng.standard_normal((m, dim))
    wd = _zipf_weights(m, s, rng.permutation(m))
    wt = _zipf_weights(m, s, rng.permutation(m))
    c = _expected_degree_scale(wd, wt, n + 6.0 * np.sqrt(n))
    ds, ts = [], []
    for d0 in range(0, m, rows_per_chunk):
        P = np.minimum(1.0, c * wd[d0:d0 + rows_per_chunk, None] * wt[None, :])
        dd, tt = np.nonzero(rng.random(P.shape) < P)
        ds.append((dd + d0).astype(np.int32))
        ts.append(tt.astype(np.int32))
    d = np.concatenate(ds)
    t = np.concatenate(ts)
    if len(d) < n:
        raise RuntimeError("zipf: drew %d pairs, fewer than %d" % (len(d), n))
    keep = np.sort(rng.choice(len(d), n, replace=False))
    d, t = d[keep], t[keep]
    y = _bilinear_labels(rng, Xd, Xt, d, t) if labels else None
    v = rng.standard_normal(n)
    return PairProblem("zipf", m, m, Xd, Xt, 1.0 / dim, d, t, v=v, y=y, lambdas=[1e-2, 1e-4])


@dataclass
class SettingSplit:
    """Training and test pairs of one prediction setting (Sec. 2): the test pairs index the
    rows of the cross kernels K(X_test_objects, X_train_objects)."""
    setting: int
    Xd_train: np.ndarray        # drugs the model is trained on
    Xt_train: np.ndarray
    Xd_test: np.ndarray         # drugs the test pairs refer to (the training drugs in settings 1, 3)
    Xt_test: np.ndarray
    d: np.ndarray               # training pairs, ids into Xd_train / Xt_train
    t: np.ndarray
    y: np.ndarray
    d_test: np.ndarray          # test pairs, ids into Xd_test / Xt_test
    t_test: np.ndarray


def setting_split(p, setting, test_frac=0.25, seed=0):
    """Split the pairs of problem `p` for prediction setting 1-4 (Sec. 2):
    1 random pairs held out (both objects seen in training); 2 pairs of held-out drugs (new
    drugs, known targets); 3 pairs of held-out targets; 4 pairs whose drug and target are both
    held out (training keeps only pairs with neither).  Held-out objects are a `test_frac`
    share of the ids, drawn at random; ids are renumbered densely on both sides."""
    rng = np.random.default_rng(seed)
    y = p.y if p.y is not None else rng.standard_normal(p.n)
    if setting == 1:
        test = rng.random(p.n) < test_frac
        return SettingSplit(1, p.Xd, p.Xt, p.Xd, p.Xt, p.d[~test], p.t[~test], y[~test],
                            p.d[test], p.t[test])
    new_d = rng.random(p.m) < test_frac if setting in (2, 4) else np.zeros(p.m, bool)
    new_t = rng.random(p.q) < test_frac if setting in (3, 4) else np.zeros(p.q, bool)
    nd, nt = new_d[p.d], new_t[p.t]
    train = ~nd & ~nt
    test = (nd | nt) if setting != 4 else (nd & nt)

    def renumber(mask):
        ids = np.full(len(mask), -1, np.int64)
        ids[mask] = np.arange(int(mask.sum()))
        return ids

    keep_d, keep_t = ~new_d, ~new_t
    tr_d, tr_t = renumber(keep_d), renumber(keep_t)
    te_dmask = new_d if setting in (2, 4) else keep_d
    te_tmask = new_t if setting in (3, 4) else keep_t
    te_d, te_t = renumber(te_dmask), renumber(te_tmask)
    return SettingSplit(setting, p.Xd[keep_d], p.Xt[keep_t], p.Xd[te_dmask], p.Xt[te_tmask],
                        tr_d[p.d[train]].astype(np.int32), tr_t[p.t[train]].astype(np.int32), y[train],
                        te_d[p.d[test]].astype(np.int32), te_t[p.t[test]].astype(np.int32))


def fingerprints(rng, rows, length, density):
    """Random binary fingerprints: (bits as a rows x length 0/1 uint8 array, the same bit-packed
    into rows x ceil(length / 32) uint32 words, bit j of word w = feature 32 w + j)."""
    bits = (rng.random((rows, length)) < density).astype(np.uint8)
    words = (length + 31) // 32
    padded = np.zeros((rows, words * 32), np.uint8)
    padded[:, :length] = bits
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    packed = (padded.reshape(rows, words, 32).astype(np.uint64) * weights).sum(axis=2).astype(np.uint32)
    return bits, packed


def random_pairs(rng, n, m_ids, q_ids):
    """n pairs drawn with replacement (duplicates allowed), for edge-case tests."""
    return (rng.integers(0, m_ids, n).astype(np.int32),
            rng.integers(0, q_ids, n).astype(np.int32))


def mlp_init_params(seed=0, out_scale=0.01, n_feat=6, hidden=128, rank=32):
    """Seeded initial parameters of the preconditioner network (layout W1[128x6] b1 W2[128x128] b2
    W3[33x128] b3, float32): He-style normal draws for W1 and W2, a small output layer whose first
    row is zero, zero biases except b3[0] = log(e - 1), so that softplus(o_0) starts at 1."""
    rng = np.random.default_rng(seed)
    n_out = 1 + rank
    W1 = rng.standard_normal((hidden, n_feat)) * np.sqrt(2.0 / n_feat)
    W2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    W3 = rng.standard_normal((n_out, hidden)) * out_scale
    W3[0] = 0.0
    b3 = np.zeros(n_out)
    b3[0] = np.log(np.expm1(1.0))
    parts = [W1, np.zeros(hidden), W2, np.zeros(hidden), W3, b3]
    return np.concatenate([x.reshape(-1) for x in parts]).astype(np.float32)

