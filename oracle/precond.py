"""FP64 CPU oracle of the learned diagonal-plus-low-rank preconditioner.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written out slowly with
numpy so that the CUDA forward / backward kernels can be checked against it;
its own analytic gradient is pinned by central finite differences in
tests/test_precond_oracle.py.

Model (per training pair i, features from the kernel diagonals, the degrees
and the kernel-graph degrees  g1 = K 1,  g2 = K (g1 / mean g1)):
    f_i   = [M[d_i,d_i], N[t_i,t_i], log(1+deg d_i), log(1+deg t_i), slog(g1_i), slog(g2_i)],
    slog(x) = sign(x) log(1 + |x|),
    x_i   = (f_i - mu) / sigma                       (fixed normalisation)
    h1    = relu(W1 x + b1)        (128)
    h2    = relu(W2 h1 + b2)       (128)
    o     = W3 h2 + b3             (33)
    D_i   = c softplus(o_0),  V_i = o_{1..32}     (c: fixed output scale, set from
                                                the training pairs before training)
Training learns V only (the gradient of o_0 is held at zero and the o_0 row
of W3 starts at zero), so D stays c softplus(b3_0) = c and
    P = c (I + V V^T)^{-1} = c I - c V (I + V^T V)^{-1} V^T,
a constant diagonal minus a learned rank-32 term (the structure of a Nystrom
preconditioner, with the subspace predicted per pair by the network).
Preconditioner (SPD for any outputs, Woodbury form of a diagonal matrix
minus a rank-32 term):
    P r = s * (z - V (I + V^T V)^{-1} V^T z),   s = sqrt(D), z = s * r
Training loss on residual -> correction pairs (r_k, e_k = a* - a_k):
    L = (1/K) sum_k ||P r_k - e_k||^2 / ||e_k||^2
"""
import numpy as np

HIDDEN = 128
RANK = 32
NOUT = 1 + RANK
N_FEAT = 6
SHAPES = [("W1", (HIDDEN, N_FEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (NOUT, HIDDEN)), ("b3", (NOUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, off = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[off:off + k], dtype=np.float64).reshape(shp)
        off += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def slog(x):
    return np.sign(x) * np.log1p(np.abs(x))


def pair_features(M, N, d, t, m_cols, q_cols, matvec=None):
    """Raw features: kernel diagonals, log(1 + degree) of the pair's drug and target, and
    the signed logs of the kernel-graph degrees g1 = K 1 and g2 = K (g1 / mean g1), where
    matvec(v) = K v is the pairwise kernel matrix of the training pairs (zeros if None)."""
    deg_d = np.bincount(d, minlength=m_cols).astype(np.float64)
    deg_t = np.bincount(t, minlength=q_cols).astype(np.float64)
    n = len(d)
    if matvec is not None:
        g1 = matvec(np.ones(n))
        g2 = matvec(g1 / np.mean(g1))
    else:
        g1 = g2 = np.zeros(n)
    return np.stack([np.diag(M)[d], np.diag(N)[t], np.log1p(deg_d[d]), np.log1p(deg_t[t]),
                     slog(g1), slog(g2)], axis=1)


def normalisation(F):
    """Per-feature mean and standard deviation (a zero deviation is replaced by 1)."""
    mu = F.mean(axis=0)
    sd = F.std(axis=0)
    sd[sd == 0] = 1.0
    return mu, sd


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def mlp_forward(theta, X):
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (X, z1, h1, z2, h2)


def mlp_backward(theta, cache, g_o):
    p = unpack(theta)
    X, z1, h1, z2, h2 = cache
    g = {"W3": g_o.T @ h2, "b3": g_o.sum(axis=0)}
    g_h2 = g_o @ p["W3"]
    g_z2 = g_h2 * (z2 > 0)
    g["W2"] = g_z2.T @ h1
    g["b2"] = g_z2.sum(axis=0)
    g_h1 = g_z2 @ p["W2"]
    g_z1 = g_h1 * (z1 > 0)
    g["W1"] = g_z1.T @ X
    g["b1"] = g_z1.sum(axis=0)
    return pack(g)


def outputs_to_DV(o, scale=1.0):
    return scale * softplus(o[:, 0]), o[:, 1:]


def data_scale(R, E):
    """Output scale c = sum e.e / sum r.e: the scalar with e ~ c r in the least-squares sense
    weighted towards the corrections (it approaches 1 / lambda, the inverse on the
    small-eigenvalue directions that dominate ||e||)."""
    return float(np.sum(E * E) / np.sum(R * E))


def apply_P(D, V, r):
    """P r with P = S (I + V V^T)^{-1} S, S = diag(sqrt(D)) (Woodbury form)."""
    s = np.sqrt(D)
    z = s * r
    G = np.eye(V.shape[1]) + V.T @ V
    c = np.linalg.solve(G, V.T @ z)
    return s * (z - V @ c)


def P_matrix(D, V):
    """The explicit matrix S (I + V V^T)^{-1} S (small n only)."""
    S = np.diag(np.sqrt(D))
    return S @ np.linalg.inv(np.eye(len(D)) + V @ V.T) @ S


def loss_and_output_grad(o, R, E, scale=1.0, learn_diag=False):
    """L = mean_k ||P r_k - e_k||^2 / ||e_k||^2 and dL/do (n x 33)."""
    D, V = outputs_to_DV(o, scale)
    n, K = R.shape
    s = np.sqrt(D)
    G = np.eye(V.shape[1]) + V.T @ V
    Ginv = np.linalg.inv(G)
    L = 0.0
    g_s = np.zeros(n)
    g_V = np.zeros_like(V)
    for k in range(K):
        r, e = R[:, k], E[:, k]
        ee = float(e @ e)
        z = s * r
        h = V.T @ z
        c = Ginv @ h
        y = z - V @ c
        out = s * y
        rho = out - e
        L += float(rho @ rho) / ee / K
        g_out = 2.0 * rho / ee / K
        g_s += y * g_out
        g_y = s * g_out
        g_z = g_y.copy()
        g_V += -np.outer(g_y, c)
        g_c = -(V.T @ g_y)
        g_h = Ginv @ g_c
        g_G = -np.outer(g_h, c)
        g_V += V @ (g_G + g_G.T)
        g_V += np.outer(z, g_h)
        g_z += V @ g_h
        g_s += r * g_z
    g_D = g_s / (2.0 * s)
    g_o = np.zeros_like(o)
    g_o[:, 0] = g_D * scale * sigmoid(o[:, 0]) if learn_diag else 0.0
    g_o[:, 1:] = g_V
    return L, g_o


def loss_and_grad(theta, X, R, E, scale=1.0, learn_diag=False):
    o, cache = mlp_forward(theta, X)
    L, g_o = loss_and_output_grad(o, R, E, scale, learn_diag)
    return L, mlp_backward(theta, cache, g_o)


def init_params(seed=0, out_scale=0.01):
    """He-style initialisation from a seeded generator; small output layer and
    softplus(b3[0]) = 1, so that the initial P is close to c I."""
    rng = np.random.default_rng(seed)
    b3 = np.zeros(NOUT)
    b3[0] = np.log(np.expm1(1.0))
    W3 = rng.standard_normal((NOUT, HIDDEN)) * out_scale
    W3[0] = 0.0
    p = {"W1": rng.standard_normal((HIDDEN, N_FEAT)) * np.sqrt(2.0 / N_FEAT), "b1": np.zeros(HIDDEN),
         "W2": rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN), "b2": np.zeros(HIDDEN),
         "W3": W3, "b3": b3}
    return pack(p)
