"""Batched KRR (many uneven problems x several lambdas in one persistent launch, CUDA graph)
against the oracle: every (problem, lambda) solution is compared with a dense Cholesky solve
of (K + lambda I) a = y, and the FP64 residual the library reports is recomputed by the oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_2009_01054_gb300 import gvt, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def H():
    from paper_2009_01054_gb300 import build
    build.build()
    h = gvt.Handle()
    yield h
    h.close()


def small_batch(n_probs=7, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_probs):
        m, q = int(rng.integers(9, 60)), int(rng.integers(5, 45))
        rho = float(rng.uniform(0.1, 0.6))
        n = max(1, int(round(rho * m * q)))
        Xd, Xt = rng.standard_normal((m, 6)), rng.standard_normal((q, 6))
        cells = rng.choice(m * q, n, replace=False)
        d, t = (cells // q).astype(np.int32), (cells % q).astype(np.int32)
        y = rng.standard_normal(n)
        out.append(dict(Xd=Xd, Xt=Xt, d=d, t=t, y=y, g=1.0 / 6))
    return out


ENGINES = [gvt.GVT_STAGE1_SIMT, gvt.GVT_STAGES_TC_F16X3, gvt.GVT_STAGES_AUTO]


def with_engine(H, engine, fn):
    gvt.gvt_set_stage1_engine(H.h, engine)
    try:
        return fn()
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)


def device_problem(H, p):
    M = gvt.gaussian_kernel(H, torch.as_tensor(p["Xd"], device=DEV), gamma=p["g"])
    N = gvt.gaussian_kernel(H, torch.as_tensor(p["Xt"], device=DEV), gamma=p["g"])
    out = dict(M=M, N=N, d=torch.as_tensor(p["d"], device=DEV), t=torch.as_tensor(p["t"], device=DEV))
    if "y" in p:
        out["y"] = torch.as_tensor(p["y"], device=DEV)
    return out


@pytest.mark.parametrize("engine", [gvt.GVT_STAGE1_SIMT, gvt.GVT_STAGES_TC_F16X3])
@pytest.mark.parametrize("lambdas", [[1e-3, 1e-2, 1e-1, 1.0], list(np.logspace(-3, 0, 16)), [0.5]])
def test_batched_solve_matches_cholesky(H, lambdas, engine):
    batch = small_batch()
    probs = [device_problem(H, p) for p in batch]
    A, st, info, rr = with_engine(H, engine, lambda: gvt.krr_solve_batched(H, probs, lambdas, rel_tol=1e-8))
    assert st == 0, (st, info.iterations, info.refinements, info.rel_residual)
    for b, p in enumerate(batch):
        Mo, No = orc.gaussian_kernel(p["Xd"], gamma=p["g"]), orc.gaussian_kernel(p["Xt"], gamma=p["g"])
        K = orc.kernel_matrix("kronecker", Mo, No, p["d"], p["t"], p["d"], p["t"])
        a = A[b].cpu().numpy()
        for c, lam in enumerate(lambdas):
            ref = orc.krr_solve_dense(K, p["y"], lam)
            res = np.linalg.norm(p["y"] - (K @ a[:, c] + lam * a[:, c])) / np.linalg.norm(p["y"])
            assert res <= 1.05e-8, (b, c, res)
            assert abs(rr[b][c] - res) <= 1e-9 + 0.05 * res
            assert np.max(np.abs(a[:, c] - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref))) / lam, (b, c)


def test_batched_rejects_bad_input(H):
    M = torch.eye(4, dtype=torch.float64, device=DEV)
    d = torch.tensor([0, 5], dtype=torch.int32, device=DEV)
    probs = [dict(M=M, N=M, d=d, t=torch.tensor([0, 1], dtype=torch.int32, device=DEV),
                  y=torch.ones(2, dtype=torch.float64, device=DEV))]
    with pytest.raises(gvt.GvtError) as e:
        gvt.krr_solve_batched(H, probs, [0.1])
    assert e.value.status == 2
    with pytest.raises(gvt.GvtError) as e:
        gvt.krr_solve_batched(H, probs, [0.1] * 17)
    assert e.value.status == 1


def product_batch(seed=5):
    """Problems of the batched product whose GEMM tiles (128 rows by 256 columns, K in 64-blocks)
    all have ragged edges, one without pairs and one with repeated pairs."""
    rng = np.random.default_rng(seed)
    shapes = [(70, 150, 0.10), (200, 40, 0.3), (33, 300, 0.05), (129, 257, 0.02), (12, 9, 0.0), (64, 64, 0.5)]
    out = []
    for i, (m, q, rho) in enumerate(shapes):
        n = int(round(rho * m * q))
        Xd, Xt = rng.standard_normal((m, 6)), rng.standard_normal((q, 6))
        cells = rng.choice(m * q, n, replace=False)
        d, t = (cells // q).astype(np.int32), (cells % q).astype(np.int32)
        if i == 5:   # 40 pairs listed twice
            d, t = np.concatenate([d, d[:40]]), np.concatenate([t, t[:40]])
        out.append(dict(Xd=Xd, Xt=Xt, d=d, t=t, g=1.0 / 6))
    return out


def normwise(u, ref):
    return float(np.max(np.abs(u - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n_cols", [13, 3])
def test_batched_product_matches_oracle(H, engine, n_cols):
    """The batched FP32 operator, w = R (M kron N) R^T v + shift v per problem and column, against
    the oracle's FP64 double sum, every output: FP32-class, normwise 1e-5 per column."""
    batch = product_batch()
    rng = np.random.default_rng(7)
    probs = [device_problem(H, p) for p in batch]
    V = [rng.standard_normal((len(p["d"]), n_cols)) for p in batch]
    shifts = list(np.linspace(0.0, 0.5, n_cols))
    vt = [torch.as_tensor(v, dtype=torch.float32, device=DEV) for v in V]
    W = with_engine(H, engine, lambda: gvt.matvec_batched(H, probs, vt, shifts))
    for b, p in enumerate(batch):
        if len(p["d"]) == 0:
            assert W[b].numel() == 0
            continue
        Mo, No = orc.gaussian_kernel(p["Xd"], gamma=p["g"]), orc.gaussian_kernel(p["Xt"], gamma=p["g"])
        v64 = vt[b].double().cpu().numpy()
        ref = orc.pairwise_matvec("kronecker", Mo, No, p["d"], p["t"], p["d"], p["t"], v64) + v64 * np.array(shifts)
        w = W[b].double().cpu().numpy()
        for c in range(n_cols):
            err = normwise(w[:, c], ref[:, c])
            assert err <= 1e-5, (engine, b, c, err)


def test_batched_engines_agree_and_tensor_cores_run(H):
    """The tensor-core operator gives the SIMT operator's outputs to FP32 rounding, and on this
    batch the forced engine takes a different path (not bitwise equal)."""
    batch = product_batch(seed=9)
    probs = [device_problem(H, p) for p in batch]
    rng = np.random.default_rng(3)
    vt = [torch.as_tensor(rng.standard_normal((len(p["d"]), 16)), dtype=torch.float32, device=DEV) for p in batch]
    Ws = with_engine(H, gvt.GVT_STAGE1_SIMT, lambda: gvt.matvec_batched(H, probs, vt))
    Wt = with_engine(H, gvt.GVT_STAGES_TC_F16X3, lambda: gvt.matvec_batched(H, probs, vt))
    differ = False
    for a, b in zip(Ws, Wt):
        if a.numel() == 0:
            continue
        a64, b64 = a.double().cpu().numpy(), b.double().cpu().numpy()
        assert normwise(b64, a64) <= 2e-5
        differ |= not np.array_equal(a64, b64)
    assert differ


def test_batched_product_full_size_sampled(H):
    """All 256 problems of the full batched configuration (m, q ~ U{32..512}, density ~ U[5 %, 60 %],
    16 columns) in one call on the tensor-core engine; 200 sampled outputs of the three largest
    problems and the smallest one against the oracle."""
    ps = synth.batched(256)
    rng = np.random.default_rng(1)
    probs, vt = [], []
    for p in ps:
        probs.append(device_problem(H, dict(Xd=p.Xd, Xt=p.Xt, d=p.d, t=p.t, g=p.gamma)))
        vt.append(torch.as_tensor(rng.standard_normal((p.n, 16)), dtype=torch.float32, device=DEV))
    shifts = list(ps[0].lambdas)
    W = with_engine(H, gvt.GVT_STAGES_TC_F16X3, lambda: gvt.matvec_batched(H, probs, vt, shifts))
    order = np.argsort([p.n for p in ps])
    for b in list(order[-3:]) + [order[0]]:
        p = ps[b]
        rows = np.sort(rng.choice(p.n, min(200, p.n), replace=False))
        Mo, No = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
        v64 = vt[b].double().cpu().numpy()
        ref = orc.pairwise_matvec("kronecker", Mo, No, p.d[rows], p.t[rows], p.d, p.t, v64)
        ref += v64[rows] * np.array(shifts)
        w = W[b].double().cpu().numpy()[rows]
        for c in range(16):
            err = normwise(w[:, c], ref[:, c])
            assert err <= 1e-5, (b, c, err)
