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


@pytest.mark.parametrize("lambdas", [[1e-3, 1e-2, 1e-1, 1.0], list(np.logspace(-3, 0, 16)), [0.5]])
def test_batched_solve_matches_cholesky(H, lambdas):
    batch = small_batch()
    probs = []
    for p in batch:
        M = gvt.gaussian_kernel(H, torch.as_tensor(p["Xd"], device=DEV), gamma=p["g"])
        N = gvt.gaussian_kernel(H, torch.as_tensor(p["Xt"], device=DEV), gamma=p["g"])
        probs.append(dict(M=M, N=N, d=torch.as_tensor(p["d"], device=DEV), t=torch.as_tensor(p["t"], device=DEV),
                          y=torch.as_tensor(p["y"], device=DEV)))
    A, st, info, rr = gvt.krr_solve_batched(H, probs, lambdas, rel_tol=1e-8)
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
