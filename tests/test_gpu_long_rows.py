"""The sparse SIMT stages on long rows, against the FP64 oracle.

Homogeneous 6000 x 6000 Gaussian kernels with 150k pairs: the factor (144 MB in FP32) does not
fit in L2, so stage 1 runs several passes of column tiles over 1024-row blocks of B^T (the last
ragged), and the sampled gather-dot streams rows of 6000.  Kronecker (one term) and MLPK (ten
terms, squared factors) on 300 sampled output rows, each a sum over all pairs: FP32 within the
normwise 1e-5 tolerance, FP64 within 1e-10.
"""
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


@pytest.fixture(scope="module")
def prob():
    rng = np.random.default_rng(21)
    m, dim, n = 6000, 16, 150_000
    X = rng.standard_normal((m, dim))
    d, t = synth.random_pairs(rng, n, m, m)
    v = rng.standard_normal(n)
    return dict(X=X, d=d, t=t, v=v, g=1.0 / dim, m=m, Mo=orc.gaussian_kernel(X, gamma=1.0 / dim))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("kind", ["kronecker", "mlpk"])
def test_long_rows_match_the_oracle(H, prob, kind, dtype):
    p = prob
    M = gvt.gaussian_kernel(H, torch.as_tensor(p["X"], device=DEV), gamma=p["g"], dtype=dtype)
    plan = gvt.Plan(H, tuple(M.shape), tuple(M.shape), p["d"], p["t"])
    v = torch.as_tensor(p["v"], dtype=dtype, device=DEV)
    u = gvt.pairwise_kernel_matvec(plan, kind, M, M, v).double().cpu().numpy()
    plan.close()
    rows = np.sort(np.random.default_rng(5).choice(len(p["d"]), 300, replace=False))
    vv = v.double().cpu().numpy()
    ref = orc.pairwise_matvec(kind, p["Mo"], p["Mo"], p["d"][rows], p["t"][rows], p["d"], p["t"], vv)
    err = float(np.max(np.abs(u[rows] - ref)) / np.max(np.abs(ref)))
    tol = 1e-5 if dtype == torch.float32 else 1e-10
    print("%s %s: normwise error %.2e" % (kind, dtype, err))
    assert err <= tol, err
