"""Multi-shift CG for a lambda sweep on the GPU against the oracle's multi-shift CG (itself
pinned by per-shift plain CG iterates) and against direct solves and separate CG runs."""
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


@pytest.mark.parametrize("kind", ["kronecker", "poly2d"])
def test_sweep_matches_oracle_iterates_and_direct_solves(H, kind):
    p = synth.small(0)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    Mo, No = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    mv = lambda x: orc.pairwise_matvec(kind, Mo, No, p.d, p.t, p.d, p.t, x)
    lams = [3e-2, 1e-3, 1.0, 1e-1, 1e-2]
    y = torch.as_tensor(p.y, device=DEV)
    for k in (1, 2, 5):
        A, st, info, _ = gvt.krr_cg_solve_multishift(H, plan, kind, M, N, y, lams, rel_tol=0.0, max_iter=k)
        assert st == gvt.GVT_ERR_NOT_CONVERGED and info.iterations == k
        ref, it, _ = orc.cg_multishift(mv, p.y, lams, tol=0.0, max_iter=k)
        An = A.cpu().numpy()
        assert np.max(np.abs(An - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), k
    A, st, info, rr = gvt.krr_cg_solve_multishift(H, plan, kind, M, N, y, lams, rel_tol=1e-10, max_iter=20000)
    assert st == 0
    K = orc.kernel_matrix(kind, Mo, No, p.d, p.t, p.d, p.t)
    An = A.cpu().numpy()
    for s, lam in enumerate(lams):
        ref = orc.krr_solve_dense(K, p.y, lam)
        res = orc.relative_residual(mv, An[:, s], p.y, lam)
        assert res <= 1e-9 and abs(rr[s] - res) <= 1e-12 + 1e-3 * res, (s, res, rr[s])
        assert np.max(np.abs(An[:, s] - ref)) <= 1e-6 * max(1.0, np.max(np.abs(ref))) / lam, s
    plan.close()


def test_merget_sweep_against_separate_solves(H):
    """Merget-shaped (m=2000, q=250, 120k pairs): the sweep lambda in {1e-4, 1e-2, 1} in one
    multi-shift run reaches the same solutions as three FP64 CG solves."""
    import time
    p = synth.merget(0)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    y = torch.as_tensor(p.y, device=DEV)
    lams = [1e-4, 1e-2, 1.0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A, st, info, rr = gvt.krr_cg_solve_multishift(H, plan, "kronecker", M, N, y, lams, rel_tol=1e-6)
    torch.cuda.synchronize()
    ms_sweep = (time.perf_counter() - t0) * 1e3
    assert st == 0 and max(rr) <= 1.05e-6
    ms_sep = 0.0
    for s, lam in enumerate(lams):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a, st, inf = gvt.krr_cg_solve(H, plan, "kronecker", M, N, y, lam, rel_tol=1e-6, check_every=10)
        torch.cuda.synchronize()
        ms_sep += (time.perf_counter() - t0) * 1e3
        assert st == 0
        diff = torch.norm(A[:, s] - a) / torch.norm(a)
        assert float(diff) <= 1e-4 / lam * 1e-2 + 1e-5, (s, float(diff))
    print("multi-shift sweep %.1f ms (%d iterations) vs three CG solves %.1f ms" % (ms_sweep, info.iterations,
                                                                                  ms_sep))
    plan.close()
