"""Squared-hinge SVM (Newton's method over active sets) on pairwise kernels on the GPU against the
oracle's Newton iteration (pinned by the optimality conditions and an independent minimiser) and
against the optimality conditions themselves, computed from the oracle's explicit kernel matrix:
a = 0 outside S = {y_i f_i < 1} and (K_SS + lambda I) a_S = y_S.  Small drug-target sample
(Kronecker) and a homogeneous MLPK problem; plus the all-active case, which is kernel ridge
regression, and argument errors."""
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


def _setup(H, kind, seed=7):
    p = synth.small(0) if kind not in gvt.HOMOGENEOUS else synth.homogeneous(0, m=64, n=1000)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    Mo, No = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    rng = np.random.default_rng(seed)
    y = np.where(rng.standard_normal(p.n) + 0.8 * np.sin(p.d + 0.5 * p.t) > 0, 1.0, -1.0)
    K = orc.kernel_matrix(kind, Mo, No, p.d, p.t, p.d, p.t)    # explicit n x n (n = 1000)
    mv = lambda x: K @ x
    return p, M, N, plan, y, mv, K


@pytest.mark.parametrize("kind", ["kronecker", "mlpk"])
def test_svm_matches_the_oracle_and_is_optimal(H, kind):
    p, M, N, plan, y, mv, K = _setup(H, kind)
    lam = 0.05
    a, st, info = gvt.svm_newton_solve(H, plan, kind, M, N, torch.as_tensor(y, device=DEV), lam)
    assert st == 0
    ref, it, cg, ok = orc.svm_newton(mv, y, lam)
    assert ok
    an = a.cpu().numpy()
    print("%s: %d Newton steps, %d CG iterations, gradient %.1e (oracle %d steps, %d CG)"
          % (kind, info.refinements, info.iterations, info.rel_residual, it, cg))
    assert np.max(np.abs(an - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref)))
    # optimality from the explicit kernel matrix
    f = K @ an
    S = y * f < 1.0
    assert 0 < S.sum() < p.n
    assert np.all(an[~S] == 0.0)
    want = np.linalg.solve(K[np.ix_(S, S)] + lam * np.eye(S.sum()), y[S])
    assert np.max(np.abs(an[S] - want)) <= 1e-8 * max(1.0, np.max(np.abs(want)))
    assert info.rel_residual <= 1e-9
    plan.close()


def test_svm_all_active_is_kernel_ridge_regression(H):
    p, M, N, plan, y, mv, K = _setup(H, "kronecker", seed=8)
    lam = 200.0                                   # f stays small: every pair is active
    a, st, _ = gvt.svm_newton_solve(H, plan, "kronecker", M, N, torch.as_tensor(y, device=DEV), lam)
    assert st == 0
    yt = torch.as_tensor(y, device=DEV)
    b, st2, _ = gvt.krr_cg_solve(H, plan, "kronecker", M, N, yt, lam, rel_tol=1e-13)
    assert st2 == 0
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(y * mv(an) < 1.0)
    assert np.max(np.abs(an - bn)) <= 1e-10 * np.max(np.abs(bn))
    plan.close()


def test_svm_arguments_and_iteration_cap(H):
    p, M, N, plan, y, mv, K = _setup(H, "kronecker")
    yt = torch.as_tensor(y, device=DEV)
    with pytest.raises(gvt.GvtError):
        gvt.svm_newton_solve(H, plan, "kronecker", M, N, yt, 0.0)
    with pytest.raises(gvt.GvtError):
        gvt.svm_newton_solve(H, plan, "kronecker", M.float(), N.float(), yt, 0.1)
    a, st, info = gvt.svm_newton_solve(H, plan, "kronecker", M, N, yt, 0.05, newton_iters=1)
    assert st == gvt.GVT_ERR_NOT_CONVERGED and info.refinements == 1
    ref, _, _, _ = orc.svm_newton(mv, y, 0.05, newton_iters=1)
    assert np.max(np.abs(a.cpu().numpy() - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref)))
    plan.close()


@pytest.mark.parametrize("kind", ["kronecker", "mlpk"])
def test_hinge_svm_subgradient_matches_the_oracle(H, kind):
    """The hinge-loss SVM by kernelised sub-gradient steps: after 200 steps the GPU coefficients
    and objective equal the oracle's (the same deterministic sequence of FP64 products and
    margin tests; on this problem no margin comes within 1e-8 of 1, so rounding cannot flip a
    test)."""
    p, M, N, plan, y, mv, K = _setup(H, kind)
    lam = 2e-3          # small enough that pairs leave the margin (about half by step 200)
    a, J, info = gvt.svm_subgradient_solve(H, plan, kind, M, N, torch.as_tensor(y, device=DEV), lam, 200)
    ref, fref, Jref = orc.hinge_svm_subgradient(mv, y, lam, 200)
    an = a.cpu().numpy()
    print("%s: hinge objective %.6f (oracle %.6f)" % (kind, J, Jref))
    assert info.iterations == 200
    assert np.max(np.abs(an - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert abs(J - Jref) <= 1e-10 * abs(Jref)
    assert abs(J - orc.hinge_svm_objective(K @ an, an, y, lam)) <= 1e-10 * abs(J)
    # pairs left the margin during the run: the iterate is not the all-active fixed point y / (lam n)
    assert np.max(np.abs(an - y / (lam * p.n))) > 0.1 / (lam * p.n)
    plan.close()
