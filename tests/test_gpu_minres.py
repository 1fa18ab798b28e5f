"""MINRES (the solver of Sec. 6) on the GPU against the oracle's MINRES (itself pinned by the
Krylov minimum-residual property): iterate by iterate, through the recorded iterates used for
early stopping, and converged (residual recomputed by the oracle, same solution as CG)."""
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


def _setup(H, kind):
    p = synth.small(0) if kind not in gvt.HOMOGENEOUS else synth.homogeneous(0, m=64, n=1000)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    Mo, No = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    mv = lambda x: orc.pairwise_matvec(kind, Mo, No, p.d, p.t, p.d, p.t, x)
    y = p.y if p.y is not None else np.random.default_rng(3).standard_normal(p.n)
    return p, M, N, plan, mv, y


@pytest.mark.parametrize("kind", ["kronecker", "mlpk"])
def test_iterates_and_records_match_the_oracle(H, kind):
    p, M, N, plan, mv, y = _setup(H, kind)
    lam = 1e-2
    yd = torch.as_tensor(y, device=DEV)
    for k in (1, 3, 8):
        a, st, info, _ = gvt.krr_minres_solve(H, plan, kind, M, N, yd, lam, rel_tol=0.0, max_iter=k)
        assert st == gvt.GVT_ERR_NOT_CONVERGED and info.iterations == k
        ref, _, rel, _ = orc.minres_solve(mv, y, lam, tol=0.0, max_iter=k)
        an = a.cpu().numpy()
        assert np.max(np.abs(an - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), k
        assert abs(info.rel_residual - orc.relative_residual(mv, an, y, lam)) <= 1e-10
    a, st, info, rec = gvt.krr_minres_solve(H, plan, kind, M, N, yd, lam, rel_tol=0.0, max_iter=20,
                                            record_every=5, n_records=4)
    _, _, _, recs = orc.minres_solve(mv, y, lam, tol=0.0, max_iter=20, record_every=5)
    assert rec.shape == (p.n, 4) and len(recs) == 4
    for j in range(4):
        r = rec[:, j].cpu().numpy()
        if j == 0:   # after 5 steps the two runs still agree to rounding
            assert np.max(np.abs(r - recs[j])) <= 1e-8 * max(1.0, np.max(np.abs(recs[j])))
        # later, Lanczos rounding separates the iterates of the two runs, but both stay minimum-
        # residual iterates of the same Krylov dimension: their residual norms agree
        res_gpu = orc.relative_residual(mv, r, y, lam)
        res_orc = orc.relative_residual(mv, recs[j], y, lam)
        print("k=%d: residual %.6e (oracle MINRES %.6e)" % (5 * (j + 1), res_gpu, res_orc))
        assert abs(res_gpu - res_orc) <= 1e-3 * res_orc, j
    assert np.array_equal(rec[:, 3].cpu().numpy(), a.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("kind", ["kronecker", "symmetric"])
def test_converged_solution_matches_cg_and_the_oracle_residual(H, kind):
    p, M, N, plan, mv, y = _setup(H, kind)
    lam = 1e-2
    yd = torch.as_tensor(y, device=DEV)
    a, st, info, _ = gvt.krr_minres_solve(H, plan, kind, M, N, yd, lam, rel_tol=1e-9, max_iter=5000)
    assert st == 0
    an = a.cpu().numpy()
    rr = orc.relative_residual(mv, an, y, lam)
    print("%s: MINRES %d iterations, residual %.2e (oracle %.2e)" % (kind, info.iterations, info.rel_residual, rr))
    assert rr <= 1.2e-9 and abs(info.rel_residual - rr) <= 1e-12 + 1e-3 * rr
    c, st, _ = gvt.krr_cg_solve(H, plan, kind, M, N, yd, lam, rel_tol=1e-10, max_iter=5000)
    assert st == 0
    cn = c.cpu().numpy()
    assert np.max(np.abs(an - cn)) <= 1e-6 * np.max(np.abs(cn)) / lam
    plan.close()


def test_early_stopping_on_a_validation_setting(H):
    """New drugs held out (setting 2): MINRES iterates recorded every 4 steps, each one used to
    predict the held-out pairs through the cross kernels. The iterate is chosen by validation
    error and by validation AUC (the paper's measure), and the chosen iterates' predictions equal
    the oracle's product."""
    p = synth.merget(0, m=200, q=60, dim=8, n=4000)
    sp = synth.setting_split(p, 2, seed=4)
    g = p.gamma
    M = gvt.gaussian_kernel(H, torch.as_tensor(sp.Xd_train, device=DEV), gamma=g)
    N = gvt.gaussian_kernel(H, torch.as_tensor(sp.Xt_train, device=DEV), gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), sp.d, sp.t)
    a, st, info, rec = gvt.krr_minres_solve(H, plan, "kronecker", M, N, torch.as_tensor(sp.y, device=DEV), 1e-4,
                                            rel_tol=0.0, max_iter=60, record_every=4, n_records=15)
    Mx = gvt.gaussian_kernel(H, torch.as_tensor(sp.Xd_test, device=DEV), torch.as_tensor(sp.Xd_train, device=DEV),
                             gamma=g)
    Nx = gvt.gaussian_kernel(H, torch.as_tensor(sp.Xt_test, device=DEV), torch.as_tensor(sp.Xt_train, device=DEV),
                             gamma=g)
    pplan = gvt.Plan(H, tuple(Mx.shape), tuple(Nx.shape), sp.d, sp.t, sp.d_test, sp.t_test)
    preds = []
    for j in range(15):
        pr = gvt.predict(pplan, "kronecker", Mx, Nx, rec[:, j].contiguous()).cpu().numpy()
        preds.append(pr)
    # validation targets: the labels of the held-out pairs
    Xd_rows = {tuple(r) for r in np.round(sp.Xd_test, 12)}
    new_d = np.array([tuple(r) in Xd_rows for r in np.round(p.Xd, 12)])
    yv = p.y[new_d[p.d]]
    assert len(yv) == len(sp.d_test)
    errs = [float(np.mean((pr - yv) ** 2)) for pr in preds]
    best = int(np.argmin(errs))
    print("validation MSE by recorded iterate:", ["%.3f" % e for e in errs], "best", 4 * (best + 1))
    # the paper's measure: AUC with the labels above their median taken as interacting pairs
    pos = yv > np.median(yv)
    aucs = [orc.auc(pr, pos) for pr in preds]
    best_auc = int(np.argmax(aucs))
    print("validation AUC by recorded iterate:", ["%.3f" % a for a in aucs], "best", 4 * (best_auc + 1))
    assert aucs[best_auc] > 0.6     # the bilinear labels carry signal that the early iterates pick up
    ref_auc = orc.pairwise_matvec("kronecker", orc.gaussian_kernel(sp.Xd_test, sp.Xd_train, gamma=g),
                                  orc.gaussian_kernel(sp.Xt_test, sp.Xt_train, gamma=g), sp.d_test, sp.t_test,
                                  sp.d, sp.t, rec[:, best_auc].cpu().numpy())
    assert abs(orc.auc(ref_auc, pos) - aucs[best_auc]) <= 1e-3
    ref = orc.pairwise_matvec("kronecker", orc.gaussian_kernel(sp.Xd_test, sp.Xd_train, gamma=g),
                              orc.gaussian_kernel(sp.Xt_test, sp.Xt_train, gamma=g), sp.d_test, sp.t_test,
                              sp.d, sp.t, rec[:, best].cpu().numpy())
    assert np.max(np.abs(preds[best] - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    pplan.close()
    plan.close()
