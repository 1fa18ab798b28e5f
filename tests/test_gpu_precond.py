"""Learned preconditioner on the GPU against the FP64 oracle, and what it gains.

* features, network outputs, P r, the loss and its parameter gradient computed
  by the library's kernels equal the oracle's (oracle/precond.py, itself pinned
  by finite differences) to FP32 accuracy;
* training on residual -> correction pairs from the exact solver lowers the
  loss; flexible CG with the trained P reaches the FP64 relative residual 1e-6
  (re-checked by the oracle), alone and inside mixed-precision refinement, and
  the test prints what the trained network gains over plain CG (iterations and
  time; on these Gaussian-kernel problems the gain is negative, which is why
  plain CG stays the default and the fallback);
* a preconditioner that cannot converge within its flexible-CG budget hands
  over to plain CG, and the solution is still correct.
"""
import time
import numpy as np
import pytest

import oracle as orc
from oracle import precond as lp
from paper_2009_01054_gb300 import gvt

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


def zipf_problem(m=150, q=120, n=6000, s=1.1, dim=8, seed=0):
    """Pairs whose drug and target degrees follow a truncated power law (no repeats)."""
    rng = np.random.default_rng(seed)
    Xd, Xt = rng.standard_normal((m, dim)), rng.standard_normal((q, dim))
    pd = np.arange(1, m + 1) ** -s
    pt = np.arange(1, q + 1) ** -s
    pd, pt = pd / pd.sum(), pt / pt.sum()
    perm_d, perm_t = rng.permutation(m), rng.permutation(q)
    keys = set()
    while len(keys) < n:
        dd = perm_d[rng.choice(m, 4 * n, p=pd)]
        tt = perm_t[rng.choice(q, 4 * n, p=pt)]
        for a, b in zip(dd, tt):
            keys.add(int(a) * q + int(b))
            if len(keys) == n:
                break
    k = np.array(sorted(keys))
    d, t = (k // q).astype(np.int32), (k % q).astype(np.int32)
    y = rng.standard_normal(n)
    return Xd, Xt, d, t, y, 1.0 / dim


def setup(H, n=6000):
    Xd, Xt, d, t, y, g = zipf_problem(n=n)
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    return dict(M=M, N=N, plan=plan, d=d, t=t, y=y, Mo=Mo, No=No)


def oracle_X(P):
    mv = lambda v: orc.pairwise_matvec("kronecker", P["Mo"], P["No"], P["d"], P["t"], P["d"], P["t"], v)
    F = lp.pair_features(P["Mo"], P["No"], P["d"], P["t"], P["Mo"].shape[0], P["No"].shape[0], matvec=mv)
    mu, sd = lp.normalisation(F)
    return (F - mu) / sd


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(np.max(np.abs(b)), 1e-300))


def test_forward_apply_and_gradient_match_oracle(H):
    P = setup(H, n=3000)
    theta = lp.init_params(3, out_scale=0.2)
    theta = theta + 0.02 * np.random.default_rng(1).standard_normal(theta.shape)
    pc = gvt.Precond(H, P["plan"], "kronecker", P["M"], P["N"], theta)
    mu, sd, X = pc.features()
    Xo = oracle_X(P)
    assert rel(X.cpu().numpy(), Xo) <= 1e-5
    th32 = theta.astype(np.float32).astype(np.float64)   # the GPU holds FP32 parameters
    o_ref, _ = lp.mlp_forward(th32, X.double().cpu().numpy())
    O = pc.outputs().cpu().numpy()
    assert rel(O, o_ref) <= 1e-5
    D, V = lp.outputs_to_DV(O.astype(np.float64))
    r = np.random.default_rng(2).standard_normal(len(P["d"]))
    z = pc.apply(torch.as_tensor(r, device=DEV)).cpu().numpy()
    assert rel(z, lp.apply_P(D, V, r)) <= 1e-5
    K = 5
    rng = np.random.default_rng(3)
    R = rng.standard_normal((len(P["d"]), K)).astype(np.float32)
    E = rng.standard_normal((len(P["d"]), K)).astype(np.float32)
    for scale in (1.0, 37.5):
        pc.scale(scale)
        loss, g = pc.loss_grad(torch.as_tensor(R, device=DEV), torch.as_tensor(E, device=DEV))
        L_ref, g_ref = lp.loss_and_grad(th32, X.double().cpu().numpy(), R.astype(np.float64),
                                        E.astype(np.float64), scale)
        assert abs(loss - L_ref) <= 1e-5 * abs(L_ref), scale
        assert rel(g, g_ref) <= 1e-4, scale
    pc.close()
    P["plan"].close()


def timed_solve(H, P, y, lam, **kw):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a, st, info = gvt.krr_cg_solve(H, P["plan"], "kronecker", P["M"], P["N"], y, lam, rel_tol=1e-6, **kw)
    torch.cuda.synchronize()
    return a, st, info, (time.perf_counter() - t0) * 1e3


def oracle_residual(P, a, lam):
    mv = lambda x: orc.pairwise_matvec("kronecker", P["Mo"], P["No"], P["d"], P["t"], P["d"], P["t"], x)
    return orc.relative_residual(mv, a.cpu().numpy(), P["y"], lam)


def test_training_lowers_loss_and_reports_the_gain_over_plain_cg(H):
    P = setup(H, n=6000)
    lam = 1e-2
    y = torch.as_tensor(P["y"], device=DEV)
    a_star, st, info = gvt.krr_cg_solve(H, P["plan"], "kronecker", P["M"], P["N"], y, lam, rel_tol=1e-12,
                                        max_iter=20000)
    assert st == 0
    a_plain, st, info_plain, ms_plain = timed_solve(H, P, y, lam)
    assert st == 0
    plain_iters = info_plain.iterations
    iters = list(range(0, min(plain_iters, 64), 2))
    R, E = gvt.cg_record_pairs(H, P["plan"], "kronecker", P["M"], P["N"], y, lam, a_star, iters)
    pc = gvt.Precond(H, P["plan"], "kronecker", P["M"], P["N"], lp.init_params(0, out_scale=0.01))
    hist = pc.train(R, E, steps=400, batch=8, lr=3e-3)
    c = pc.scale()
    assert abs(c - lp.data_scale(R.double().cpu().numpy(), E.double().cpu().numpy())) <= 1e-5 * abs(c)
    assert np.mean(hist[-20:]) < 0.95 * np.mean(hist[:5])
    a, st, info, ms = timed_solve(H, P, y, lam, precond=pc, max_iter=20000)
    assert st == 0
    rr = oracle_residual(P, a, lam)
    print("plain CG: %d iterations, %.1f ms; learned flexible CG: %d iterations, %.1f ms (fallback %d); "
          "gain x%.2f in iterations; scale %.3g; loss %.3f -> %.3f; oracle residual %.2e"
          % (plain_iters, ms_plain, info.iterations, ms, info.precond_fallback, plain_iters / info.iterations,
             c, np.mean(hist[:5]), np.mean(hist[-20:]), rr))
    assert rr <= 1.05e-6
    # the preconditioner does not change the solution
    assert float(torch.norm(a - a_plain) / torch.norm(a_plain)) <= 1e-4
    # the same preconditioner inside mixed-precision refinement
    a2, st, info2, ms2 = timed_solve(H, P, y, lam, mode=gvt.GVT_SOLVE_MIXED_IR, precond=pc, max_iter=20000)
    assert st == 0 and oracle_residual(P, a2, lam) <= 1.05e-6
    print("mixed refinement with the learned P: %d inner iterations, %.1f ms (fallback %d)"
          % (info2.iterations, ms2, info2.precond_fallback))
    pc.close()
    P["plan"].close()


@pytest.mark.parametrize("mode", [gvt.GVT_SOLVE_FP64_CG, gvt.GVT_SOLVE_MIXED_IR])
def test_flexible_cg_budget_falls_back_to_plain_cg(H, mode):
    P = setup(H, n=3000)
    lam = 1e-2
    y = torch.as_tensor(P["y"], device=DEV)
    # large random low-rank outputs: a poor preconditioner, far from (K + lam I)^-1
    pc = gvt.Precond(H, P["plan"], "kronecker", P["M"], P["N"], lp.init_params(5, out_scale=1.0))
    pc.scale(1.0 / lam)
    a, st, info, _ = timed_solve(H, P, y, lam, mode=mode, precond=pc, precond_budget=5, max_iter=20000)
    assert st == 0 and info.precond_fallback == 1
    assert oracle_residual(P, a, lam) <= 1.05e-6
    _, st, info0, _ = timed_solve(H, P, y, lam, mode=mode)
    assert st == 0 and info0.precond_fallback == 0
    pc.close()
    P["plan"].close()
