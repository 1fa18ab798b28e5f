"""Learned preconditioner on the GPU against the FP64 oracle, and what it gains.

* FP32 network (SIMT): features, network outputs, P r, the loss and its
  parameter gradient computed by the library's kernels equal the oracle's
  (oracle/precond.py, itself pinned by finite differences) to FP32 accuracy;
* BF16 network on the tensor cores (the default): outputs within the BF16
  bound of the oracle's; P r and the loss at the network's own outputs equal
  the oracle's to FP32 accuracy; the gradient equals the oracle's backward of
  the same output gradient within the BF16 bound of the backward products;
* training pairs recorded by FP32 CG (the handle's engine) and stored in BF16
  train the network as the FP64-recorded FP32 pairs do;
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


# BF16 bounds, unit roundoff u = 2^-9 for BF16 operands with FP32 accumulation.  The bound of a
# rounded sum is stated against the sum of the magnitudes of its terms (the network's sums cancel
# heavily, so a plain normwise ratio says little):
# * forward: the three layers round their input activations and weights once each, so an output
#   is off by a few u of the magnitudes feeding it: max|o - o*| <= 8u max(|W3| |h2| + |b3|);
# * backward: each weight-gradient entry sum_p g_p h_p (and each bias sum) is off by at most about
#   8u of sum_p |g_p| |h_p| with the backward magnitudes |g| propagated through |W| (a ReLU mask
#   that flips where z ~ 0 moves one term, within that magnitude).
BF16_U = 2.0 ** -9


def bf16_magnitudes(theta, cache, g_o):
    """Magnitude sums of the backward products: for each parameter block, sum over pairs of
    |gradient flowing in| x |activation|, the gradients propagated with |W| and without masks."""
    pp = lp.unpack(theta)
    X, z1, h1, z2, h2 = cache
    ag_o = np.abs(g_o)
    ag_h2 = ag_o @ np.abs(pp["W3"])
    ag_h1 = ag_h2 @ np.abs(pp["W2"])
    return {"W3": ag_o.T @ np.abs(h2), "b3": ag_o.sum(0), "W2": ag_h2.T @ np.abs(h1), "b2": ag_h2.sum(0),
            "W1": ag_h1.T @ np.abs(X), "b1": ag_h1.sum(0)}


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_forward_apply_and_gradient_match_oracle(H, dtype):
    P = setup(H, n=3000)
    theta = lp.init_params(3, out_scale=0.2)
    theta = theta + 0.02 * np.random.default_rng(1).standard_normal(theta.shape)
    pc = gvt.Precond(H, P["plan"], "kronecker", P["M"], P["N"], theta)
    pc.set_dtype(gvt.GVT_F32 if dtype == "f32" else gvt.GVT_BF16)
    mu, sd, X = pc.features()
    Xo = oracle_X(P)
    assert rel(X.cpu().numpy(), Xo) <= 1e-5
    th32 = theta.astype(np.float32).astype(np.float64)   # the GPU holds FP32 parameters
    Xg = X.double().cpu().numpy()
    o_ref, cache = lp.mlp_forward(th32, Xg)
    O = pc.outputs().cpu().numpy()
    err_o = rel(O, o_ref)
    if dtype == "f32":
        print("f32 network: outputs vs oracle %.2e" % err_o)
        assert err_o <= 1e-5
    else:
        pp = lp.unpack(th32)
        mag_o = np.abs(cache[4]) @ np.abs(pp["W3"]).T + np.abs(pp["b3"])
        err_m = float(np.max(np.abs(O - o_ref)) / np.max(mag_o))
        print("bf16 network: outputs vs oracle %.2e normwise, %.2e of the magnitudes (bound %.1e)"
              % (err_o, err_m, 8 * BF16_U))
        assert err_m <= 8 * BF16_U
    # P r from the network's own outputs: FP32/FP64 arithmetic in both dtypes
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
        if dtype == "f32":
            L_ref, g_ref = lp.loss_and_grad(th32, Xg, R.astype(np.float64), E.astype(np.float64), scale)
            assert abs(loss - L_ref) <= 1e-5 * abs(L_ref), scale
            assert rel(g, g_ref) <= 1e-4, scale
        else:
            # the loss and its output gradient at the network's own outputs, then the oracle's
            # backward of that output gradient
            L_ref, g_o = lp.loss_and_output_grad(O.astype(np.float64), R.astype(np.float64),
                                                 E.astype(np.float64), scale)
            g_ref = lp.mlp_backward(th32, cache, g_o)
            mags = bf16_magnitudes(th32, cache, g_o)
            gu, gr = lp.unpack(np.asarray(g, np.float64)), lp.unpack(g_ref)
            errs = {k: float(np.max(np.abs(gu[k] - gr[k])) / np.max(mags[k])) for k in mags}
            print("bf16 network, scale %g: loss %.4e vs %.4e; gradient errors of the magnitudes %s (normwise %.2e)"
                  % (scale, loss, L_ref, " ".join("%s %.1e" % kv for kv in sorted(errs.items())), rel(g, g_ref)))
            assert abs(loss - L_ref) <= 1e-5 * abs(L_ref), scale
            assert max(errs.values()) <= 8 * BF16_U, (scale, errs)
    pc.close()
    P["plan"].close()


def test_fp32_recorded_bf16_stored_pairs_match_and_train(H):
    """Pairs recorded by FP32 CG on FP32 kernel matrices and stored in BF16 agree with the FP64 CG's
    FP32-stored pairs over the first iterations: the first residual (y itself) to BF16 rounding, the
    next ones within 2 % (FP32 CG's iterates then drift from FP64 CG's as rounding differences grow,
    as CG's do: 0.4 % by the eighth iteration, 58 % by the tenth on this problem); and they train the
    BF16 network (the loss falls)."""
    P = setup(H, n=3000)
    lam = 1e-1
    y = torch.as_tensor(P["y"], device=DEV)
    a_star, st, _ = gvt.krr_cg_solve(H, P["plan"], "kronecker", P["M"], P["N"], y, lam, rel_tol=1e-10,
                                     max_iter=20000)
    assert st == 0
    iters = list(range(0, 10, 2))
    R64, E64 = gvt.cg_record_pairs(H, P["plan"], "kronecker", P["M"], P["N"], y, lam, a_star, iters)
    Rb, Eb = gvt.cg_record_pairs(H, P["plan"], "kronecker", P["M"].float(), P["N"].float(), y, lam, a_star, iters,
                                 store=torch.bfloat16)
    assert Rb.dtype == torch.bfloat16
    for k in range(len(iters)):
        er = float(torch.norm(Rb[:, k].double() - R64[:, k].double()) / torch.norm(R64[:, k].double()))
        ee = float(torch.norm(Eb[:, k].double() - E64[:, k].double()) / torch.norm(E64[:, k].double()))
        print("iteration %d: residual %.1e, correction %.1e apart" % (iters[k], er, ee))
        tol = 2 * 2.0 ** -9 if k == 0 else 2e-2
        assert er <= tol and ee <= tol, (k, er, ee)
    pc = gvt.Precond(H, P["plan"], "kronecker", P["M"], P["N"], lp.init_params(0, out_scale=0.01))
    hist = pc.train(Rb, Eb, steps=200, batch=5, lr=3e-3)
    print("BF16-stored pairs: loss %.3f -> %.3f" % (np.mean(hist[:5]), np.mean(hist[-10:])))
    assert np.mean(hist[-10:]) < 0.95 * np.mean(hist[:5])
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
