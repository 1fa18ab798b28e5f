"""Kernel logistic regression (Newton's method) on pairwise kernels on the GPU against the
oracle's Newton iteration (pinned by the optimality condition) and the optimality condition
itself, on the small drug-target sample and on a homogeneous MLPK problem."""
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


@pytest.mark.parametrize("kind", ["kronecker", "mlpk"])
def test_klr_matches_the_oracle_and_is_optimal(H, kind):
    p = synth.small(0) if kind not in gvt.HOMOGENEOUS else synth.homogeneous(0, m=64, n=1000)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    Mo, No = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    rng = np.random.default_rng(5)
    y = np.where(rng.standard_normal(p.n) + 0.5 * np.sin(p.d) > 0, 1.0, -1.0)
    lam = 0.05
    a, st, info = gvt.klr_newton_solve(H, plan, kind, M, N, torch.as_tensor(y, device=DEV), lam)
    assert st == 0
    mv = lambda x: orc.pairwise_matvec(kind, Mo, No, p.d, p.t, p.d, p.t, x)
    ref, it, _ = orc.klr_newton(mv, y, lam)
    an = a.cpu().numpy()
    print("%s: %d Newton steps, %d CG iterations (oracle %d Newton steps)"
          % (kind, info.refinements, info.iterations, it))
    assert np.max(np.abs(an - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref)))
    f = mv(an)
    sig = 1.0 / (1.0 + np.exp(y * f))
    assert np.max(np.abs(lam * an - y * sig)) <= 1e-8
    plan.close()
