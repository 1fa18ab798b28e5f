"""Training and prediction in the four settings of Sec. 2 (random pairs; new drugs; new
targets; both new), with rectangular cross kernels K(X_test, X_train) for the unseen objects:
the training solve is checked by the oracle's residual, and the predictions (FP64, and FP32 on
the automatic engine) against the oracle's product with the same dual coefficients."""
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


def _gauss(H, X, Y, g, dtype=torch.float64):
    return gvt.gaussian_kernel(H, torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV), gamma=g,
                               dtype=dtype)


@pytest.mark.parametrize("setting", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["kronecker", "linear", "poly2d"])
def test_train_and_predict_in_each_setting(H, setting, kind):
    p = synth.merget(0, m=300, q=80, dim=8, n=6000)
    sp = synth.setting_split(p, setting, seed=2)
    g = p.gamma
    M = _gauss(H, sp.Xd_train, sp.Xd_train, g)
    N = _gauss(H, sp.Xt_train, sp.Xt_train, g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), sp.d, sp.t)
    lam = 1e-2
    a, st, info = gvt.krr_cg_solve(H, plan, kind, M, N, torch.as_tensor(sp.y, device=DEV), lam, rel_tol=1e-8,
                                   max_iter=20000)
    assert st == 0
    Mo = orc.gaussian_kernel(sp.Xd_train, gamma=g)
    No = orc.gaussian_kernel(sp.Xt_train, gamma=g)
    mv = lambda x: orc.pairwise_matvec(kind, Mo, No, sp.d, sp.t, sp.d, sp.t, x)
    an = a.cpu().numpy()
    assert orc.relative_residual(mv, an, sp.y, lam) <= 1.05e-8
    Mx = _gauss(H, sp.Xd_test, sp.Xd_train, g)
    Nx = _gauss(H, sp.Xt_test, sp.Xt_train, g)
    pplan = gvt.Plan(H, tuple(Mx.shape), tuple(Nx.shape), sp.d, sp.t, sp.d_test, sp.t_test)
    pred = gvt.predict(pplan, kind, Mx, Nx, a).cpu().numpy()
    ref = orc.pairwise_matvec(kind, orc.gaussian_kernel(sp.Xd_test, sp.Xd_train, gamma=g),
                              orc.gaussian_kernel(sp.Xt_test, sp.Xt_train, gamma=g),
                              sp.d_test, sp.t_test, sp.d, sp.t, an)
    scale = max(np.max(np.abs(ref)), 1e-300)
    assert np.max(np.abs(pred - ref)) / scale <= 1e-10
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_AUTO)
    try:
        pred32 = gvt.predict(pplan, kind, Mx.float(), Nx.float(), a.float()).double().cpu().numpy()
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    Mxo = orc.gaussian_kernel(sp.Xd_test, sp.Xd_train, gamma=g)
    Nxo = orc.gaussian_kernel(sp.Xt_test, sp.Xt_train, gamma=g)
    a32 = an.astype(np.float32).astype(np.float64)
    ref32 = orc.pairwise_matvec(kind, Mxo, Nxo, sp.d_test, sp.t_test, sp.d, sp.t, a32)
    # The dual coefficients of a lambda = 1e-2 solve cancel strongly inside each prediction sum.
    # The FP32 bound is stated relative to the summed magnitudes max_i (|K||a|)_i (these kernels
    # have nonnegative entries, so |K| = K): an FP32 sum is exact only to a multiple of
    # 2^-24 * sum_j |terms_j|, whatever its value.  The plain normwise error max|u - u*| / max|u*|
    # is printed beside it with the cancellation factor max|K||a| / max|u*| that separates them.
    mag = orc.pairwise_matvec(kind, Mxo, Nxo, sp.d_test, sp.t_test, sp.d, sp.t, np.abs(a32))
    diff = np.max(np.abs(pred32 - ref32))
    err = diff / np.max(mag)
    plain = diff / max(np.max(np.abs(ref32)), 1e-300)
    cancel = np.max(mag) / max(np.max(np.abs(ref32)), 1e-300)
    print("setting %d %s: FP32 prediction error %.2e of max |K||a|, normwise %.2e, cancellation x%.1f"
          % (setting, kind, err, plain, cancel))
    assert err <= 1e-5
    pplan.close()
    plan.close()
