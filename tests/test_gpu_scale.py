"""Full-size kernel-filling configuration: m = q = 20000 objects, 256-d
features, 10M pairs with power-law degrees (Zipf 1.1 weights).

The GVT product runs on the whole sample, and 200 sampled output rows are
checked against the FP64 oracle; each row is a sum over all 10M input pairs.
* FP32 operands under the automatic engine (here the dense tensor-core
  stages): normwise error within the FP32 tolerance 1e-5;
* FP64 operands (SIMT stages): within 1e-10.
The oracle evaluates only the kernel rows these outputs need.
"""
import time

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


def test_kernel_filling_scale_sampled_parity(H):
    t0 = time.perf_counter()
    p = synth.zipf(0)
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(p.n, 200, replace=False))
    # kernel rows of the sampled outputs only (the oracle's M and N for those rows)
    ud, id_ = np.unique(p.d[rows], return_inverse=True)
    ut, it_ = np.unique(p.t[rows], return_inverse=True)
    Mo = orc.gaussian_kernel(p.Xd[ud], p.Xd, gamma=p.gamma)
    No = orc.gaussian_kernel(p.Xt[ut], p.Xt, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    for dtype, tol, engine in ((torch.float32, 1e-5, gvt.GVT_STAGES_AUTO),
                               (torch.float64, 1e-10, gvt.GVT_STAGE1_SIMT)):
        M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=dtype)
        N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma, dtype=dtype)
        v = torch.as_tensor(p.v, dtype=dtype, device=DEV)
        gvt.gvt_set_stage1_engine(H.h, engine)
        try:
            gvt.pairwise_kernel_matvec(plan, "kronecker", M, N, v)   # warm-up (workspace)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            u = gvt.pairwise_kernel_matvec(plan, "kronecker", M, N, v)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t1) * 1e3
            gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        finally:
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
        vin = v.double().cpu().numpy()
        ref = orc.pairwise_matvec("kronecker", Mo, No, id_, it_, p.d, p.t, vin)
        got = u.double().cpu().numpy()[rows]
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print("%s: product %.1f ms (%.2e pair-terms/s), error vs FP64 on 200 rows %.2e (generation %.1f s)"
              % (dtype, ms, float(p.n) * p.n / (ms / 1e3), err, gen_s))
        assert err <= tol
        del M, N, v, u
    plan.close()
