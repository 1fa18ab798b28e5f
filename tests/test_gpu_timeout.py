"""Failure detection on the GPU without a fault: a bounded wait of the tensor-core GEMM is made
to run out, and the kernel's timeout path is checked end to end.

gvt_set_tc_stall_test makes the GEMM's MMA thread wait about 1 ms (2e6 SM cycles) on an mbarrier
that nothing arrives on.  The wait expires; the kernel's other threads stop waiting, it waits
(bounded) for the tile copies it had issued, frees its tensor memory and returns, and the
handle's device error word holds GVT_ERR_TIMEOUT.  The context stays usable: with the switch off,
the same GEMM on the same handle is correct, and so are a dense-engine product and a
mixed-precision solve, which themselves report GVT_ERR_TIMEOUT while the switch is on.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2009_01054_gb300 import gvt, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
STALL = 2_000_000     # SM cycles, about 1 ms at 2 GHz


@pytest.fixture(scope="module")
def H():
    from paper_2009_01054_gb300 import build
    build.build()
    h = gvt.Handle()
    yield h
    gvt.gvt_set_tc_stall_test(h.h, 0)
    h.close()


def _gemm(H, A, B, C):
    M, K = A.shape
    N = B.shape[0]
    gvt.gvt_tc_gemm_bf16(H.h, gvt.ptr(A), K, gvt.ptr(B), K, gvt.ptr(C), N, M, N, K, gvt.stream_ptr())
    torch.cuda.synchronize()


def test_expired_wait_reports_timeout_and_the_next_gemm_is_correct(H):
    g = torch.Generator(device=DEV).manual_seed(5)
    A = torch.randn(256, 256, generator=g, device=DEV).to(torch.bfloat16)
    B = torch.randn(256, 256, generator=g, device=DEV).to(torch.bfloat16)
    C = torch.zeros(256, 256, device=DEV)
    gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())          # a clean error word to start
    gvt.gvt_set_tc_stall_test(H.h, STALL)
    try:
        _gemm(H, A, B, C)
        with pytest.raises(gvt.GvtError) as e:
            gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        assert e.value.status == gvt.GVT_ERR_TIMEOUT
    finally:
        gvt.gvt_set_tc_stall_test(H.h, 0)
    gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())          # reading it cleared the word
    _gemm(H, A, B, C)
    gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    ref = (A.double() @ B.double().T).cpu().numpy()
    err = np.max(np.abs(C.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


def test_stall_switch_is_refused_in_the_sm_pair_form_and_checks_its_argument(H):
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device=DEV)
    C = torch.zeros(128, 128, device=DEV)
    with pytest.raises(gvt.GvtError) as e:
        gvt.gvt_set_tc_stall_test(H.h, -1)
    assert e.value.status == gvt.GVT_ERR_INVALID_ARG
    gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_ON)
    gvt.gvt_set_tc_stall_test(H.h, STALL)
    try:
        with pytest.raises(gvt.GvtError) as e:
            gvt.gvt_tc_gemm_bf16(H.h, gvt.ptr(A), 64, gvt.ptr(A), 64, gvt.ptr(C), 128, 128, 128, 64,
                                 gvt.stream_ptr())
        assert e.value.status == gvt.GVT_ERR_UNSUPPORTED
    finally:
        gvt.gvt_set_tc_stall_test(H.h, 0)
        gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_AUTO)


def test_product_and_solve_report_the_timeout_then_recover(H):
    rng = np.random.default_rng(8)
    m, q, dim = 200, 60, 8
    Xd, Xt = rng.standard_normal((m, dim)), rng.standard_normal((q, dim))
    n = int(0.4 * m * q)
    cells = rng.choice(m * q, n, replace=False)
    d, t = (cells // q).astype(np.int32), (cells % q).astype(np.int32)
    g = 1.0 / dim
    M64 = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g)
    N64 = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g)
    plan = gvt.Plan(H, (m, m), (q, q), d, t)
    v = torch.as_tensor(rng.standard_normal(n), dtype=torch.float32, device=DEV)
    y = torch.as_tensor(rng.standard_normal(n), device=DEV)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X3)
    gvt.gvt_set_tc_stall_test(H.h, STALL)
    try:
        gvt.pairwise_kernel_matvec(plan, "kronecker", M64.float(), N64.float(), v)
        torch.cuda.synchronize()
        with pytest.raises(gvt.GvtError) as e:
            gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        assert e.value.status == gvt.GVT_ERR_TIMEOUT
        with pytest.raises(gvt.GvtError) as e:
            gvt.krr_cg_solve(H, plan, "kronecker", M64, N64, y, 1e-1, mode=gvt.GVT_SOLVE_MIXED_IR, max_iter=50)
        assert e.value.status == gvt.GVT_ERR_TIMEOUT
    finally:
        gvt.gvt_set_tc_stall_test(H.h, 0)
    gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    try:
        u = gvt.pairwise_kernel_matvec(plan, "kronecker", M64.float(), N64.float(), v).double().cpu().numpy()
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M64, N64, y, 1e-1, mode=gvt.GVT_SOLVE_MIXED_IR)
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    ref = orc.pairwise_matvec("kronecker", Mo, No, d, t, d, t, v.double().cpu().numpy())
    assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) <= 1e-5
    assert st == 0
    mv = lambda x: orc.pairwise_matvec("kronecker", Mo, No, d, t, d, t, x)
    assert orc.relative_residual(mv, a.cpu().numpy(), y.cpu().numpy(), 1e-1) <= 1.05e-6
    plan.close()
