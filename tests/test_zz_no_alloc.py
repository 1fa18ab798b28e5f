"""The allocation-free Kronecker product gvt_matvec_static.

Callers that cannot allocate device memory (a framework that owns all device
memory through its own pool, or a latency-bound loop where cudaMalloc and
cudaFree are not allowed) use gvt_matvec_static, whose scratch is a fixed
static device array.  This file checks, through the C ABI, that two calls in
a row agree with the FP64 oracle's product and with the existing gvt_matvec
(plan + handle) within the tolerances of the other parity tests (1e-10 FP64,
1e-5 FP32, normwise), that the shared array is cleared between calls, that a
call leaves the device's free memory and torch's allocation unchanged, and
that requests beyond its size are refused.  It is named so that pytest
collects it last.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2009_01054_gb300 import gvt, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}


def normwise(u, ref):
    return float(np.max(np.abs(u - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _static(M, N, d, t, do, to, v, m_shape, q_shape, sym=True, check_memory=False):
    """One call through the C ABI into a preallocated output; with check_memory, the device's free
    bytes and torch's allocated bytes are read right before and after the call itself."""
    u = torch.empty(do.numel() if do is not None else d.numel(), dtype=v.dtype, device="cuda")
    mats = (gvt.matrix(M, sym), gvt.matrix(N, sym))
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()) if check_memory else None
    gvt.gvt_matvec_static(m_shape[0], m_shape[1], q_shape[0], q_shape[1],
                          gvt.ptr(d), gvt.ptr(t), d.numel(),
                          gvt.ptr(do) if do is not None else None,
                          gvt.ptr(to) if to is not None else None,
                          do.numel() if do is not None else 0,
                          mats[0], mats[1], gvt.ptr(v), gvt.ptr(u),
                          gvt.dtype_code(v), gvt.stream_ptr())
    torch.cuda.synchronize()
    if check_memory:
        after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        assert after == before, (before, after)   # the call allocated no device memory
    return u.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", ["small_predict", "small_train", "rect_nonsym"])
def test_static_matches_planned_matvec_twice(dtype, case):
    from paper_2009_01054_gb300 import build
    build.build()
    H = gvt.Handle()
    rng = np.random.default_rng(4)
    if case.startswith("small"):
        p = synth.small(0)
        Xd, Xt, Yd, Yt = p.Xd, p.Xt, p.Xd, p.Xt
        d, t = p.d, p.t
        do, to = (p.d_pred, p.t_pred) if case == "small_predict" else (None, None)
        v = p.v
        sym = True
    else:   # cross kernels (prediction side 25 x 17, training side 300 x 90): transposed reads
        Xd, Xt = rng.standard_normal((300, 6)), rng.standard_normal((90, 6))
        Yd, Yt = rng.standard_normal((25, 6)), rng.standard_normal((17, 6))
        d, t = synth.random_pairs(rng, 5000, 300, 90)
        do, to = synth.random_pairs(rng, 2000, 25, 17)
        v = rng.standard_normal(5000)
        sym = False
    dev = "cuda"
    M = gvt.gaussian_kernel(H, torch.as_tensor(Yd, device=dev), torch.as_tensor(Xd, device=dev),
                            gamma=1.0 / Xd.shape[1], dtype=dtype)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Yt, device=dev), torch.as_tensor(Xt, device=dev),
                            gamma=1.0 / Xd.shape[1], dtype=dtype)
    dd = torch.as_tensor(d, dtype=torch.int32, device=dev)
    tt = torch.as_tensor(t, dtype=torch.int32, device=dev)
    ddo = None if do is None else torch.as_tensor(do, dtype=torch.int32, device=dev)
    tto = None if to is None else torch.as_tensor(to, dtype=torch.int32, device=dev)
    vv = torch.as_tensor(v, dtype=dtype, device=dev)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), dd, tt, ddo, tto)
    n_out = plan.n_out
    ref = torch.empty(n_out, dtype=dtype, device=dev)
    gvt.gvt_matvec(plan.p, gvt.matrix(M, sym), gvt.matrix(N, sym), gvt.ptr(vv), gvt.ptr(ref), 1,
                   gvt.dtype_code(vv), gvt.stream_ptr())
    torch.cuda.synchronize()
    ref = ref.double().cpu().numpy()
    # the oracle's product on the same (dtype-rounded) kernel matrices and v, in FP64
    d_o = d if do is None else do
    t_o = t if to is None else to
    oref = orc.pairwise_matvec("kronecker", M.double().cpu().numpy(), N.double().cpu().numpy(),
                               d_o, t_o, d, t, vv.double().cpu().numpy())
    u1 = _static(M, N, dd, tt, ddo, tto, vv, tuple(M.shape), tuple(N.shape), sym)
    u2 = _static(M, N, dd, tt, ddo, tto, vv, tuple(M.shape), tuple(N.shape), sym, check_memory=True)
    print("%s %s: static vs oracle %.2e / %.2e, vs gvt_matvec %.2e" %
          (case, dtype, normwise(u1, oref), normwise(u2, oref), normwise(u1, ref)))
    assert normwise(u1, oref) <= TOL[dtype]
    assert normwise(u2, oref) <= TOL[dtype]     # second call: the shared array was cleared
    assert normwise(u1, ref) <= TOL[dtype]
    assert normwise(u2, ref) <= TOL[dtype]
    plan.close()
    H.close()


def test_static_refuses_oversized_and_bad_indices():
    from paper_2009_01054_gb300 import build
    build.build()
    dev = "cuda"
    big = torch.zeros((2100, 2100), dtype=torch.float64, device=dev)   # 2100^2 * 8 B > 16 MiB
    d = torch.zeros(4, dtype=torch.int32, device=dev)
    v = torch.zeros(4, dtype=torch.float64, device=dev)
    u = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(gvt.GvtError) as e:
        gvt.gvt_matvec_static(2100, 2100, 2100, 2100, gvt.ptr(d), gvt.ptr(d), 4, None, None, 0,
                              gvt.matrix(big, True), gvt.matrix(big, True), gvt.ptr(v), gvt.ptr(u),
                              gvt.GVT_F64, gvt.stream_ptr())
    assert e.value.status == 1 and "static scratch" in str(e.value)
    small = torch.eye(8, dtype=torch.float64, device=dev)
    bad = torch.tensor([0, 9, 1, 2], dtype=torch.int32, device=dev)
    with pytest.raises(gvt.GvtError) as e:
        gvt.gvt_matvec_static(8, 8, 8, 8, gvt.ptr(bad), gvt.ptr(d), 4, None, None, 0,
                              gvt.matrix(small, True), gvt.matrix(small, True), gvt.ptr(v), gvt.ptr(u),
                              gvt.GVT_F64, gvt.stream_ptr())
    assert e.value.status == 2
