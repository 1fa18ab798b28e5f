"""Per-tile dense/sparse stages (gvt_set_stage_tiles) against the FP64 oracle.

Ids are relabelled by decreasing degree; W^T tiles (256 x 64) and output tiles (128 x 256) with
more pairs than the break-even count run on the tensor-core GEMM (block-sparse stage 1, tile-list
stage 2), the remaining pairs on the SIMT stages.  On a Zipf-degree sample (power-law degrees: a
dense corner and a sparse tail, so both parts carry work, checked through the library's stage
statistics) the forced per-tile product equals the oracle's within the FP32 tolerance on the
FP16x3 engine and within the single-pass rounding bound on the FP16x1 engine, on 300 sampled
output rows (each a sum over all pairs), for training and prediction plans; and it agrees with
the dense engine's product to FP32 rounding.
"""
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


@pytest.fixture(scope="module")
def zp():
    return synth.zipf(3, m=3000, dim=16, n=400_000)


def _rows_ref(p, rows, v, d_out=None, t_out=None):
    d_o = p.d if d_out is None else d_out
    t_o = p.t if t_out is None else t_out
    ud, id_ = np.unique(d_o[rows], return_inverse=True)
    ut, it_ = np.unique(t_o[rows], return_inverse=True)
    Mo = orc.gaussian_kernel(p.Xd[ud], p.Xd, gamma=p.gamma)
    No = orc.gaussian_kernel(p.Xt[ut], p.Xt, gamma=p.gamma)
    ref = orc.pairwise_matvec("kronecker", Mo, No, id_.astype(np.int32), it_.astype(np.int32), p.d, p.t, v)
    mag = orc.pairwise_matvec("kronecker", Mo, No, id_.astype(np.int32), it_.astype(np.int32), p.d, p.t, np.abs(v))
    return ref, mag


def _product(H, plan, M, N, v, engine, tiles):
    gvt.gvt_set_stage1_engine(H.h, engine)
    gvt.gvt_set_stage_tiles(H.h, tiles)
    gvt.gvt_stats_enable(H.h, True)
    try:
        u = gvt.pairwise_kernel_matvec(plan, "kronecker", M, N, v).double().cpu().numpy()
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        stats = gvt.gvt_stats_read(H.h)
    finally:
        gvt.gvt_stats_enable(H.h, False)
        gvt.gvt_set_stage_tiles(H.h, gvt.GVT_TILES_AUTO)
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    return u, stats


@pytest.mark.parametrize("engine,bound", [(gvt.GVT_STAGES_AUTO, 1e-5), (gvt.GVT_STAGES_TC_F16X1, 4 * 2.0 ** -11)])
def test_per_tile_training_product_matches_oracle(H, zp, engine, bound):
    p = zp
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    u, st = _product(H, plan, M, N, v, engine, gvt.GVT_TILES_ON)
    rows = np.sort(np.random.default_rng(5).choice(p.n, 300, replace=False))
    ref, mag = _rows_ref(p, rows, v.double().cpu().numpy())
    err = float(np.max(np.abs(u[rows] - ref)) / np.max(np.abs(ref)))
    err_m = float(np.max(np.abs(u[rows] - ref)) / np.max(mag))
    print("engine %d per tile: error %.2e normwise, %.2e of max |K||v|; GEMM %d launches (useful %.2e of "
          "%.2e flops), sparse stage 1 %d, sparse stage 2 %d launches"
          % (engine, err, err_m, st["tc_gemm"]["launches"], st["tc_gemm"]["useful_flops"], st["tc_gemm"]["flops"],
             st["sparse_stage1"]["launches"], st["sparse_stage2"]["launches"]))
    # both parts carry work: the GEMM serves the dense tiles, the SIMT kernels the rest
    assert st["tc_gemm"]["launches"] == 2
    assert st["sparse_stage1"]["launches"] == 1 and st["sparse_stage2"]["launches"] == 1
    assert 0 < st["tc_gemm"]["useful_flops"] < st["stage1"]["flops"] + st["stage2"]["flops"]
    assert 0 < st["sparse_stage1"]["flops"] < st["stage1"]["flops"]
    if engine == gvt.GVT_STAGES_AUTO:
        assert err <= bound
        # the dense engine's product on the same data agrees to FP32 rounding
        ud, _ = _product(H, plan, M, N, v, engine, gvt.GVT_TILES_OFF)
        assert float(np.max(np.abs(u - ud)) / np.max(np.abs(ud))) <= 1e-5
    else:
        assert err_m <= bound
    plan.close()


def test_per_tile_prediction_product_matches_oracle(H, zp):
    """A prediction plan (output pairs = a different Zipf sample over the same ids): stage 2's
    output tiles come from the output pairs' own degrees."""
    p = zp
    q = synth.zipf(4, m=3000, dim=16, n=300_000)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t, q.d, q.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    u, st = _product(H, plan, M, N, v, gvt.GVT_STAGES_AUTO, gvt.GVT_TILES_ON)
    rows = np.sort(np.random.default_rng(6).choice(q.n, 300, replace=False))
    ref, _ = _rows_ref(p, rows, v.double().cpu().numpy(), q.d, q.t)
    err = float(np.max(np.abs(u[rows] - ref)) / np.max(np.abs(ref)))
    print("prediction per tile: error %.2e, GEMM %d launches" % (err, st["tc_gemm"]["launches"]))
    assert st["tc_gemm"]["launches"] == 2
    assert err <= 1e-5
    plan.close()


def test_per_tile_in_a_mixed_solve(H, zp):
    """Mixed-precision refinement whose inner operator runs the per-tile single-pass stages reaches
    the FP64 relative residual 1e-6 (the solver's own FP64 residual; the outer products are FP64)."""
    p = synth.zipf(5, m=3000, dim=16, n=400_000, labels=True)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    gvt.gvt_set_stage_tiles(H.h, gvt.GVT_TILES_ON)
    try:
        a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, torch.as_tensor(p.y, device=DEV), 1.0,
                                       mode=gvt.GVT_SOLVE_MIXED_IR, inner_dtype=gvt.GVT_F16, max_iter=4000)
    finally:
        gvt.gvt_set_stage_tiles(H.h, gvt.GVT_TILES_AUTO)
    print("per-tile single-pass inner: status %d, %d inner iterations, %d refinements, residual %.2e"
          % (st, info.iterations, info.refinements, info.rel_residual))
    assert st == 0 and info.rel_residual <= 1e-6
    rows = np.sort(np.random.default_rng(7).choice(p.n, 200, replace=False))
    Ka, _ = _rows_ref(p, rows, a.cpu().numpy())
    r = p.y[rows] - Ka - a.cpu().numpy()[rows]
    est = float(np.sqrt(p.n * np.mean(r * r)) / np.linalg.norm(p.y))
    print("oracle estimate of the residual on 200 rows: %.2e" % est)
    assert est <= 2e-6
    plan.close()


def test_per_tile_sm_pairs_match_one_sm(H, zp):
    """The block-sparse stage-1 GEMM in the SM-pair form (two CTAs per 256-row tile sharing the N
    tile's k-block list, some lists empty): the per-tile product equals the oracle within the FP32
    tolerance and the one-SM form's product to FP32 rounding."""
    p = zp
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    u1, _ = _product(H, plan, M, N, v, gvt.GVT_STAGES_AUTO, gvt.GVT_TILES_ON)
    gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_ON)
    try:
        u2, st = _product(H, plan, M, N, v, gvt.GVT_STAGES_AUTO, gvt.GVT_TILES_ON)
    finally:
        gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_AUTO)
    rows = np.sort(np.random.default_rng(8).choice(p.n, 300, replace=False))
    ref, _ = _rows_ref(p, rows, v.double().cpu().numpy())
    err = float(np.max(np.abs(u2[rows] - ref)) / np.max(np.abs(ref)))
    diff = float(np.max(np.abs(u2 - u1)) / np.max(np.abs(u1)))
    print("per tile on SM pairs: error %.2e, difference to one SM %.2e" % (err, diff))
    assert st["tc_gemm"]["launches"] == 2
    assert err <= 1e-5 and diff <= 2e-6
    plan.close()


@pytest.mark.parametrize("symmetric", [True, False])
def test_per_tile_single_pass_squared_factors(H, zp, symmetric):
    """One term with squared factors, (M o M) x (N o N), on the single-pass per-tile stages, with
    the kernel matrices passed as symmetric or not (stage 1 then works on B itself or on a
    transposed copy).  Stage 2's sparse remainder reads the dense stages' FP16 operands (entries
    squared before rounding, rows relabelled and scaled by powers of two); the product stays
    within the single-pass bound of the oracle's, 4u of the term magnitudes (u = 2^-11)."""
    p = zp
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=DEV), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    d = gvt.gvt_desc()
    d.kind, d.n_terms, d.homogeneous = -1, 1, 0
    t = d.terms[0]
    t.coef = 1.0
    t.factor_a, t.factor_b = gvt.GVT_FACTOR_M_SQ, gvt.GVT_FACTOR_N_SQ
    t.out_a, t.out_b, t.in_a, t.in_b = gvt.GVT_FIRST, gvt.GVT_SECOND, gvt.GVT_FIRST, gvt.GVT_SECOND
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X1)
    gvt.gvt_set_stage_tiles(H.h, gvt.GVT_TILES_ON)
    gvt.gvt_stats_enable(H.h, True)
    try:
        u = gvt.pairwise_kernel_matvec(plan, d, M, N, v, symmetric=symmetric).double().cpu().numpy()
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
        st = gvt.gvt_stats_read(H.h)
    finally:
        gvt.gvt_stats_enable(H.h, False)
        gvt.gvt_set_stage_tiles(H.h, gvt.GVT_TILES_AUTO)
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    rows = np.sort(np.random.default_rng(9).choice(p.n, 300, replace=False))
    ud, id_ = np.unique(p.d[rows], return_inverse=True)
    ut, it_ = np.unique(p.t[rows], return_inverse=True)
    Mo = orc.gaussian_kernel(p.Xd[ud], p.Xd, gamma=p.gamma) ** 2
    No = orc.gaussian_kernel(p.Xt[ut], p.Xt, gamma=p.gamma) ** 2
    vv = v.double().cpu().numpy()
    ia, it = id_.astype(np.int32), it_.astype(np.int32)
    ref = orc.pairwise_matvec("kronecker", Mo, No, ia, it, p.d, p.t, vv)
    mag = orc.pairwise_matvec("kronecker", Mo, No, ia, it, p.d, p.t, np.abs(vv))
    err_m = float(np.max(np.abs(u[rows] - ref)) / np.max(mag))
    print("squared factors, single pass per tile (symmetric %s): %.2e of max |K||v|; sparse stage 1 %d, "
          "sparse stage 2 %d launches" % (symmetric, err_m, st["sparse_stage1"]["launches"],
                                          st["sparse_stage2"]["launches"]))
    assert st["tc_gemm"]["launches"] == 2
    assert st["sparse_stage1"]["launches"] == 1 and st["sparse_stage2"]["launches"] == 1
    assert err_m <= 4 * 2.0 ** -11
    plan.close()
