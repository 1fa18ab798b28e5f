"""Tensor-core dense stage 1 (tcgen05 BF16 GEMM on hi/lo splits) against references.

* the raw GEMM C = A B^T on BF16 inputs against an FP64 product of the same
  BF16 values (tolerance 1e-5 of max |C|: FP32 accumulation);
* the Kronecker / poly2d products with GVT_STAGE1_TC_BF16X3 against the FP64
  oracle: each product of hi/lo splits is accurate to 3 * 2^-18 relative, so
  the normwise error is bounded by 1.2e-5 * sum|terms| / |u|; the test
  asserts 1e-4 and prints the measured error;
* both stages on the tensor cores with FP16 hi/lo splits of power-of-two
  scaled rows (GVT_STAGES_TC_F16X3), and the cost-model engine
  (GVT_STAGES_AUTO), for all nine kernels on ragged heterogeneous and
  homogeneous samples, training and cross-kernel prediction plans, against the
  FP64 oracle within the FP32 tolerance 1e-5;
* a mixed-precision solve whose inner operator uses the tensor cores reaches
  the FP64 relative residual 1e-6 checked by the oracle;
* the GEMM's two tile forms (one SM per 128-row tile, an SM pair per 256-row
  tile) on the raw GEMM and on the dense engine's products;
* the single-pass FP16 stages (GVT_STAGES_TC_F16X1) within their rounding
  bound, and mixed-precision solves on that inner operator reaching 1e-6.
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


def normwise(u, ref):
    return float(np.max(np.abs(u - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture
def pairs(H, request):
    """Tile form of the tensor-core GEMM for one test; the handle goes back to the default after."""
    gvt.gvt_set_tc_pairs(H.h, request.param)
    yield request.param
    gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_AUTO)


@pytest.mark.parametrize("pairs", [gvt.GVT_TC_PAIRS_OFF, gvt.GVT_TC_PAIRS_ON], indirect=True,
                         ids=["one_sm", "sm_pair"])
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (129, 17, 64), (300, 250, 192), (2000, 250, 6144),
                                   (1000, 1000, 1024), (37, 300, 128), (4000, 100, 512), (640, 2000, 2048),
                                   (2000, 1800, 512), (2000, 2000, 6144)])
def test_tc_gemm_bf16(H, pairs, M, N, K):
    g = torch.Generator(device=DEV).manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, device=DEV).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device=DEV).to(torch.bfloat16)
    C = torch.full((M, N + 3), 7.0, device=DEV)           # ldc > N: padding must stay untouched
    gvt.gvt_tc_gemm_bf16(H.h, gvt.ptr(A), K, gvt.ptr(B), K, gvt.ptr(C), N + 3, M, N, K, gvt.stream_ptr())
    gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    ref = (A.double() @ B.double().T).cpu().numpy()
    c = C.cpu().numpy()
    assert np.all(c[:, N:] == 7.0)
    err = np.max(np.abs(c[:, :N] - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


def _problem(seed=3, m=300, q=80, dim=12, rho=0.25):
    rng = np.random.default_rng(seed)
    Xd, Xt = rng.standard_normal((m, dim)), rng.standard_normal((q, dim))
    n = int(rho * m * q)
    cells = rng.choice(m * q, n, replace=False)
    d, t = (cells // q).astype(np.int32), (cells % q).astype(np.int32)
    return Xd, Xt, d, t, rng.standard_normal(n), 1.0 / dim


@pytest.mark.parametrize("kind", ["kronecker", "poly2d", "symmetric", "mlpk"])
def test_tc_engine_pairwise_parity(H, kind):
    Xd, Xt, d, t, v, g = _problem()
    if kind in gvt.HOMOGENEOUS:
        Xt = Xd
        rng = np.random.default_rng(5)
        d, t = synth.random_pairs(rng, 12000, Xd.shape[0], Xd.shape[0])
        v = rng.standard_normal(len(d))
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g, dtype=torch.float32)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    vv = torch.as_tensor(v, dtype=torch.float32, device=DEV)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_TC_BF16X3)
    try:
        u = gvt.pairwise_kernel_matvec(plan, kind, M, N, vv).double().cpu().numpy()
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    u32 = gvt.pairwise_kernel_matvec(plan, kind, M, N, vv).double().cpu().numpy()
    ref = orc.pairwise_matvec(kind, Mo, No, d, t, d, t, v.astype(np.float32))
    err = normwise(u, ref)
    print("%s: tensor-core stage 1 error vs FP64 %.2e (FP32 SIMT %.2e)" % (kind, err, normwise(u32, ref)))
    assert err <= 1e-4
    plan.close()


def test_mixed_ir_with_tensor_core_inner_operator(H):
    Xd, Xt, d, t, v, g = _problem(seed=4)
    y = np.random.default_rng(6).standard_normal(len(d))
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    lam = 1e-1
    a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, torch.as_tensor(y, device=DEV), lam,
                                   mode=gvt.GVT_SOLVE_MIXED_IR, inner_dtype=gvt.GVT_BF16)
    assert st == 0, (st, info.iterations, info.refinements, info.rel_residual)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    mv = lambda x: orc.pairwise_matvec("kronecker", Mo, No, d, t, d, t, x)
    rr = orc.relative_residual(mv, a.cpu().numpy(), y, lam)
    print("bf16x3 inner: %d inner iterations, %d refinements, oracle residual %.2e"
          % (info.iterations, info.refinements, rr))
    assert rr <= 1.05e-6
    plan.close()


ALL_KINDS = ["kronecker", "gaussian", "linear", "poly2d", "cartesian", "symmetric", "antisymmetric", "ranking",
             "mlpk"]


def _engine_product(H, engine, plan, kind, M, N, v, predict=False):
    gvt.gvt_set_stage1_engine(H.h, engine)
    try:
        f = gvt.predict if predict else gvt.pairwise_kernel_matvec
        u = f(plan, kind, M, N, v).double().cpu().numpy()
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    return u


@pytest.mark.parametrize("engine", [gvt.GVT_STAGES_TC_F16X3, gvt.GVT_STAGES_AUTO])
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_f16x3_stages_meet_the_fp32_tolerance(H, engine, kind):
    """Training product on a ragged sample: 300 x 80 (heterogeneous) or 300 x 300 (homogeneous kernels),
    none of the extents a multiple of the 64-wide split or the 128-row GEMM tile."""
    rng = np.random.default_rng(11)
    m, q, dim = 300, (300 if kind in gvt.HOMOGENEOUS else 80), 12
    Xd = rng.standard_normal((m, dim))
    Xt = Xd if kind in gvt.HOMOGENEOUS else rng.standard_normal((q, dim))
    n = int(0.3 * m * q)
    d, t = synth.random_pairs(rng, n, m, q)
    v = rng.standard_normal(n)
    g = 1.0 / dim
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g, dtype=torch.float32)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    vv = torch.as_tensor(v, dtype=torch.float32, device=DEV)
    u = _engine_product(H, engine, plan, kind, M, N, vv)
    ref = orc.pairwise_matvec(kind, Mo, No, d, t, d, t, vv.double().cpu().numpy())
    err = normwise(u, ref)
    print("%s engine %d: error vs FP64 %.2e" % (kind, engine, err))
    assert err <= 1e-5
    plan.close()


@pytest.mark.parametrize("kind", ["kronecker", "symmetric", "mlpk"])
def test_sm_pair_tiles_agree_with_single_sm_tiles(H, kind):
    """The dense engine with 256-row SM-pair tiles and with 128-row one-SM tiles: both meet the FP32
    tolerance against the FP64 oracle and agree with each other to FP32 rounding (ragged 430 x 430 or
    430 x 150: two pairs, the second with a partly empty odd half)."""
    rng = np.random.default_rng(21)
    m, q, dim = 430, (430 if kind in gvt.HOMOGENEOUS else 150), 12
    Xd = rng.standard_normal((m, dim))
    Xt = Xd if kind in gvt.HOMOGENEOUS else rng.standard_normal((q, dim))
    d, t = synth.random_pairs(rng, int(0.3 * m * q), m, q)
    v = rng.standard_normal(len(d))
    g = 1.0 / dim
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g, dtype=torch.float32)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    vv = torch.as_tensor(v, dtype=torch.float32, device=DEV)
    ref = orc.pairwise_matvec(kind, orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g),
                              d, t, d, t, vv.double().cpu().numpy())
    out = {}
    try:
        for mode in (gvt.GVT_TC_PAIRS_OFF, gvt.GVT_TC_PAIRS_ON):
            gvt.gvt_set_tc_pairs(H.h, mode)
            out[mode] = _engine_product(H, gvt.GVT_STAGES_TC_F16X3, plan, kind, M, N, vv)
    finally:
        gvt.gvt_set_tc_pairs(H.h, gvt.GVT_TC_PAIRS_AUTO)
    e1, e2 = normwise(out[gvt.GVT_TC_PAIRS_OFF], ref), normwise(out[gvt.GVT_TC_PAIRS_ON], ref)
    diff = normwise(out[gvt.GVT_TC_PAIRS_ON], out[gvt.GVT_TC_PAIRS_OFF])
    print("%s: one SM %.2e, SM pair %.2e, between them %.2e" % (kind, e1, e2, diff))
    assert e1 <= 1e-5 and e2 <= 1e-5
    assert diff <= 2e-6
    plan.close()


@pytest.mark.parametrize("kind", ["kronecker", "linear", "cartesian", "mlpk"])
def test_f16x3_cross_kernel_prediction(H, kind):
    """Prediction for pairs of unseen objects: M_pred (mbar x m) and N_pred (qbar x q) rectangular."""
    rng = np.random.default_rng(12)
    homo = kind in gvt.HOMOGENEOUS
    m, q, mb, qb, dim = 260, (260 if homo else 130), 70, (70 if homo else 90), 10
    Xd, Xdn = rng.standard_normal((m, dim)), rng.standard_normal((mb, dim))
    Xt, Xtn = (Xd, Xdn) if homo else (rng.standard_normal((q, dim)), rng.standard_normal((qb, dim)))
    g = 1.0 / dim
    n, nh = int(0.35 * m * q), 3000
    d, t = synth.random_pairs(rng, n, m, q)
    dh, th = rng.integers(0, mb, nh).astype(np.int32), rng.integers(0, qb, nh).astype(np.int32)
    if kind == "cartesian":   # identity factors need one id space: predict on training objects
        mb, qb, Xdn, Xtn = m, q, Xd, Xt
        dh, th = rng.integers(0, m, nh).astype(np.int32), rng.integers(0, q, nh).astype(np.int32)
    Mp = gvt.gaussian_kernel(H, torch.as_tensor(Xdn, device=DEV), torch.as_tensor(Xd, device=DEV), gamma=g,
                             dtype=torch.float32)
    Np = gvt.gaussian_kernel(H, torch.as_tensor(Xtn, device=DEV), torch.as_tensor(Xt, device=DEV), gamma=g,
                             dtype=torch.float32)
    Mo = orc.gaussian_kernel(Xdn, Xd, gamma=g)
    No = orc.gaussian_kernel(Xtn, Xt, gamma=g)
    plan = gvt.Plan(H, tuple(Mp.shape), tuple(Np.shape), d, t, dh, th)
    a = rng.standard_normal(n)
    aa = torch.as_tensor(a, dtype=torch.float32, device=DEV)
    u = _engine_product(H, gvt.GVT_STAGES_TC_F16X3, plan, kind, Mp, Np, aa, predict=True)
    ref = orc.pairwise_matvec(kind, Mo, No, dh, th, d, t, aa.double().cpu().numpy())
    err = normwise(u, ref)
    print("%s prediction, FP16x3 stages: error vs FP64 %.2e" % (kind, err))
    assert err <= 1e-5
    plan.close()


def test_auto_engine_on_a_dense_sample_and_mixed_solve(H):
    """A dense homogeneous sample (600 objects, 28 % of the pairs), where the cost model picks the
    tensor-core stages, and a mixed-precision solve whose inner FP32 operator runs under that engine."""
    rng = np.random.default_rng(13)
    m, dim = 600, 16
    X = rng.standard_normal((m, dim))
    g = 1.0 / dim
    n = 100000
    d, t = synth.random_pairs(rng, n, m, m)
    M32 = gvt.gaussian_kernel(H, torch.as_tensor(X, device=DEV), gamma=g, dtype=torch.float32)
    M64 = gvt.gaussian_kernel(H, torch.as_tensor(X, device=DEV), gamma=g)
    Mo = orc.gaussian_kernel(X, gamma=g)
    plan = gvt.Plan(H, tuple(M32.shape), tuple(M32.shape), d, t)
    v = rng.standard_normal(n)
    u = _engine_product(H, gvt.GVT_STAGES_AUTO, plan, "kronecker", M32, M32,
                        torch.as_tensor(v, dtype=torch.float32, device=DEV))
    rows = rng.choice(n, 200, replace=False)
    ref = orc.pairwise_matvec("kronecker", Mo, Mo, d[rows], t[rows], d, t, v.astype(np.float32).astype(np.float64))
    err = float(np.max(np.abs(u[rows] - ref)) / np.max(np.abs(ref)))
    print("auto engine, dense sample: error vs FP64 on 200 sampled rows %.2e" % err)
    assert err <= 1e-5
    y = rng.standard_normal(n)
    lam = 1e-1
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_AUTO)
    try:
        a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M64, M64, torch.as_tensor(y, device=DEV), lam,
                                       mode=gvt.GVT_SOLVE_MIXED_IR)
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    assert st == 0
    # the FP64 residual of the returned solution, recomputed on sampled rows by the oracle
    Ka = orc.pairwise_matvec("kronecker", Mo, Mo, d[rows], t[rows], d, t, a.cpu().numpy())
    r = y[rows] - Ka - lam * a.cpu().numpy()[rows]
    print("auto engine mixed solve: %d inner iterations, %d refinements, reported residual %.2e, "
          "sampled-row residual max %.2e" % (info.iterations, info.refinements, info.rel_residual,
                                             np.max(np.abs(r))))
    assert info.rel_residual <= 1e-6
    assert np.max(np.abs(r)) <= 1e-5 * np.max(np.abs(y))
    plan.close()


def test_split_copies_do_not_outlive_a_solve(H):
    """A solve keeps split copies of its kernel matrices across its products; a later solve on
    other matrices in the same workspace must not see them (it converges as on a fresh handle)."""
    rng = np.random.default_rng(21)
    m, q, dim = 300, 160, 12
    n = int(0.3 * m * q)
    d, t = synth.random_pairs(rng, n, m, q)
    y = rng.standard_normal(n)
    lam = 1e-1
    runs = []
    for scale in (1.0, 0.5):
        Xd, Xt = scale * rng.standard_normal((m, dim)), rng.standard_normal((q, dim))
        M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=1.0 / dim)
        N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=1.0 / dim)
        runs.append((Xd, Xt, M, N))
    plan = gvt.Plan(H, (m, m), (q, q), d, t)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X3)
    try:
        its = []
        for Xd, Xt, M, N in runs:
            a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, torch.as_tensor(y, device=DEV), lam,
                                           mode=gvt.GVT_SOLVE_MIXED_IR)
            assert st == 0
            Mo, No = orc.gaussian_kernel(Xd, gamma=1.0 / dim), orc.gaussian_kernel(Xt, gamma=1.0 / dim)
            mv = lambda x: orc.pairwise_matvec("kronecker", Mo, No, d, t, d, t, x)
            assert orc.relative_residual(mv, a.cpu().numpy(), y, lam) <= 1.05e-6
            its.append((info.iterations, info.refinements))
        H2 = gvt.Handle()
        gvt.gvt_set_stage1_engine(H2.h, gvt.GVT_STAGES_TC_F16X3)
        plan2 = gvt.Plan(H2, (m, m), (q, q), d, t)
        _, st, info2 = gvt.krr_cg_solve(H2, plan2, "kronecker", runs[1][2], runs[1][3],
                                        torch.as_tensor(y, device=DEV), lam, mode=gvt.GVT_SOLVE_MIXED_IR)
        print("second solve: %d inner iterations, %d refinements; on a fresh handle %d, %d"
              % (its[1][0], its[1][1], info2.iterations, info2.refinements))
        # a stale split of the first matrices would turn every inner solve into one for the wrong
        # operator (more refinements or no convergence); split-K rounding order moves counts a little
        assert st == 0 and info2.refinements == its[1][1]
        assert abs(info2.iterations - its[1][0]) <= 0.25 * info2.iterations + 3
        plan2.close()
        H2.close()
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    plan.close()


def test_dense_engine_is_reproducible_without_split_k(H):
    """The FP16x3 stages at the benchmark shape (2000 x 2000 GEMMs, no K split): MLPK -- whose
    same-component terms sum whole segments into one W cell -- gives bit-identical results on
    repeated runs."""
    p = synth.homogeneous(0)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=DEV), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.m, p.m), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X3)
    try:
        outs = [gvt.pairwise_kernel_matvec(plan, "mlpk", M, M, v).clone() for _ in range(3)]
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    plan.close()


def test_factor_cache_scope_reuses_splits_and_keys_by_matrix(H):
    """Inside gvt_factor_cache_begin/end the dense engine reuses split copies of the kernel matrices
    across products. At the benchmark shape (no K split) the products are bit-identical to those
    made without the scope. A second matrix with another pointer, used inside the same scope, gets
    its own split: its product matches the one made outside the scope. Ending a scope that is not
    open is an argument error."""
    p = synth.homogeneous(0)
    X = torch.as_tensor(p.Xd, device=DEV)
    M1 = gvt.gaussian_kernel(H, X, gamma=p.gamma, dtype=torch.float32)
    M2 = gvt.gaussian_kernel(H, X, gamma=2 * p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.m, p.m), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=DEV)
    kinds = ["kronecker", "symmetric", "mlpk"]
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X3)
    try:
        ref = {(k, i): gvt.pairwise_kernel_matvec(plan, k, Mx, Mx, v).clone()
               for k in kinds for i, Mx in enumerate((M1, M2))}
        gvt.gvt_factor_cache_begin(H.h)
        try:
            got = {(k, i): gvt.pairwise_kernel_matvec(plan, k, Mx, Mx, v).clone()
                   for k in kinds for i, Mx in enumerate((M1, M2))}
            again = gvt.pairwise_kernel_matvec(plan, "mlpk", M1, M1, v).clone()
        finally:
            gvt.gvt_factor_cache_end(H.h)
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    for key in ref:
        assert torch.equal(ref[key], got[key]), key
    assert torch.equal(again, ref[("mlpk", 0)])
    assert not torch.equal(ref[("kronecker", 0)], ref[("kronecker", 1)])
    with pytest.raises(gvt.GvtError):
        gvt.gvt_factor_cache_end(H.h)
    plan.close()


@pytest.mark.parametrize("kind", ["kronecker", "gaussian", "poly2d", "cartesian", "symmetric"])
def test_single_pass_f16_stages_within_their_rounding_bound(H, kind):
    """GVT_STAGES_TC_F16X1: the dense stages as one tcgen05 pass over FP16 hi parts of power-of-two
    scaled rows.  Each operand entry is rounded once to FP16 (unit roundoff u = 2^-11) in stage 1
    (N or M and W) and once more in stage 2 (A and S), so each term of u_i is off by at most about
    4u of its magnitude: |u_i - u*_i| <= 4u (|K||v|)_i plus FP32 accumulation.  These kernels have
    nonnegative formulas on Gaussian bases, so |K| = K and (|K||v|)_i is the oracle's product with
    |v|.  The test asserts 8u (a factor 2 of margin) on 300 sampled rows of a sample dense and
    large enough (1000 x 600 or 1000 x 1000 objects, 30 % of the pairs) that the cost model picks
    the tensor cores (checked through the library's GEMM statistics)."""
    rng = np.random.default_rng(17)
    m, q, dim = 1000, (1000 if kind in gvt.HOMOGENEOUS else 600), 12
    Xd = rng.standard_normal((m, dim))
    Xt = Xd if kind in gvt.HOMOGENEOUS else rng.standard_normal((q, dim))
    n = int(0.3 * m * q)
    d, t = synth.random_pairs(rng, n, m, q)
    v = rng.standard_normal(n)
    g = 1.0 / dim
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g, dtype=torch.float32)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g, dtype=torch.float32)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    vv = torch.as_tensor(v, dtype=torch.float32, device=DEV)
    gvt.gvt_stats_enable(H.h, True)
    u = _engine_product(H, gvt.GVT_STAGES_TC_F16X1, plan, kind, M, N, vv)
    stats = gvt.gvt_stats_read(H.h)
    gvt.gvt_stats_enable(H.h, False)
    v64 = vv.double().cpu().numpy()
    rows = np.sort(rng.choice(n, 300, replace=False))
    ref = orc.pairwise_matvec(kind, Mo, No, d[rows], t[rows], d, t, v64)
    mag = orc.pairwise_matvec(kind, Mo, No, d[rows], t[rows], d, t, np.abs(v64))
    u = u[rows]
    err = float(np.max(np.abs(u - ref)) / np.max(mag))
    print("%s single-pass FP16 stages: error %.2e of max |K||v| (normwise %.2e), %d GEMM launches"
          % (kind, err, normwise(u, ref), stats["tc_gemm"]["launches"]))
    assert stats["tc_gemm"]["launches"] > 0
    assert err <= 8 * 2.0 ** -11
    plan.close()


@pytest.mark.parametrize("lam", [1e-1, 1e-2])
def test_mixed_ir_with_single_pass_f16_inner_operator(H, lam):
    """Mixed-precision refinement whose inner FP32 CG runs on the single-pass FP16 tensor-core
    stages (inner_dtype = GVT_F16) reaches the FP64 relative residual 1e-6, recomputed by the
    oracle over all pairs."""
    Xd, Xt, d, t, v, g = _problem(seed=4, rho=0.4)
    y = np.random.default_rng(6).standard_normal(len(d))
    M = gvt.gaussian_kernel(H, torch.as_tensor(Xd, device=DEV), gamma=g)
    N = gvt.gaussian_kernel(H, torch.as_tensor(Xt, device=DEV), gamma=g)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t)
    a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, torch.as_tensor(y, device=DEV), lam,
                                   mode=gvt.GVT_SOLVE_MIXED_IR, inner_dtype=gvt.GVT_F16, max_iter=20000)
    Mo, No = orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g)
    mv = lambda x: orc.pairwise_matvec("kronecker", Mo, No, d, t, d, t, x)
    rr = orc.relative_residual(mv, a.cpu().numpy(), y, lam)
    print("single-pass FP16 inner, lambda %g: status %d, %d inner iterations, %d refinements, oracle residual %.2e"
          % (lam, st, info.iterations, info.refinements, rr))
    assert st == 0, (st, info.iterations, info.refinements, info.rel_residual)
    assert rr <= 1.05e-6
    plan.close()
