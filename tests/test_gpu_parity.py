"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (normwise, ||u - u*||_inf / ||u*||_inf): 1e-10 for FP64 results,
1e-5 for FP32 results.  Inputs are the seeded synthetic workloads; both sides
build their Gaussian base kernels from the same features.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2009_01054_gb300 import gvt, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}
KINDS = list(gvt.KERNELS)
DEV = "cuda"


def normwise(u, ref):
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(u - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture(scope="module")
def H():
    from paper_2009_01054_gb300 import build
    build.build()
    h = gvt.Handle()
    yield h
    h.close()


def to_dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def gpu_gauss(H, X, gamma, dtype, Y=None):
    return gvt.gaussian_kernel(H, to_dev(X), None if Y is None else to_dev(Y), gamma, dtype=dtype)


def problem_kernels(H, p, dtype):
    M = gpu_gauss(H, p.Xd, p.gamma, dtype)
    N = M if p.homogeneous else gpu_gauss(H, p.Xt, p.gamma, dtype)
    return M, N


def oracle_kernels(p):
    M = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    N = M if p.homogeneous else orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    return M, N


def run(H, kind, M, N, d_in, t_in, v, d_out=None, t_out=None, symmetric=True, m_shape=None, q_shape=None):
    m_shape = m_shape or tuple(M.shape)
    q_shape = q_shape or (tuple(M.shape) if N is None else tuple(N.shape))
    plan = gvt.Plan(H, m_shape, q_shape, d_in, t_in, d_out, t_out)
    u = gvt.pairwise_kernel_matvec(plan, kind, M, None if kind in gvt.HOMOGENEOUS else N,
                                   to_dev(v, M.dtype), symmetric=symmetric)
    torch.cuda.synchronize()
    out = u.double().cpu().numpy()
    plan.close()
    return out


def test_gaussian_base_kernel(H):
    p = synth.small(0)
    Mg = gpu_gauss(H, p.Xd, p.gamma, torch.float64).cpu().numpy()
    Mo = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    np.testing.assert_allclose(Mg, Mo, rtol=1e-13, atol=1e-15)
    Xc = np.random.default_rng(1).standard_normal((33, 16))
    Kc = gpu_gauss(H, p.Xd, p.gamma, torch.float64, Y=Xc).cpu().numpy()
    np.testing.assert_allclose(Kc, orc.gaussian_kernel(p.Xd, Xc, gamma=p.gamma), rtol=1e-13, atol=1e-15)
    K32 = gpu_gauss(H, p.Xd, p.gamma, torch.float32).cpu().numpy()
    assert np.array_equal(K32, Mo.astype(np.float32)) or np.max(np.abs(K32 - Mo)) < 1e-7


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_kronecker_small_train_and_predict(H, dtype):
    p = synth.small(0)
    M, N = problem_kernels(H, p, dtype)
    Mo, No = oracle_kernels(p)
    u = run(H, "kronecker", M, N, p.d, p.t, p.v)
    ref = orc.pairwise_matvec("kronecker", Mo, No, p.d, p.t, p.d, p.t, p.v)
    assert normwise(u, ref) <= TOL[dtype]
    up = run(H, "kronecker", M, N, p.d, p.t, p.v, p.d_pred, p.t_pred)
    refp = orc.pairwise_matvec("kronecker", Mo, No, p.d_pred, p.t_pred, p.d, p.t, p.v)
    assert normwise(up, refp) <= TOL[dtype]


def _mixed_problem(kind, seed=5, m=150, q=70, n=3000, n_out=1700):
    rng = np.random.default_rng(seed)
    q = m if kind in gvt.HOMOGENEOUS else q
    Xd = rng.standard_normal((m, 8))
    Xt = Xd if kind in gvt.HOMOGENEOUS else rng.standard_normal((q, 8))
    d, t = synth.random_pairs(rng, n, m, q)
    do, to = synth.random_pairs(rng, n_out, m, q)
    v = rng.standard_normal(n)
    return Xd, Xt, d, t, do, to, v, 1.0 / 8


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", KINDS)
def test_every_kernel_small_ragged(H, kind, dtype):
    """Ragged shapes (150 x 70 ids, 3000 pairs with repeats), prediction pairs != training pairs."""
    Xd, Xt, d, t, do, to, v, g = _mixed_problem(kind)
    M = gpu_gauss(H, Xd, g, dtype)
    N = gpu_gauss(H, Xt, g, dtype)
    Mo = orc.gaussian_kernel(Xd, gamma=g)
    No = orc.gaussian_kernel(Xt, gamma=g)
    u = run(H, kind, M, N, d, t, v, do, to)
    ref = orc.pairwise_matvec(kind, Mo, No, do, to, d, t, v)
    assert normwise(u, ref) <= TOL[dtype], kind
    ut = run(H, kind, M, N, d, t, v)
    reft = orc.pairwise_matvec(kind, Mo, No, d, t, d, t, v)
    assert normwise(ut, reft) <= TOL[dtype], kind


def test_multiple_columns(H):
    Xd, Xt, d, t, do, to, v, g = _mixed_problem("poly2d", n=1000, n_out=600)
    V = np.random.default_rng(3).standard_normal((1000, 3))
    M = gpu_gauss(H, Xd, g, torch.float64)
    N = gpu_gauss(H, Xt, g, torch.float64)
    plan = gvt.Plan(H, tuple(M.shape), tuple(N.shape), d, t, do, to)
    U = gvt.pairwise_kernel_matvec(plan, "poly2d", M, N, to_dev(V)).cpu().numpy()
    ref = orc.pairwise_matvec("poly2d", orc.gaussian_kernel(Xd, gamma=g), orc.gaussian_kernel(Xt, gamma=g),
                              do, to, d, t, V)
    assert normwise(U, ref) <= 1e-10


def test_cross_kernel_prediction_nonsymmetric(H):
    """Rectangular cross kernels (new drugs and targets, Setting 4) exercise the transpose path."""
    rng = np.random.default_rng(8)
    Xd, Xt = rng.standard_normal((90, 6)), rng.standard_normal((40, 6))
    Xd2, Xt2 = rng.standard_normal((25, 6)), rng.standard_normal((17, 6))
    g = 1.0 / 6
    d, t = synth.random_pairs(rng, 700, 90, 40)
    do, to = synth.random_pairs(rng, 300, 25, 17)
    v = rng.standard_normal(700)
    for kind in ["kronecker", "linear", "poly2d"]:
        Mx = gpu_gauss(H, Xd2, g, torch.float64, Y=Xd)
        Nx = gpu_gauss(H, Xt2, g, torch.float64, Y=Xt)
        plan = gvt.Plan(H, (25, 90), (17, 40), d, t, do, to)
        u = gvt.predict(plan, kind, Mx, Nx, to_dev(v)).cpu().numpy()
        ref = orc.pairwise_matvec(kind, orc.gaussian_kernel(Xd2, Xd, gamma=g),
                                  orc.gaussian_kernel(Xt2, Xt, gamma=g), do, to, d, t, v)
        assert normwise(u, ref) <= 1e-10, kind


def test_edge_cases(H):
    rng = np.random.default_rng(9)
    m, q = 37, 29
    Xd, Xt = rng.standard_normal((m, 4)), rng.standard_normal((q, 4))
    M = gpu_gauss(H, Xd, 0.25, torch.float64)
    N = gpu_gauss(H, Xt, 0.25, torch.float64)
    Mo, No = orc.gaussian_kernel(Xd, gamma=0.25), orc.gaussian_kernel(Xt, gamma=0.25)
    # no input pairs: u = 0
    do, to = synth.random_pairs(rng, 10, m, q)
    u = run(H, "kronecker", M, N, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), do, to)
    assert np.all(u == 0) and u.shape == (10,)
    # one pair
    u = run(H, "mlpk", M, None, np.array([3], np.int32), np.array([5], np.int32), np.array([2.0]),
            np.array([1, 5], np.int32), np.array([2, 3], np.int32), m_shape=(m, m), q_shape=(m, m))
    ref = orc.pairwise_matvec("mlpk", Mo, None, [1, 5], [2, 3], [3], [5], [2.0])
    assert normwise(u, ref) <= 1e-10
    # every pair in one drug column (one long segment), 33 outputs (ragged warp tail)
    d = np.zeros(5000, np.int32)
    t = rng.integers(0, q, 5000).astype(np.int32)
    v = rng.standard_normal(5000)
    do, to = synth.random_pairs(rng, 33, m, q)
    for kind in ["kronecker", "cartesian", "linear"]:
        u = run(H, kind, M, N, d, t, v, do, to)
        ref = orc.pairwise_matvec(kind, Mo, No, do, to, d, t, v)
        assert normwise(u, ref) <= 1e-10, kind


def test_index_out_of_bounds_is_rejected(H):
    d = torch.tensor([0, 4, 2], dtype=torch.int32, device=DEV)
    t = torch.tensor([1, 1, 3], dtype=torch.int32, device=DEV)
    with pytest.raises(gvt.GvtError) as e:
        gvt.Plan(H, (4, 4), (5, 5), d, t)
    assert e.value.status == 2 and "d_in" in str(e.value)
    with pytest.raises(gvt.GvtError) as e:
        gvt.Plan(H, (4, 4), (5, 5), t, t, torch.tensor([0], dtype=torch.int32, device=DEV),
                 torch.tensor([-1], dtype=torch.int32, device=DEV))
    assert e.value.status == 2


def test_results_are_bitwise_reproducible(H):
    Xd, Xt, d, t, do, to, v, g = _mixed_problem("mlpk", n=4000)
    M = gpu_gauss(H, Xd, g, torch.float32)
    u1 = run(H, "mlpk", M, None, d, t, v, do, to)
    u2 = run(H, "mlpk", M, None, d, t, v, do, to)
    assert np.array_equal(u1, u2)


@pytest.mark.slow
@pytest.mark.parametrize("engine", [gvt.GVT_STAGE1_SIMT, gvt.GVT_STAGES_AUTO])
def test_full_size_homogeneous_all_kernels_sampled(H, engine):
    """m = q = 2000, n = 200k (the benchmark workload), FP32 on the GPU on the SIMT engine and
    on the automatic engine the benchmark times (dense tensor-core stages at this density),
    256 sampled outputs checked against the FP64 oracle (each against all 200k inputs)."""
    p = synth.homogeneous(0)
    M = gpu_gauss(H, p.Xd, p.gamma, torch.float32)
    Mo = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.m, p.m), p.d, p.t)
    v = to_dev(p.v, torch.float32)
    idx = np.random.default_rng(0).choice(p.n, 256, replace=False)
    gvt.gvt_set_stage1_engine(H.h, engine)
    try:
        for kind in KINDS:
            u = gvt.pairwise_kernel_matvec(plan, kind, M, M, v).double().cpu().numpy()
            ref = orc.pairwise_matvec(kind, Mo, Mo, p.d[idx], p.t[idx], p.d, p.t, p.v.astype(np.float32))
            assert normwise(u[idx], ref) <= 1e-5, kind
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    plan.close()


def test_dense_engine_edge_cases(H):
    """The FP16x3 tensor-core stages on degenerate inputs: no input pairs, one pair, all pairs in
    one column, repeated pairs, id ranges below one 64-wide split block."""
    rng = np.random.default_rng(19)
    m, q = 37, 29
    Xd, Xt = rng.standard_normal((m, 4)), rng.standard_normal((q, 4))
    M = gpu_gauss(H, Xd, 0.25, torch.float32)
    N = gpu_gauss(H, Xt, 0.25, torch.float32)
    Mo, No = orc.gaussian_kernel(Xd, gamma=0.25), orc.gaussian_kernel(Xt, gamma=0.25)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_TC_F16X3)
    try:
        do, to = synth.random_pairs(rng, 10, m, q)
        u = run(H, "kronecker", M, N, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), do, to)
        assert np.all(u == 0) and u.shape == (10,)
        u = run(H, "mlpk", M, None, np.array([3], np.int32), np.array([5], np.int32), np.array([2.0]),
                np.array([1, 5], np.int32), np.array([2, 3], np.int32), m_shape=(m, m), q_shape=(m, m))
        ref = orc.pairwise_matvec("mlpk", Mo, None, [1, 5], [2, 3], [3], [5], np.float32([2.0]))
        assert normwise(u, ref) <= 1e-5
        d = np.zeros(5000, np.int32)                       # one drug column
        t = rng.integers(0, q, 5000).astype(np.int32)      # many repeated pairs
        v = rng.standard_normal(5000).astype(np.float32)
        do, to = synth.random_pairs(rng, 33, m, q)
        for kind in ["kronecker", "cartesian", "linear", "poly2d"]:
            u = run(H, kind, M, N, d, t, v, do, to)
            ref = orc.pairwise_matvec(kind, Mo, No, do, to, d, t, v.astype(np.float64))
            assert normwise(u, ref) <= 1e-5, kind
        gvt.gvt_check_device_errors(H.h, gvt.stream_ptr())
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)


@pytest.mark.parametrize("kind", ["kronecker", "symmetric", "poly2d"])
@pytest.mark.parametrize("mode", [gvt.GVT_SOLVE_FP64_CG, gvt.GVT_SOLVE_MIXED_IR])
def test_krr_solve_small_matches_cholesky(H, kind, mode):
    p = synth.small(0) if kind not in gvt.HOMOGENEOUS else synth.homogeneous(0, m=64, n=1000)
    M, N = problem_kernels(H, p, torch.float64)
    Mo, No = oracle_kernels(p)
    lam = 1e-2
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    a, st, info = gvt.krr_cg_solve(H, plan, kind, M, N, to_dev(p.y), lam, mode=mode, rel_tol=1e-8)
    assert st == 0, (st, info.iterations)
    a = a.cpu().numpy()
    K = orc.kernel_matrix(kind, Mo, No, p.d, p.t, p.d, p.t)
    a_ref = orc.krr_solve_dense(K, p.y, lam)
    mv = lambda x: orc.pairwise_matvec(kind, Mo, No, p.d, p.t, p.d, p.t, x)
    assert orc.relative_residual(mv, a, p.y, lam) <= 1e-8 * 1.01 + 1e-12
    assert info.rel_residual <= 1e-8
    assert normwise(a, a_ref) <= 1e-5   # (K + lam I)^-1 amplifies the 1e-8 residual
    plan.close()


def test_solve_then_predict(H):
    p = synth.small(0)
    M, N = problem_kernels(H, p, torch.float64)
    Mo, No = oracle_kernels(p)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, to_dev(p.y), 1e-2)
    assert st == 0 and info.rel_residual <= 1e-6
    pp = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t, p.d_pred, p.t_pred)
    pred = gvt.predict(pp, "kronecker", M, N, a, symmetric=True).cpu().numpy()
    ref = orc.pairwise_matvec("kronecker", Mo, No, p.d_pred, p.t_pred, p.d, p.t, a.cpu().numpy())
    assert normwise(pred, ref) <= 1e-10


def test_solve_reports_not_converged_and_warm_start_resumes(H):
    p = synth.small(0)
    M, N = problem_kernels(H, p, torch.float64)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    y = to_dev(p.y)
    a5, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, y, 1e-3, max_iter=5)
    assert st == 7 and info.iterations == 5
    a, st, info2 = gvt.krr_cg_solve(H, plan, "kronecker", M, N, y, 1e-3, a0=a5)
    assert st == 0 and info2.rel_residual <= 1e-6


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["kronecker", "poly2d", "symmetric", "mlpk", "cartesian"])
def test_tall_tiles_medium(H, kind, dtype):
    """m = q = 900 ids (stage-1 tiles of 1024 rows, partly empty), 20k pairs, every output checked."""
    rng = np.random.default_rng(17)
    m = 900
    X = rng.standard_normal((m, 10))
    d, t = synth.random_pairs(rng, 20000, m, m)
    v = rng.standard_normal(20000)
    M = gpu_gauss(H, X, 0.1, dtype)
    Mo = orc.gaussian_kernel(X, gamma=0.1)
    u = run(H, kind, M, M, d, t, v)
    ref = orc.pairwise_matvec(kind, Mo, Mo, d, t, d, t, v)
    assert normwise(u, ref) <= TOL[dtype], kind


def test_tanimoto_base_kernel_and_product(H):
    """Tanimoto kernel of bit-packed fingerprints (Sec. 5) against the oracle: FP64 bit-exact (a
    ratio of integers rounded once), FP32 the rounded FP64 value, rectangular and ragged; then a
    Kronecker product with a Tanimoto drug kernel and a Gaussian target kernel."""
    rng = np.random.default_rng(41)
    bits_a, pa = synth.fingerprints(rng, 300, 167, 0.15)
    bits_b, pb = synth.fingerprints(rng, 220, 167, 0.15)
    bits_a[5] = 0
    pa[5] = 0
    Xa = torch.as_tensor(pa.view(np.int32), device=DEV)
    Xb = torch.as_tensor(pb.view(np.int32), device=DEV)
    K = gvt.tanimoto_kernel(H, Xa, Xb).cpu().numpy()
    Ko = orc.tanimoto_kernel(bits_a, bits_b)
    assert np.array_equal(K, Ko)
    K32 = gvt.tanimoto_kernel(H, Xa, Xb, dtype=torch.float32).cpu().numpy()
    assert np.array_equal(K32, Ko.astype(np.float32))
    Mt = gvt.tanimoto_kernel(H, Xa)
    Mo = orc.tanimoto_kernel(bits_a)
    assert np.array_equal(Mt.cpu().numpy(), Mo)
    Xt = rng.standard_normal((40, 6))
    N = gpu_gauss(H, Xt, 1.0 / 6, torch.float64)
    No = orc.gaussian_kernel(Xt, gamma=1.0 / 6)
    d, t = synth.random_pairs(rng, 3000, 300, 40)
    v = rng.standard_normal(3000)
    do, to = synth.random_pairs(rng, 500, 300, 40)
    u = run(H, "kronecker", Mt, N, d, t, v, do, to)
    ref = orc.pairwise_matvec("kronecker", Mo, No, do, to, d, t, v)
    assert normwise(u, ref) <= 1e-10


def test_linear_base_kernel_on_similarity_rows_and_product(H):
    """Linear kernel on the rows of a symmetric similarity matrix (Sec. 5, Metz) against the oracle:
    FP64 within 1e-13 of max |K| (the GPU sums in another order), FP32 and BF16 the rounded values;
    ragged (131 rows, 131-d) and rectangular (new rows against training rows); then a Kronecker
    product with a linear drug kernel and a linear target kernel against the oracle."""
    rng = np.random.default_rng(43)
    A = rng.uniform(0.0, 1.0, (131, 131))
    Sd = (A + A.T) / 2
    np.fill_diagonal(Sd, 1.0)
    X = torch.as_tensor(Sd, device=DEV)
    K = gvt.linear_kernel(H, X).cpu().numpy()
    Ko = orc.linear_kernel(Sd)
    assert np.max(np.abs(K - Ko)) <= 1e-13 * np.max(np.abs(Ko))
    Xn = rng.uniform(0.0, 1.0, (37, 131))
    Kx = gvt.linear_kernel(H, torch.as_tensor(Xn, device=DEV), X).cpu().numpy()
    Kxo = orc.linear_kernel(Xn, Sd)
    assert Kx.shape == (37, 131) and np.max(np.abs(Kx - Kxo)) <= 1e-13 * np.max(np.abs(Kxo))
    K32 = gvt.linear_kernel(H, X, dtype=torch.float32).cpu().numpy()
    assert np.max(np.abs(K32 - Ko) / np.abs(Ko)) <= 2 ** -24 * 1.0001   # one rounding of the FP64 sum
    K16 = gvt.linear_kernel(H, X, dtype=torch.bfloat16).float().cpu().numpy()
    assert np.max(np.abs(K16 - Ko) / np.abs(Ko)) <= 2 ** -8 * 1.0001
    B = rng.uniform(0.0, 1.0, (45, 45))
    St = (B + B.T) / 2
    Mg = gvt.linear_kernel(H, X)
    Ng = gvt.linear_kernel(H, torch.as_tensor(St, device=DEV))
    d, t = synth.random_pairs(rng, 2500, 131, 45)
    v = rng.standard_normal(2500)
    u = run(H, "kronecker", Mg, Ng, d, t, v, d, t)
    ref = orc.pairwise_matvec("kronecker", Ko, orc.linear_kernel(St), d, t, d, t, v)
    assert normwise(u, ref) <= 1e-10
    E = gvt.linear_kernel(H, X[:0], X)
    assert E.shape == (0, 131)
