"""Python binding of the C ABI in ``include/gvt.h`` (argument marshalling only).

The raw functions carry the ABI names (``gvt_create``, ``gvt_plan_create``,
``gvt_matvec``, ``gvt_pairwise_kernel_matvec``, ``gvt_krr_cg_solve``,
``gvt_predict`` ...) and raise :class:`GvtError` on a non-zero status.  The
small classes below (:class:`Handle`, :class:`Plan`) only turn torch tensors
into device pointers and streams.  Every step of the computation runs in
``libgvt.so``; there is no fallback: importing works without the library, the
first call raises if it is missing.
"""
import ctypes
import os

from . import build as _build

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

# ---------------------------------------------------------------- enums (gvt.h)
GVT_OK = 0
GVT_ERR_INVALID_ARG, GVT_ERR_INDEX_OOB, GVT_ERR_UNSUPPORTED, GVT_ERR_ALLOC, GVT_ERR_CUDA = 1, 2, 3, 4, 5
GVT_ERR_BREAKDOWN, GVT_ERR_NOT_CONVERGED, GVT_ERR_TIMEOUT = 6, 7, 8
STATUS_NAMES = {0: "GVT_OK", 1: "GVT_ERR_INVALID_ARG", 2: "GVT_ERR_INDEX_OOB",
                3: "GVT_ERR_UNSUPPORTED", 4: "GVT_ERR_ALLOC", 5: "GVT_ERR_CUDA",
                6: "GVT_ERR_BREAKDOWN", 7: "GVT_ERR_NOT_CONVERGED", 8: "GVT_ERR_TIMEOUT"}
GVT_F64, GVT_F32, GVT_BF16, GVT_F16 = 0, 1, 2, 3
KERNELS = {"kronecker": 0, "gaussian": 1, "linear": 2, "poly2d": 3, "cartesian": 4,
           "symmetric": 5, "antisymmetric": 6, "ranking": 7, "mlpk": 8}
HOMOGENEOUS = {"symmetric", "antisymmetric", "ranking", "mlpk"}
GVT_FACTOR_M, GVT_FACTOR_N, GVT_FACTOR_M_SQ, GVT_FACTOR_N_SQ, GVT_FACTOR_ONES, GVT_FACTOR_IDENTITY = range(6)
GVT_FIRST, GVT_SECOND = 0, 1
GVT_SOLVE_FP64_CG, GVT_SOLVE_MIXED_IR = 0, 1
GVT_STAGE1_SIMT, GVT_STAGE1_TC_BF16X3, GVT_STAGES_TC_F16X3, GVT_STAGES_AUTO, GVT_STAGES_TC_F16X1 = 0, 1, 2, 3, 4
GVT_TC_PAIRS_AUTO, GVT_TC_PAIRS_OFF, GVT_TC_PAIRS_ON = 0, 1, 2
GVT_MAX_TERMS = 16


class gvt_term(ctypes.Structure):
    _fields_ = [("coef", c_dbl), ("factor_a", c_i32), ("factor_b", c_i32),
                ("out_a", c_i32), ("out_b", c_i32), ("in_a", c_i32), ("in_b", c_i32)]


class gvt_desc(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("n_terms", c_i32), ("homogeneous", c_i32),
                ("reserved", c_i32), ("terms", gvt_term * GVT_MAX_TERMS)]


class gvt_matrix(ctypes.Structure):
    _fields_ = [("data", c_vp), ("rows", c_i64), ("cols", c_i64), ("ld", c_i64),
                ("dtype", c_i32), ("symmetric", c_i32)]


class gvt_solve_opts(ctypes.Structure):
    _fields_ = [("rel_tol", c_dbl), ("max_iter", c_i64), ("mode", c_i32),
                ("inner_dtype", c_i32), ("inner_tol", c_dbl), ("max_refine", c_i32),
                ("check_every", c_i32), ("precond_budget", c_i32), ("precond", c_vp),
                ("history", c_vp), ("history_cap", c_i32), ("reserved_opts", c_i32)]


class gvt_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_i64), ("refinements", c_i32), ("status", c_i32),
                ("rel_residual", c_dbl), ("time_ms", c_dbl), ("precond_fallback", c_i32), ("history_len", c_i32)]


class gvt_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", c_i64), ("ms", c_dbl), ("flops", c_dbl), ("bytes", c_dbl),
                ("useful_flops", c_dbl)]


GVT_STAT_STAGE1, GVT_STAT_STAGE2, GVT_STAT_ONE_SIDED, GVT_STAT_TC_GEMM = 0, 1, 2, 3
GVT_STAT_SPARSE_STAGE1, GVT_STAT_SPARSE_STAGE2, GVT_STAT_COUNT = 4, 5, 6
STAT_NAMES = ["stage1", "stage2", "one_sided", "tc_gemm", "sparse_stage1", "sparse_stage2"]


class gvt_problem(ctypes.Structure):
    _fields_ = [("m", c_i64), ("q", c_i64), ("n", c_i64), ("M", c_vp), ("N", c_vp), ("d", c_vp),
                ("t", c_vp), ("y", c_vp), ("a", c_vp)]


class GvtError(RuntimeError):
    def __init__(self, status, func, msg):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (func, STATUS_NAMES.get(status, status), msg))


# (name, restype, argtypes) of every entry point declared in include/gvt.h
_P = ctypes.POINTER
SIGNATURES = [
    ("gvt_last_error", ctypes.c_char_p, []),
    ("gvt_version", c_i32, []),
    ("gvt_create", c_i32, [_P(c_vp)]),
    ("gvt_destroy", c_i32, [c_vp]),
    ("gvt_plan_create", c_i32, [c_vp, c_i64, c_i64, c_i64, c_i64, c_vp, c_vp, c_i64,
                                c_vp, c_vp, c_i64, c_vp, _P(c_vp)]),
    ("gvt_plan_destroy", c_i32, [c_vp]),
    ("gvt_plan_sizes", c_i32, [c_vp, _P(c_i64), _P(c_i64)]),
    ("gvt_matvec", c_i32, [c_vp, _P(gvt_matrix), _P(gvt_matrix), c_vp, c_vp, c_i64, c_i32, c_vp]),
    ("gvt_desc_make", c_i32, [c_i32, _P(gvt_desc)]),
    ("gvt_pairwise_kernel_matvec", c_i32, [c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix),
                                           c_vp, c_vp, c_i64, c_i32, c_vp]),
    ("gvt_predict", c_i32, [c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_vp,
                            c_i64, c_i32, c_vp]),
    ("gvt_gaussian_kernel", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_i64, c_dbl, c_vp, c_i64,
                                    c_i32, c_vp]),
    ("gvt_convert", c_i32, [c_vp, c_i32, c_vp, c_i32, c_i64, c_vp]),
    ("gvt_solve_opts_default", c_i32, [_P(gvt_solve_opts)]),
    ("gvt_stats_enable", c_i32, [c_vp, c_i32]),
    ("gvt_stats_read", c_i32, [c_vp, c_vp]),
    ("gvt_launch_count", c_i64, []),
    ("gvt_tanimoto_kernel", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_i64, c_vp, c_i64, c_i32, c_vp]),
    ("gvt_linear_kernel", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_i64, c_vp, c_i64, c_i32, c_vp]),
    ("gvt_krr_cg_solve_multishift", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_vp,
                                            c_i32, c_vp, c_dbl, c_i64, c_vp, _P(gvt_solve_info), c_vp]),
    ("gvt_klr_newton_solve", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_dbl, c_vp,
                                     c_i32, c_dbl, c_dbl, c_i64, _P(gvt_solve_info), c_vp]),
    ("gvt_svm_newton_solve", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_dbl, c_vp,
                                     c_i32, c_dbl, c_i64, _P(gvt_solve_info), c_vp]),
    ("gvt_svm_subgradient_solve", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_dbl,
                                          c_vp, c_i64, c_vp, _P(gvt_solve_info), c_vp]),
    ("gvt_krr_minres_solve", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_dbl,
                                     c_vp, c_dbl, c_i64, c_i64, c_i64, c_vp, _P(gvt_solve_info), c_vp]),
    ("gvt_krr_cg_solve", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix),
                                 c_vp, c_dbl, c_vp, _P(gvt_solve_opts), _P(gvt_solve_info), c_vp]),
    ("gvt_krr_cg_solve_batched", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, _P(gvt_solve_opts), c_vp,
                                         _P(gvt_solve_info), c_vp]),
    ("gvt_matvec_batched", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    ("gvt_set_stage1_engine", c_i32, [c_vp, c_i32]),
    ("gvt_set_tc_pairs", c_i32, [c_vp, c_i32]),
    ("gvt_factor_cache_begin", c_i32, [c_vp]),
    ("gvt_factor_cache_end", c_i32, [c_vp]),
    ("gvt_precond_num_params", c_i64, []),
    ("gvt_precond_set_dtype", c_i32, [c_vp, c_i32]),
    ("gvt_precond_create", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_vp,
                                   _P(c_vp)]),
    ("gvt_precond_destroy", c_i32, [c_vp]),
    ("gvt_precond_params", c_i32, [c_vp, c_vp, c_i32, c_vp]),
    ("gvt_precond_features", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("gvt_precond_outputs", c_i32, [c_vp, c_vp, c_vp]),
    ("gvt_precond_apply", c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp]),
    ("gvt_precond_loss_grad", c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    ("gvt_precond_scale", c_i32, [c_vp, c_vp, c_vp]),
    ("gvt_precond_train", c_i32, [c_vp, c_vp, c_vp, c_i32, c_i64, c_i32, c_i32, c_dbl, c_vp, c_vp]),
    ("gvt_cg_record_pairs", c_i32, [c_vp, c_vp, _P(gvt_desc), _P(gvt_matrix), _P(gvt_matrix), c_vp, c_dbl,
                                     c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_i32, c_vp]),
    ("gvt_check_device_errors", c_i32, [c_vp, c_vp]),
    ("gvt_tc_gemm_bf16", c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_i64, c_i64, c_i64, c_vp]),
    ("gvt_set_tc_stall_test", c_i32, [c_vp, c_i64]),
    ("gvt_set_stage_tiles", c_i32, [c_vp, c_i32]),
    ("gvt_matvec_static", c_i32, [c_i64, c_i64, c_i64, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_i64,
                                  _P(gvt_matrix), _P(gvt_matrix), c_vp, c_vp, c_i32, c_vp]),
]

_lib = None


def lib_path():
    return _build.LIB


def load():
    """Load libgvt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libgvt.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2009_01054_gb300.build)")
        lib = ctypes.CDLL(_build.LIB)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def last_error():
    return load().gvt_last_error().decode()


def _call(name, *args):
    st = getattr(load(), name)(*args)
    if st != GVT_OK:
        raise GvtError(st, name, last_error())
    return st


# ---------------------------------------------------------------- raw ABI calls
def gvt_version():
    return int(load().gvt_version())


def gvt_create():
    h = c_vp()
    _call("gvt_create", ctypes.byref(h))
    return h


def gvt_destroy(h):
    _call("gvt_destroy", h)


def gvt_plan_create(h, m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in, d_out, t_out, n_out, stream):
    p = c_vp()
    _call("gvt_plan_create", h, m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in,
          d_out, t_out, n_out, stream, ctypes.byref(p))
    return p


def gvt_plan_destroy(p):
    _call("gvt_plan_destroy", p)


def gvt_desc_make(kind):
    d = gvt_desc()
    _call("gvt_desc_make", KERNELS.get(kind, kind) if isinstance(kind, str) else kind, ctypes.byref(d))
    return d


def gvt_matvec(plan, M, N, v, u, k_cols, dtype, stream):
    _call("gvt_matvec", plan, ctypes.byref(M), ctypes.byref(N), v, u, k_cols, dtype, stream)


def gvt_pairwise_kernel_matvec(plan, desc, M, N, v, u, k_cols, dtype, stream):
    _call("gvt_pairwise_kernel_matvec", plan, ctypes.byref(desc), ctypes.byref(M),
          ctypes.byref(N) if N is not None else None, v, u, k_cols, dtype, stream)


def gvt_predict(plan, desc, M, N, a, p, k_cols, dtype, stream):
    _call("gvt_predict", plan, ctypes.byref(desc), ctypes.byref(M),
          ctypes.byref(N) if N is not None else None, a, p, k_cols, dtype, stream)


def gvt_gaussian_kernel(h, X, rows_x, Y, rows_y, dim, gamma, K, ldk, out_dtype, stream):
    _call("gvt_gaussian_kernel", h, X, rows_x, Y, rows_y, dim, gamma, K, ldk, out_dtype, stream)


def gvt_convert(src, src_dtype, dst, dst_dtype, n, stream):
    _call("gvt_convert", src, src_dtype, dst, dst_dtype, n, stream)


def gvt_stats_enable(h, on):
    _call("gvt_stats_enable", h, 1 if on else 0)


def gvt_stats_read(h):
    """dict kind -> {launches, ms, flops, bytes, useful_flops}"""
    arr = (gvt_kernel_stats * GVT_STAT_COUNT)()
    _call("gvt_stats_read", h, ctypes.cast(arr, c_vp))
    return {STAT_NAMES[k]: dict(launches=arr[k].launches, ms=arr[k].ms, flops=arr[k].flops,
                                bytes=arr[k].bytes, useful_flops=arr[k].useful_flops)
            for k in range(GVT_STAT_COUNT)}


def gvt_launch_count():
    return int(load().gvt_launch_count())


def gvt_matvec_static(m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in, d_out, t_out, n_out,
                      M, N, v, u, dtype, stream):
    """Allocation-free Kronecker product (see include/gvt.h); raises on a non-zero status."""
    _call("gvt_matvec_static", m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in, d_out, t_out,
          n_out, ctypes.byref(M), ctypes.byref(N), v, u, dtype, stream)


def gvt_krr_cg_solve_batched(h, probs, lambdas, opts, stream):
    """probs: list of gvt_problem; returns (status, info, rel_residuals[n_probs][n_lambda])."""
    arr = (gvt_problem * len(probs))(*probs)
    lam = (c_dbl * len(lambdas))(*lambdas)
    rr = (c_dbl * (len(probs) * len(lambdas)))()
    info = gvt_solve_info()
    st = load().gvt_krr_cg_solve_batched(h, ctypes.cast(arr, c_vp), len(probs), ctypes.cast(lam, c_vp),
                                         len(lambdas), ctypes.byref(opts), ctypes.cast(rr, c_vp),
                                         ctypes.byref(info), stream)
    if st not in (GVT_OK, 6, 7):
        raise GvtError(st, "gvt_krr_cg_solve_batched", last_error())
    res = [[rr[b * len(lambdas) + c] for c in range(len(lambdas))] for b in range(len(probs))]
    return st, info, res


def gvt_matvec_batched(h, probs, shifts, v_ptrs, w_ptrs, stream):
    """probs: list of gvt_problem; v_ptrs / w_ptrs: device pointers per problem (FP32, n x n_cols
    column-major); raises on a non-zero status."""
    arr = (gvt_problem * len(probs))(*probs)
    sh = (c_dbl * len(shifts))(*shifts)
    vin = (c_vp * len(probs))(*[c_vp(x) for x in v_ptrs])
    wout = (c_vp * len(probs))(*[c_vp(x) for x in w_ptrs])
    _call("gvt_matvec_batched", h, ctypes.cast(arr, c_vp), len(probs), ctypes.cast(sh, c_vp), len(shifts),
          ctypes.cast(vin, c_vp), ctypes.cast(wout, c_vp), stream)


def matvec_batched(handle, problems, vectors, shifts=None, stream=None):
    """The batched FP32 operator: for every problem (dict with CUDA tensors M, N (FP64), d, t
    (int32)) and every column c of its vectors (n x n_cols FP32 tensor),
    w[:, c] = R (M kron N) R^T v[:, c] + shifts[c] v[:, c].  Returns the list of w (n x n_cols)."""
    torch = _torch()
    keep, probs, vin, outs = [], [], [], []
    for p, v in zip(problems, vectors):
        d = p["d"].to(torch.int32).contiguous()
        t = p["t"].to(torch.int32).contiguous()
        M = p["M"].to(torch.float64).contiguous()
        N = p["N"].to(torch.float64).contiguous()
        vt = v.to(torch.float32).t().contiguous()          # n_cols x n: column c at + c * n
        w = torch.empty_like(vt)
        keep += [d, t, M, N, vt]
        vin.append(vt.data_ptr())
        outs.append(w)
        probs.append(gvt_problem(M.shape[0], N.shape[0], d.numel(), c_vp(M.data_ptr()), c_vp(N.data_ptr()),
                                 c_vp(d.data_ptr()), c_vp(t.data_ptr()), None, None))
    n_cols = vectors[0].shape[1]
    shifts = [0.0] * n_cols if shifts is None else list(shifts)
    gvt_matvec_batched(handle.h, probs, shifts, vin, [w.data_ptr() for w in outs], stream_ptr(stream))
    return [w.t() for w in outs]


def krr_solve_batched(handle, problems, lambdas, rel_tol=1e-6, inner_tol=1e-3, max_iter=20000,
                      max_refine=30, check_every=5, stream=None):
    """problems: list of dicts with CUDA tensors M, N (FP64), d, t (int32), y (FP64).
    Returns (list of a tensors (n x n_lambda), status, info, rel_residuals)."""
    torch = _torch()
    keep, probs, outs = [], [], []
    for p in problems:
        d = p["d"].to(torch.int32).contiguous()
        t = p["t"].to(torch.int32).contiguous()
        y = p["y"].to(torch.float64).contiguous()
        M = p["M"].to(torch.float64).contiguous()
        N = p["N"].to(torch.float64).contiguous()
        n = d.numel()
        a = torch.zeros((len(lambdas), n), dtype=torch.float64, device=y.device)
        keep += [d, t, y, M, N, a]
        outs.append(a)
        probs.append(gvt_problem(M.shape[0], N.shape[0], n, c_vp(M.data_ptr()), c_vp(N.data_ptr()),
                                 c_vp(d.data_ptr()), c_vp(t.data_ptr()), c_vp(y.data_ptr()),
                                 c_vp(a.data_ptr())))
    o = gvt_solve_opts_default()
    o.rel_tol, o.inner_tol, o.max_iter, o.max_refine, o.check_every = rel_tol, inner_tol, max_iter, max_refine, check_every
    st, info, rr = gvt_krr_cg_solve_batched(handle.h, probs, list(lambdas), o, stream_ptr(stream))
    return [a.t() for a in outs], st, info, rr


class Precond:
    """Learned preconditioner of a training plan (gvt_precond_*)."""

    def __init__(self, handle, plan, kind, M, N, theta, symmetric=True, stream=None):
        import numpy as np
        self.n_params = int(load().gvt_precond_num_params())
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.n_params
        self.p = c_vp()
        _call("gvt_precond_create", handle.h, plan.p, ctypes.byref(_desc(kind)), ctypes.byref(matrix(M, symmetric)),
              ctypes.byref(matrix(N, symmetric)) if N is not None else None, th.ctypes.data_as(c_vp),
              stream_ptr(stream), ctypes.byref(self.p))
        self.n = plan.n_in

    def set_dtype(self, dtype):
        """Arithmetic of the network: GVT_BF16 (tensor cores, the default) or GVT_F32 (SIMT)."""
        _call("gvt_precond_set_dtype", self.p, int(dtype))

    def params(self):
        import numpy as np
        out = np.zeros(self.n_params, dtype=np.float32)
        _call("gvt_precond_params", self.p, out.ctypes.data_as(c_vp), 0, stream_ptr())
        return out

    def set_params(self, theta):
        import numpy as np
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _call("gvt_precond_params", self.p, th.ctypes.data_as(c_vp), 1, stream_ptr())

    def features(self):
        import numpy as np
        torch = _torch()
        musd = np.zeros(12, dtype=np.float32)
        X = torch.empty((self.n, 6), dtype=torch.float32, device="cuda")
        _call("gvt_precond_features", self.p, musd.ctypes.data_as(c_vp), ptr(X), stream_ptr())
        torch.cuda.synchronize()
        return musd[:6], musd[6:], X

    def outputs(self):
        torch = _torch()
        O = torch.empty((self.n, 33), dtype=torch.float32, device="cuda")
        _call("gvt_precond_outputs", self.p, ptr(O), stream_ptr())
        torch.cuda.synchronize()
        return O

    def apply(self, r):
        z = _torch().empty_like(r)
        _call("gvt_precond_apply", self.p, ptr(r), ptr(z), dtype_code(r), stream_ptr())
        return z

    def loss_grad(self, R, E):
        """R, E: CUDA float32 tensors n x K (K <= 16)."""
        import numpy as np
        Rc, Ec = R.t().contiguous(), E.t().contiguous()   # column-major n x K
        loss = c_dbl()
        g = np.zeros(self.n_params, dtype=np.float32)
        _call("gvt_precond_loss_grad", self.p, ptr(Rc), ptr(Ec), R.shape[1], ctypes.byref(loss),
              g.ctypes.data_as(c_vp), stream_ptr())
        return loss.value, g

    def scale(self, value=None):
        get = c_dbl()
        if value is not None:
            v = c_dbl(value)
            _call("gvt_precond_scale", self.p, ctypes.byref(get), ctypes.byref(v))
        else:
            _call("gvt_precond_scale", self.p, ctypes.byref(get), None)
        return get.value

    def train(self, R, E, steps, batch=8, lr=1e-3):
        """R, E: CUDA tensors n x K (float32 or bfloat16), as returned by cg_record_pairs."""
        import numpy as np
        Rc, Ec = R.t().contiguous(), E.t().contiguous()
        hist = np.zeros(max(steps, 1))
        _call("gvt_precond_train", self.p, ptr(Rc), ptr(Ec), dtype_code(R), R.shape[1], steps, batch, float(lr),
              hist.ctypes.data_as(c_vp), stream_ptr())
        return hist[:steps]

    def close(self):
        if getattr(self, "p", None) is not None:
            _call("gvt_precond_destroy", self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cg_record_pairs(handle, plan, kind, M, N, y, lam, a_star, iters, symmetric=True, stream=None, store=None,
                    out=None):
    """(R, E) n x len(iters): residuals and corrections a* - a_k of plain CG in the precision of M
    and N (FP64, or FP32 on the handle's engine), stored as `store` (torch.float32 by default, or
    torch.bfloat16).  out = (R_rows, E_rows): len(iters) x n contiguous tensors to fill instead
    (for example row slices of one large buffer, so that many recordings need no concatenation)."""
    import numpy as np
    torch = _torch()
    it = np.ascontiguousarray(iters, dtype=np.int64)
    store = store or torch.float32
    if out is not None:
        R, E = out
        assert R.shape == (len(it), plan.n_in) and E.shape == R.shape and R.is_contiguous() and E.is_contiguous()
    else:
        R = torch.empty((len(it), plan.n_in), dtype=store, device="cuda")
        E = torch.empty_like(R)
    _call("gvt_cg_record_pairs", handle.h, plan.p, ctypes.byref(_desc(kind)), ctypes.byref(matrix(M, symmetric)),
          ctypes.byref(matrix(N, symmetric)) if N is not None else None, ptr(y), float(lam), ptr(a_star),
          it.ctypes.data_as(c_vp), len(it), dtype_code(M), ptr(R), ptr(E), dtype_code(R), stream_ptr(stream))
    return R.t(), E.t()


def gvt_set_stage1_engine(h, engine):
    _call("gvt_set_stage1_engine", h, engine)


def gvt_set_tc_pairs(h, mode):
    _call("gvt_set_tc_pairs", h, mode)


def gvt_factor_cache_begin(h):
    _call("gvt_factor_cache_begin", h)


def gvt_factor_cache_end(h):
    _call("gvt_factor_cache_end", h)


def gvt_check_device_errors(h, stream):
    _call("gvt_check_device_errors", h, stream)


def gvt_tc_gemm_bf16(h, A, lda, B, ldb, C, ldc, M, N, K, stream):
    _call("gvt_tc_gemm_bf16", h, A, lda, B, ldb, C, ldc, M, N, K, stream)


GVT_TILES_AUTO, GVT_TILES_OFF, GVT_TILES_ON = 0, 1, 2


def gvt_set_stage_tiles(h, mode):
    """Per-tile dense/sparse stages: GVT_TILES_AUTO (cost model, large plans), _OFF or _ON."""
    _call("gvt_set_stage_tiles", h, int(mode))


def gvt_set_tc_stall_test(h, cycles):
    """Test of the tensor-core timeout path (see include/gvt.h): cycles > 0 makes every GEMM of this
    handle stall on a barrier nothing arrives on; 0 turns it off."""
    _call("gvt_set_tc_stall_test", h, int(cycles))


def gvt_solve_opts_default():
    o = gvt_solve_opts()
    _call("gvt_solve_opts_default", ctypes.byref(o))
    return o


def gvt_krr_cg_solve(h, plan, desc, M, N, y, lam, a, opts, stream):
    """Returns (status, gvt_solve_info); NOT_CONVERGED / BREAKDOWN are returned, not raised."""
    info = gvt_solve_info()
    st = load().gvt_krr_cg_solve(h, plan, ctypes.byref(desc), ctypes.byref(M),
                                 ctypes.byref(N) if N is not None else None, y, lam, a,
                                 ctypes.byref(opts), ctypes.byref(info), stream)
    if st not in (GVT_OK, 6, 7):
        raise GvtError(st, "gvt_krr_cg_solve", last_error())
    return st, info


def gvt_krr_minres_solve(h, plan, desc, M, N, y, lam, a, rel_tol, max_iter, record_every, n_records, records,
                         stream):
    """Returns (status, gvt_solve_info); NOT_CONVERGED / BREAKDOWN are returned, not raised."""
    info = gvt_solve_info()
    st = load().gvt_krr_minres_solve(h, plan, ctypes.byref(desc), ctypes.byref(M),
                                     ctypes.byref(N) if N is not None else None, y, lam, a, rel_tol, max_iter,
                                     record_every, n_records, records, ctypes.byref(info), stream)
    if st not in (GVT_OK, 6, 7):
        raise GvtError(st, "gvt_krr_minres_solve", last_error())
    return st, info


# ---------------------------------------------------------------- torch marshalling
def _torch():
    import torch
    return torch


_DT = {"float64": GVT_F64, "float32": GVT_F32, "bfloat16": GVT_BF16}


def dtype_code(t):
    return _DT[str(t.dtype).replace("torch.", "")]


def stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_vp(s.cuda_stream)


def ptr(t):
    return c_vp(t.data_ptr()) if t is not None and t.numel() > 0 else c_vp(t.data_ptr() if t is not None else 0)


def matrix(t, symmetric=False):
    """gvt_matrix view of a 2-D CUDA tensor with unit column stride."""
    assert t.dim() == 2 and t.is_cuda and t.stride(1) == 1
    return gvt_matrix(c_vp(t.data_ptr()), t.shape[0], t.shape[1], t.stride(0), dtype_code(t),
                      1 if symmetric else 0)


class Handle:
    def __init__(self):
        self.h = gvt_create()

    def close(self):
        if self.h is not None:
            gvt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Sorted pair sample (gvt_plan_create).  d_out/t_out None = training plan."""

    def __init__(self, handle, m_shape, q_shape, d_in, t_in, d_out=None, t_out=None, stream=None):
        torch = _torch()
        self.handle = handle
        dev = torch.device("cuda")
        self.d_in = torch.as_tensor(d_in, dtype=torch.int32, device=dev).contiguous()
        self.t_in = torch.as_tensor(t_in, dtype=torch.int32, device=dev).contiguous()
        self.n_in = self.d_in.numel()
        if d_out is None:
            do = to = c_vp(0)
            self.n_out = self.n_in
        else:
            self.d_out = torch.as_tensor(d_out, dtype=torch.int32, device=dev).contiguous()
            self.t_out = torch.as_tensor(t_out, dtype=torch.int32, device=dev).contiguous()
            do, to = ptr(self.d_out), ptr(self.t_out)
            self.n_out = self.d_out.numel()
        self.p = gvt_plan_create(handle.h, m_shape[0], m_shape[1], q_shape[0], q_shape[1],
                                 ptr(self.d_in), ptr(self.t_in), self.n_in, do, to, self.n_out,
                                 stream_ptr(stream))

    def close(self):
        if getattr(self, "p", None) is not None:
            gvt_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(kind):
    return kind if isinstance(kind, gvt_desc) else gvt_desc_make(kind)


def pairwise_kernel_matvec(plan, kind, M, N, v, u=None, symmetric=True, stream=None, predict=False):
    """u = R(dhat,that) K_kind R(d,t)^T v for CUDA tensors (v: n_in or n_in x k, column-major)."""
    torch = _torch()
    desc = _desc(kind)
    vec = v.dim() == 1
    k = 1 if vec else v.shape[1]
    vv = v if vec else v.t().contiguous()          # column-major block
    if u is None:
        u = torch.empty((k, plan.n_out), dtype=v.dtype, device=v.device)
    Mm = matrix(M, symmetric)
    Nm = matrix(N, symmetric) if N is not None else None
    fn = gvt_predict if predict else gvt_pairwise_kernel_matvec
    fn(plan.p, desc, Mm, Nm, ptr(vv), ptr(u), k, dtype_code(v), stream_ptr(stream))
    return u.reshape(-1) if vec else u.t()


def predict(plan, kind, M, N, a, stream=None, symmetric=False):
    return pairwise_kernel_matvec(plan, kind, M, N, a, symmetric=symmetric, stream=stream, predict=True)


def gaussian_kernel(handle, X, Y=None, gamma=1.0, dtype=None, stream=None):
    torch = _torch()
    X = X.to(torch.float64).contiguous()
    Y = X if Y is None else Y.to(torch.float64).contiguous()
    out = torch.empty((X.shape[0], Y.shape[0]), dtype=dtype or torch.float64, device=X.device)
    gvt_gaussian_kernel(handle.h, ptr(X), X.shape[0], ptr(Y), Y.shape[0], X.shape[1], float(gamma),
                        ptr(out), out.stride(0), dtype_code(out), stream_ptr(stream))
    return out


def linear_kernel(handle, X, Y=None, dtype=None, stream=None):
    """Linear base kernel <X_a, Y_b> (rows of a similarity matrix as features), summed in FP64."""
    torch = _torch()
    X = X.to(torch.float64).contiguous()
    Y = X if Y is None else Y.to(torch.float64).contiguous()
    out = torch.empty((X.shape[0], Y.shape[0]), dtype=dtype or torch.float64, device=X.device)
    _call("gvt_linear_kernel", handle.h, ptr(X), X.shape[0], ptr(Y), Y.shape[0], X.shape[1], ptr(out),
          out.stride(0), dtype_code(out), stream_ptr(stream))
    return out


def tanimoto_kernel(handle, Xp, Yp=None, dtype=None, stream=None):
    """Tanimoto kernel of bit-packed fingerprints (CUDA int32 tensors of packed uint32 words)."""
    torch = _torch()
    Xp = Xp.to(torch.int32).contiguous()
    Yp = Xp if Yp is None else Yp.to(torch.int32).contiguous()
    out = torch.empty((Xp.shape[0], Yp.shape[0]), dtype=dtype or torch.float64, device=Xp.device)
    _call("gvt_tanimoto_kernel", handle.h, ptr(Xp), Xp.shape[0], ptr(Yp), Yp.shape[0], Xp.shape[1], ptr(out),
          out.stride(0), dtype_code(out), stream_ptr(stream))
    return out


def krr_cg_solve_multishift(handle, plan, kind, M, N, y, lambdas, rel_tol=1e-6, max_iter=10000, symmetric=True,
                            stream=None):
    """Multi-shift CG for a lambda sweep; returns (A (n x n_lambda), status, info, rel_residuals)."""
    torch = _torch()
    lam = (c_dbl * len(lambdas))(*[float(x) for x in lambdas])
    rr = (c_dbl * len(lambdas))()
    A = torch.zeros((len(lambdas), y.numel()), dtype=torch.float64, device=y.device)
    info = gvt_solve_info()
    st = load().gvt_krr_cg_solve_multishift(handle.h, plan.p, ctypes.byref(_desc(kind)),
                                            ctypes.byref(matrix(M, symmetric)),
                                            ctypes.byref(matrix(N, symmetric)) if N is not None else None,
                                            ptr(y), ctypes.cast(lam, c_vp), len(lambdas), ptr(A), float(rel_tol),
                                            int(max_iter), ctypes.cast(rr, c_vp), ctypes.byref(info),
                                            stream_ptr(stream))
    if st not in (GVT_OK, 6, 7):
        raise GvtError(st, "gvt_krr_cg_solve_multishift", last_error())
    return A.t(), st, info, [rr[k] for k in range(len(lambdas))]


def klr_newton_solve(handle, plan, kind, M, N, y, lam, newton_iters=30, cg_tol=1e-10, grad_tol=1e-10,
                     max_cg_iter=100000, symmetric=True, stream=None):
    """Kernel logistic regression (labels +-1) by Newton's method; returns (a, status, info)."""
    torch = _torch()
    a = torch.zeros_like(y)
    info = gvt_solve_info()
    st = load().gvt_klr_newton_solve(handle.h, plan.p, ctypes.byref(_desc(kind)), ctypes.byref(matrix(M, symmetric)),
                                     ctypes.byref(matrix(N, symmetric)) if N is not None else None, ptr(y),
                                     float(lam), ptr(a), int(newton_iters), float(cg_tol), float(grad_tol),
                                     int(max_cg_iter), ctypes.byref(info), stream_ptr(stream))
    if st not in (GVT_OK, 6, 7):
        raise GvtError(st, "gvt_klr_newton_solve", last_error())
    return a, st, info


def svm_newton_solve(handle, plan, kind, M, N, y, lam, newton_iters=50, cg_tol=1e-12, max_cg_iter=100000,
                     symmetric=True, stream=None):
    """Squared-hinge SVM (labels +-1) by Newton's method over active sets; returns (a, status, info)."""
    torch = _torch()
    a = torch.zeros_like(y)
    info = gvt_solve_info()
    st = load().gvt_svm_newton_solve(handle.h, plan.p, ctypes.byref(_desc(kind)), ctypes.byref(matrix(M, symmetric)),
                                     ctypes.byref(matrix(N, symmetric)) if N is not None else None, ptr(y),
                                     float(lam), ptr(a), int(newton_iters), float(cg_tol), int(max_cg_iter),
                                     ctypes.byref(info), stream_ptr(stream))
    if st not in (GVT_OK, GVT_ERR_BREAKDOWN, GVT_ERR_NOT_CONVERGED):
        raise GvtError(st, "gvt_svm_newton_solve", last_error())
    return a, st, info


def svm_subgradient_solve(handle, plan, kind, M, N, y, lam, iters, symmetric=True, stream=None):
    """Hinge-loss SVM (labels +-1) by kernelised sub-gradient steps; returns (a, objective, info)."""
    torch = _torch()
    a = torch.zeros_like(y)
    info = gvt_solve_info()
    obj = c_dbl(0.0)
    _call("gvt_svm_subgradient_solve", handle.h, plan.p, ctypes.byref(_desc(kind)), ctypes.byref(matrix(M, symmetric)),
          ctypes.byref(matrix(N, symmetric)) if N is not None else None, ptr(y), float(lam), ptr(a), int(iters),
          ctypes.byref(obj), ctypes.byref(info), stream_ptr(stream))
    return a, obj.value, info


def krr_minres_solve(handle, plan, kind, M, N, y, lam, rel_tol=1e-6, max_iter=10000, record_every=0,
                     n_records=0, symmetric=True, stream=None):
    """MINRES on (K + lam I) a = y; returns (a, status, info, records (n x n_records) or None)."""
    torch = _torch()
    a = torch.zeros_like(y)
    rec = torch.zeros((n_records, y.numel()), dtype=torch.float64, device=y.device) \
        if record_every > 0 and n_records > 0 else None
    st, info = gvt_krr_minres_solve(handle.h, plan.p, _desc(kind), matrix(M, symmetric),
                                    matrix(N, symmetric) if N is not None else None, ptr(y), float(lam), ptr(a),
                                    float(rel_tol), int(max_iter), int(record_every), int(n_records),
                                    ptr(rec) if rec is not None else None, stream_ptr(stream))
    return a, st, info, (rec.t() if rec is not None else None)


def krr_cg_solve(handle, plan, kind, M, N, y, lam, a0=None, mode=GVT_SOLVE_FP64_CG, rel_tol=1e-6,
                 max_iter=10000, inner_tol=1e-3, check_every=1, symmetric=True, stream=None,
                 inner_dtype=GVT_F32, precond=None, precond_budget=0, history=0):
    """Solve (K + lam I) a = y; returns (a, status, info), or (a, status, info, hist) when
    history > 0: hist is the list of (iteration, relative residual) pairs the solver recorded
    (at most `history` of them)."""
    torch = _torch()
    a = torch.zeros_like(y) if a0 is None else a0.clone()
    o = gvt_solve_opts_default()
    o.rel_tol, o.max_iter, o.mode, o.inner_tol, o.check_every = rel_tol, max_iter, mode, inner_tol, check_every
    o.inner_dtype = inner_dtype
    o.precond = precond.p if precond is not None else None
    o.precond_budget = precond_budget
    hbuf = None
    if history > 0:
        hbuf = (c_dbl * (2 * int(history)))()
        o.history = ctypes.cast(hbuf, c_vp)
        o.history_cap = int(history)
    st, info = gvt_krr_cg_solve(handle.h, plan.p, _desc(kind), matrix(M, symmetric),
                                matrix(N, symmetric) if N is not None else None,
                                ptr(y), float(lam), ptr(a), o, stream_ptr(stream))
    if hbuf is None:
        return a, st, info
    hist = [(int(hbuf[2 * k]), float(hbuf[2 * k + 1])) for k in range(info.history_len)]
    return a, st, info, hist
