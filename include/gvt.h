/*
 * gvt.h -- C ABI of the GB300 (sm_103a) generalized vec trick library.
 *
 * The library applies pairwise kernel matrices to vectors without forming
 * them.  With training pairs (d_j, t_j), j < n, and output pairs
 * (dhat_i, that_i), i < nhat, a drug kernel matrix M (the paper's D) and a
 * target kernel matrix N (the paper's T), the basic operation is
 *
 *     u = R(dhat, that) (M kron N) R(d, t)^T v,
 *     u_i = sum_j M[dhat_i, d_j] * N[that_i, t_j] * v_j            (Theorem 1)
 *
 * computed in O(qbar*n + m*nhat) by the two-stage generalized vec trick:
 * stage 1 forms S = N W (W is q x m sparse with v_j at (t_j, d_j)), stage 2
 * gathers u_i = <M[dhat_i, :], S[that_i, :]>.  Every pairwise kernel of
 * Table 4b is a sum of such Kronecker terms with permuted index sequences
 * (Corollary 1); the kernel ridge regression system (K + lambda I) a = y
 * (Eq. 1) is solved with conjugate gradients on top.  The same product also
 * drives the paper's MINRES with early stopping (Sec. 6), multi-shift CG over a
 * lambda sweep, batched solves of many problems, and kernel logistic
 * regression and support vector machines (Sec. 7).
 *
 * Conventions shared by every entry point:
 *  - Every data pointer is DEVICE memory owned by the caller unless stated;
 *    the library never frees caller memory.  Work is enqueued on the given
 *    stream (a cudaStream_t passed as void*, NULL = legacy default stream).
 *  - Matrices are row-major with a leading dimension ld >= cols (elements).
 *  - Index sequences are int32, 0-based.  Counts are int64.
 *  - Multi-column vectors are column-major: column c of an n x k block starts
 *    at element c*n.
 *  - Every function returns a gvt_status.  Nothing aborts, traps or throws
 *    across the ABI.  gvt_last_error() returns a message for the last
 *    failure on the calling thread.
 *  - Entry points that need a result on the host (plan validation, solver
 *    convergence) synchronise the given stream; all others are asynchronous.
 */
#ifndef GVT_H_
#define GVT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gvt_status {
    GVT_OK = 0,
    GVT_ERR_INVALID_ARG = 1,   /* bad pointer, size, dtype or shape */
    GVT_ERR_INDEX_OOB = 2,     /* an index sequence leaves the kernel matrix */
    GVT_ERR_UNSUPPORTED = 3,   /* valid request the library does not implement */
    GVT_ERR_ALLOC = 4,         /* device allocation failed */
    GVT_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    GVT_ERR_BREAKDOWN = 6,     /* CG breakdown: p^T (K + lambda I) p <= 0 or not finite */
    GVT_ERR_NOT_CONVERGED = 7, /* iteration limit reached; best iterate returned */
    GVT_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} gvt_status;

/* Element / arithmetic types.  A gvt_matrix and the vectors of a call share one dtype. */
typedef enum gvt_dtype {
    GVT_F64 = 0,
    GVT_F32 = 1,
    GVT_BF16 = 2,
    GVT_F16 = 3      /* only as a MIXED_IR inner precision (gvt_solve_opts.inner_dtype) */
} gvt_dtype;

/* Pairwise kernels of Table 4b.  GAUSSIAN is the Kronecker product of two
 * Gaussian base kernels (Sec. 4.3); the caller supplies those as M and N.
 * SYMMETRIC, ANTISYMMETRIC, RANKING and MLPK are homogeneous (Table 4a):
 * both pair components index M, N is ignored. */
typedef enum gvt_kernel_kind {
    GVT_KERNEL_KRONECKER = 0,
    GVT_KERNEL_GAUSSIAN = 1,
    GVT_KERNEL_LINEAR = 2,
    GVT_KERNEL_POLY2D = 3,
    GVT_KERNEL_CARTESIAN = 4,
    GVT_KERNEL_SYMMETRIC = 5,
    GVT_KERNEL_ANTISYMMETRIC = 6,
    GVT_KERNEL_RANKING = 7,
    GVT_KERNEL_MLPK = 8
} gvt_kernel_kind;

/* Kronecker factor of a term.  M_SQ / N_SQ are elementwise squares
 * (D^{o2} in Theorem 2), ONES the all-ones operator 1, IDENTITY the
 * identity operator I (Corollary 1). */
typedef enum gvt_factor {
    GVT_FACTOR_M = 0,
    GVT_FACTOR_N = 1,
    GVT_FACTOR_M_SQ = 2,
    GVT_FACTOR_N_SQ = 3,
    GVT_FACTOR_ONES = 4,
    GVT_FACTOR_IDENTITY = 5
} gvt_factor;

/* Which component of a pair an index comes from. */
typedef enum gvt_component {
    GVT_FIRST = 0,   /* d (drug) */
    GVT_SECOND = 1   /* t (target), or d' on a homogeneous domain */
} gvt_component;

/*
 * One Kronecker term of a pairwise kernel.  It adds
 *     coef * A[o_a(i), i_a(j)] * B[o_b(i), i_b(j)] * v_j
 * to u_i, where A = factor_a, B = factor_b, o_x(i) is component out_x of
 * output pair i and i_x(j) is component in_x of input pair j.  Choosing
 * components other than (FIRST, SECOND) is the index remapping by the
 * commutation / unification operators, R(d,t)P = R(t,d) and
 * R(d,t)Q = R(d,d) (proof of Corollary 1).
 */
typedef struct gvt_term {
    double coef;
    int32_t factor_a, factor_b;   /* gvt_factor */
    int32_t out_a, out_b;         /* gvt_component */
    int32_t in_a, in_b;           /* gvt_component */
} gvt_term;

#define GVT_MAX_TERMS 16

/* A pairwise kernel as a sum of Kronecker terms (Corollary 1). */
typedef struct gvt_desc {
    int32_t kind;          /* gvt_kernel_kind, or -1 for a caller-built sum */
    int32_t n_terms;       /* 1 .. GVT_MAX_TERMS */
    int32_t homogeneous;   /* nonzero: needs the drug and target domains to coincide */
    int32_t reserved;
    gvt_term terms[GVT_MAX_TERMS];
} gvt_desc;

/* A dense kernel matrix in device memory. */
typedef struct gvt_matrix {
    const void* data;      /* device pointer, row-major */
    int64_t rows, cols;    /* rows index output-pair ids, cols index input-pair ids */
    int64_t ld;            /* leading dimension in elements, >= cols */
    int32_t dtype;         /* gvt_dtype; must equal the call's dtype */
    int32_t symmetric;     /* nonzero: caller asserts data[a*ld+b] == data[b*ld+a] (square).
                              Lets stage 1 read columns as rows; otherwise the library
                              transposes into its workspace. */
} gvt_matrix;

typedef struct gvt_handle gvt_handle;   /* workspace, library state */
typedef struct gvt_plan gvt_plan;       /* sorted index sequences of one problem */

/* Message describing the last failure on the calling thread ("" if none).
 * The pointer stays valid until the next failing call on this thread. */
const char* gvt_last_error(void);

/* Library version, e.g. 1.0 -> 10000. */
int32_t gvt_version(void);

/* Create / destroy a handle.  The handle owns a growable device workspace
 * and must not be used by two host threads at once.  Destroying NULL is OK.
 * gvt_destroy synchronises the device before releasing memory. */
gvt_status gvt_create(gvt_handle** out);
gvt_status gvt_destroy(gvt_handle* h);

/*
 * Build a plan for a pair sample (Sec. 2: the sequences d, t; Sec. 3: the
 * sampling operators R(d,t), R(dhat,that)).
 *   m_rows, m_cols : shape of M (rows: output drug ids, cols: input drug ids)
 *   q_rows, q_cols : shape of N (rows: output target ids, cols: input target ids)
 *   d_in, t_in     : n_in input pairs (device int32); d_in < m_cols, t_in < q_cols
 *   d_out, t_out   : n_out output pairs (device int32); d_out < m_rows, t_out < q_rows.
 *                    Both NULL (and n_out ignored): output pairs = input pairs,
 *                    the training operator of Eq. (1).
 * The plan copies the sequences (the caller may free them afterwards),
 * validates every index (GVT_ERR_INDEX_OOB names the first failing array)
 * and sorts them by each component with a stable device radix sort.
 * Synchronises `stream`.  n_in or n_out may be 0.  Counts must be < 2^31.
 */
gvt_status gvt_plan_create(gvt_handle* h,
                           int64_t m_rows, int64_t m_cols, int64_t q_rows, int64_t q_cols,
                           const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                           const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                           void* stream, gvt_plan** out);

/* Release a plan (synchronises the device).  NULL is OK. */
gvt_status gvt_plan_destroy(gvt_plan* plan);

/* Number of input and output pairs of a plan. */
gvt_status gvt_plan_sizes(const gvt_plan* plan, int64_t* n_in, int64_t* n_out);

/*
 * The Kronecker product kernel matrix times k_cols vectors (Theorem 1):
 *     u = R(dhat,that) (M kron N) R(d,t)^T v
 * v : n_in x k_cols, u : n_out x k_cols (column-major, device, `dtype`).
 * M, N : kernel matrices in `dtype` (GVT_F64 or GVT_F32).  u is overwritten.
 * The ordering of the two stages is chosen by the cost
 * min(qbar*n + m*nhat, mbar*n + q*nhat) of Theorem 1.
 */
gvt_status gvt_matvec(gvt_plan* plan, const gvt_matrix* M, const gvt_matrix* N,
                      const void* v, void* u, int64_t k_cols, int32_t dtype, void* stream);

/* Fill `out` with the sum-of-Kronecker form of a Table 4b kernel
 * (Corollary 1 and its proof; MLPK has 10 terms). */
gvt_status gvt_desc_make(int32_t kind, gvt_desc* out);

/*
 * Pairwise kernel matrix times vectors:  u = R(dhat,that) K_desc R(d,t)^T v,
 * K_desc = sum over desc->terms (Corollary 1).  Same layout rules as
 * gvt_matvec; homogeneous descriptors need m_rows == q_rows and
 * m_cols == q_cols and read M only (N may be NULL).  Terms that share
 * factors and output components are merged so that each stage runs once
 * per distinct (factor, index recipe).
 */
gvt_status gvt_pairwise_kernel_matvec(gvt_plan* plan, const gvt_desc* desc,
                                      const gvt_matrix* M, const gvt_matrix* N,
                                      const void* v, void* u, int64_t k_cols,
                                      int32_t dtype, void* stream);

/*
 * Predictions for new pairs (Sec. 3, representer form; Eq. 1's prediction
 * product):  p = R(dhat,that) K_desc R(d,t)^T a, with a the dual
 * coefficients of the training pairs (the plan's input pairs) and the
 * plan's output pairs the pairs to predict.  M and N are the cross kernels
 * (rows: prediction-side ids, cols: training-side ids).
 */
gvt_status gvt_predict(gvt_plan* plan, const gvt_desc* desc,
                       const gvt_matrix* M, const gvt_matrix* N,
                       const void* a, void* p, int64_t k_cols, int32_t dtype, void* stream);

/*
 * Gaussian base kernel  K[a, b] = exp(-gamma * ||X_a - Y_b||^2)
 * (Sec. 5.2, squared norm), computed in FP64 and stored in out_dtype
 * (GVT_F64, GVT_F32 or GVT_BF16).  X: rows_x x dim, Y: rows_y x dim,
 * row-major FP64 device arrays; Y may equal X.  K: rows_x x rows_y, ld ldk.
 */
gvt_status gvt_gaussian_kernel(gvt_handle* h, const double* X, int64_t rows_x,
                               const double* Y, int64_t rows_y, int64_t dim,
                               double gamma, void* K, int64_t ldk, int32_t out_dtype,
                               void* stream);

/*
 * Linear base kernel  K[a, b] = <X_a, Y_b>  (Sec. 5, the Metz data set: the rows
 * of a drug or target similarity matrix serve as feature vectors), summed in
 * FP64 and stored in out_dtype (GVT_F64, GVT_F32 or GVT_BF16).  X: rows_x x dim,
 * Y: rows_y x dim, row-major FP64 device arrays; Y may equal X.  K: rows_x x
 * rows_y, ld ldk >= rows_y.  GVT_ERR_INVALID_ARG on NULL or negative sizes.
 */
gvt_status gvt_linear_kernel(gvt_handle* h, const double* X, int64_t rows_x,
                             const double* Y, int64_t rows_y, int64_t dim,
                             void* K, int64_t ldk, int32_t out_dtype, void* stream);

/*
 * Tanimoto (MinMax) base kernel of binary fingerprints (Sec. 5):
 *     K[a, b] = sum_i min(x_ai, y_bi) / sum_i max(x_ai, y_bi) = |x_a AND y_b| / |x_a OR y_b|,
 * with K[a, b] = 1 when both fingerprints are empty.  X: rows_x x words, Y: rows_y x
 * words, uint32 device arrays, bit-packed (bit j of word w is feature 32 w + j; bits past
 * the fingerprint length must be zero); Y may equal X.  K: rows_x x rows_y, ld ldk,
 * stored in out_dtype (GVT_F64, GVT_F32 or GVT_BF16); the ratio is formed in FP64.
 */
gvt_status gvt_tanimoto_kernel(gvt_handle* h, const uint32_t* X, int64_t rows_x,
                               const uint32_t* Y, int64_t rows_y, int64_t words,
                               void* K, int64_t ldk, int32_t out_dtype, void* stream);

/*
 * Engine of the GVT stages for FP32 products of dense x dense terms (Theorem 1's
 * two products with W densified; the engine changes how they are computed, not
 * what).  FP64 products ignore it and always run the SIMT stages.
 *  GVT_STAGE1_SIMT      : stage 1 a sparse scatter-accumulate over the sorted pairs,
 *                         stage 2 a sampled gather-dot; FP32 arithmetic (default).
 *  GVT_STAGE1_TC_BF16X3 : stage 1 only as a tcgen05 GEMM on BF16 hi/lo splits of both
 *                         operands (hi*hi + hi*lo + lo*hi, FP32 accumulation; products
 *                         accurate to ~1e-5 relative); the stage ordering then
 *                         minimises the stage-2 length.  Stage 2 stays SIMT FP32.
 *  GVT_STAGES_TC_F16X3  : both stages as tcgen05 GEMMs on FP16 hi/lo splits, every row
 *                         scaled by a power of two first (products accurate to ~2^-21
 *                         relative, FP32 class); stage 2 computes A S^T densely and
 *                         reads out the sampled entries.
 *  GVT_STAGES_AUTO      : per stage, GVT_STAGES_TC_F16X3 where a cost model (dense
 *                         GEMM time vs sparse SIMT time at measured GB300 rates)
 *                         favours it -- W dense enough -- and SIMT elsewhere.
 *  GVT_STAGES_TC_F16X1  : per stage as GVT_STAGES_AUTO, but the dense stages are a
 *                         single tcgen05 pass over the FP16 hi parts alone (row-scaled;
 *                         products accurate to about 2^-11 relative, a third of the
 *                         GEMM work).  For inner operators whose error an FP64 outer
 *                         refinement removes (gvt_solve_opts.inner_dtype = GVT_F16).
 * Affects later products made with plans of this handle.
 */
typedef enum gvt_stage1_engine {
    GVT_STAGE1_SIMT = 0,
    GVT_STAGE1_TC_BF16X3 = 1,
    GVT_STAGES_TC_F16X3 = 2,
    GVT_STAGES_AUTO = 3,
    GVT_STAGES_TC_F16X1 = 4
} gvt_stage1_engine;

gvt_status gvt_set_stage1_engine(gvt_handle* h, int32_t engine);

/* Synchronise the device and report (then clear) errors recorded by device
 * code of this handle: GVT_ERR_TIMEOUT when a bounded wait in a tensor-core
 * kernel expired. */
gvt_status gvt_check_device_errors(gvt_handle* h, void* stream);

/*
 * Keep split copies of kernel matrices across products.  Between
 * gvt_factor_cache_begin and the matching gvt_factor_cache_end, the dense
 * engines keep the 16-bit hi/lo split of each kernel matrix they read (up to
 * four; the least recently used is replaced) in handle-owned device memory and
 * reuse it in later products of this handle.  The key is the matrix pointer,
 * leading dimension, extents and split format.  The caller guarantees that
 * the contents of those matrices do not change until the scope ends, and that
 * the products of the scope are ordered on the device (one stream, or events).
 * Scopes nest.  When the outermost one ends, the copies are dropped; their
 * memory is kept for reuse and freed by gvt_destroy.  The solvers open such a
 * scope themselves for the duration of a solve.  gvt_factor_cache_end returns
 * GVT_ERR_INVALID_ARG when no scope is open.  Host-only calls: no device work.
 */
gvt_status gvt_factor_cache_begin(gvt_handle* h);
gvt_status gvt_factor_cache_end(gvt_handle* h);

/*
 * Tile form of the tensor-core GEMM of the dense engines.  Both forms compute
 * the same chunked FP32 sums; they agree to FP32 rounding.
 *  GVT_TC_PAIRS_AUTO : the library's choice (default); currently one SM per
 *                      tile, which measured as fast as SM pairs on GB300
 *  GVT_TC_PAIRS_OFF  : one SM per 128-row output tile (tcgen05.mma cta_group::1)
 *  GVT_TC_PAIRS_ON   : a cluster of two SMs per 256-row output tile
 *                      (tcgen05.mma cta_group::2), also for 128 rows or fewer
 * Returns GVT_ERR_INVALID_ARG for any other value.
 */
typedef enum gvt_tc_pairs {
    GVT_TC_PAIRS_AUTO = 0,
    GVT_TC_PAIRS_OFF = 1,
    GVT_TC_PAIRS_ON = 2
} gvt_tc_pairs;

gvt_status gvt_set_tc_pairs(gvt_handle* h, int32_t mode);

/*
 * Per-tile dense/sparse stages under GVT_STAGES_AUTO and GVT_STAGES_TC_F16X1 (FP32 products of a
 * Kronecker term whose two factors are kernel matrices).  With power-law degrees W is dense in a
 * few rows and columns and sparse elsewhere: ids are relabelled by decreasing degree (the plan
 * keeps the relabelling, built on the host on first use), W^T is cut into tiles of 256 columns by
 * 64 rows and the output grid into tiles of 128 by 256; tiles with more pairs than a measured
 * break-even count run on the tensor-core GEMM (block-sparse in stage 1, a tile list in stage 2),
 * the other pairs on the SIMT stages.  Theorem 1's cost then holds on the sparse part while the
 * dense part runs at tensor-core rate.  Results equal the other forms' to rounding.
 *  GVT_TILES_AUTO : the cost model picks SIMT, dense or per tile for each stage, on plans of at
 *                   least 2^20 pairs (default);
 *  GVT_TILES_OFF  : never per tile;
 *  GVT_TILES_ON   : per tile wherever the form applies, whatever the cost model says (tests).
 */
typedef enum gvt_stage_tiles {
    GVT_TILES_AUTO = 0,
    GVT_TILES_OFF = 1,
    GVT_TILES_ON = 2
} gvt_stage_tiles;

gvt_status gvt_set_stage_tiles(gvt_handle* h, int32_t mode);

/*
 * The tensor-core GEMM behind GVT_STAGE1_TC_BF16X3, exposed for testing:
 * C[M x N] = A[M x K] B[N x K]^T with A, B BF16 row-major (K innermost,
 * K a multiple of 64, lda and ldb multiples of 8, 16-byte aligned), C FP32
 * row-major with leading dimension ldc >= N.  The tile form is the handle's
 * (gvt_set_tc_pairs).  Asynchronous; device-side timeouts are reported by
 * gvt_check_device_errors.
 */
gvt_status gvt_tc_gemm_bf16(gvt_handle* h, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                            int64_t ldc, int64_t M, int64_t N, int64_t K, void* stream);

/*
 * Test of the tensor-core kernels' timeout path (no counterpart in the paper; failure
 * detection).  While `cycles` > 0, every tensor-core GEMM this handle launches makes its MMA
 * thread first wait that many SM clock cycles on an mbarrier that nothing arrives on.  The
 * wait expires, the kernel takes the path of any expired wait -- its other threads stop
 * waiting, it waits (bounded) for the tile copies and MMAs it issued, frees its tensor memory
 * and returns -- and GVT_ERR_TIMEOUT lands in the handle's error word (gvt_check_device_errors;
 * the GEMM's output is then invalid).  cycles = 0 (the default) turns it off.  The one-SM tile
 * form only: a GEMM in the SM-pair form (gvt_set_tc_pairs ON) returns GVT_ERR_UNSUPPORTED while
 * it is on.  GVT_ERR_INVALID_ARG for cycles outside [0, 4e9].
 */
gvt_status gvt_set_tc_stall_test(gvt_handle* h, int64_t cycles);

/* Convert n elements between dtypes (device to device, round to nearest). */
gvt_status gvt_convert(const void* src, int32_t src_dtype, void* dst, int32_t dst_dtype,
                       int64_t n, void* stream);

/* ------------------------------------------------------------------ solver */

typedef enum gvt_solve_mode {
    GVT_SOLVE_FP64_CG = 0,    /* plain CG, FP64 operator and vectors */
    GVT_SOLVE_MIXED_IR = 1    /* FP64 residual + refinement around a low-precision inner CG */
} gvt_solve_mode;

typedef struct gvt_solve_opts {
    double rel_tol;          /* target ||y - (K + lambda I) a||_2 / ||y||_2 (default 1e-6) */
    int64_t max_iter;        /* total CG iterations, inner ones included (default 10000) */
    int32_t mode;            /* gvt_solve_mode (default GVT_SOLVE_FP64_CG) */
    int32_t inner_dtype;     /* MIXED_IR inner operator: GVT_F32 (default: the handle's engine),
                                GVT_BF16 (FP32 CG with the GVT_STAGE1_TC_BF16X3 stage 1) or
                                GVT_F16 (FP32 CG with the single-pass GVT_STAGES_TC_F16X1 stages) */
    double inner_tol;        /* MIXED_IR inner relative tolerance (default 1e-3) */
    int32_t max_refine;      /* MIXED_IR outer steps (default 30) */
    int32_t check_every;     /* CG iterations between convergence checks (default 1).  The host
                                reads each check one check late, without stalling the GPU, so a
                                run may go up to check_every iterations past the one that met
                                the tolerance (they continue the same CG) */
    int32_t precond_budget;  /* flexible-CG iterations allowed (per inner solve in MIXED_IR) before
                                the solve falls back to plain CG from the current iterate;
                                0 (default): max_iter / 2 */
    const struct gvt_precond* precond;  /* learned preconditioner for flexible CG (NULL: plain CG);
                                           applies to the FP64 CG and to MIXED_IR's inner solves */
    double* history;         /* host array of 2 * history_cap doubles, or NULL: the residual
                                history as (iteration, relative residual) pairs.  FP64_CG records
                                every convergence check (the recursive residual); MIXED_IR records
                                every refinement step (the true FP64 residual, at the inner
                                iterations so far).  gvt_solve_info.history_len counts the pairs */
    int32_t history_cap;     /* pairs `history` holds (default 0) */
    int32_t reserved_opts;
} gvt_solve_opts;

typedef struct gvt_solve_info {
    int64_t iterations;      /* CG iterations performed (inner ones for MIXED_IR) */
    int32_t refinements;     /* outer refinement steps (MIXED_IR) */
    int32_t status;          /* gvt_status of the solve */
    double rel_residual;     /* final ||y - (K+lambda I)a|| / ||y||, recomputed in FP64 */
    double time_ms;          /* wall-clock time of the solve on the host */
    int32_t precond_fallback;  /* 1 if flexible CG broke down or ran out of its budget and
                                  plain CG took over (the preconditioner is then ignored) */
    int32_t history_len;     /* (iteration, residual) pairs written to opts.history */
} gvt_solve_info;

typedef struct gvt_precond gvt_precond;

/* Fill `o` with the defaults listed in gvt_solve_opts. */
gvt_status gvt_solve_opts_default(gvt_solve_opts* o);

/*
 * Kernel ridge regression (Eq. 1): solve
 *     (R K_desc R^T + lambda I) a = y
 * over the plan's input pairs (the plan must be a training plan: output
 * pairs = input pairs).  M, N: FP64 kernel matrices.  y: n FP64.
 * a: n FP64, in: warm start (set it to zero for a cold start), out: solution.
 * MIXED_IR computes the residual y - (K + lambda I)a with the FP64 operator,
 * solves for the correction with an FP32 operator (FP64 dot products and
 * step lengths) and adds it to a in FP64; the inner matrices are converted
 * into the handle's workspace.  Synchronises `stream`.  On
 * GVT_ERR_NOT_CONVERGED / GVT_ERR_BREAKDOWN `a` holds the last iterate and
 * `info` (may be NULL) is filled in.
 * The CG iterations run on a stream the handle owns, after everything queued
 * on `stream` and before anything queued on it later.  Without a
 * preconditioner and with statistics off, blocks of check_every iterations
 * are captured once into a CUDA graph after the first block and replayed
 * (the product must not change its device buffers in between, which holds
 * within one solve); the results are those of the eager loop.
 */
gvt_status gvt_krr_cg_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                            const gvt_matrix* M, const gvt_matrix* N,
                            const double* y, double lambda, double* a,
                            const gvt_solve_opts* opts, gvt_solve_info* info, void* stream);

/*
 * Multi-shift CG: the kernel ridge systems (K + lambda_s I) a_s = y for a whole sweep of
 * n_lambda <= 32 regularisation values (host array, each > 0) from one Krylov space:
 * CG on the base system with the smallest lambda, one FP64 product per iteration, and
 * every other lambda advanced by the collinear-residual recurrences of shifted CG.
 * A (device, n x n_lambda FP64, column-major, caller-owned) receives the solutions; a
 * shift stops updating when its recursive residual reaches rel_tol * ||y||.
 * rel_residuals (host, n_lambda, may be NULL): ||y - (K + lambda_s I) a_s|| / ||y||
 * recomputed in FP64 (one more product per lambda).  info (may be NULL): iterations of
 * the base system and the largest recomputed residual.  M, N FP64; a training plan.
 * Synchronises `stream` once per iteration.  GVT_ERR_NOT_CONVERGED when max_iter ends
 * the run first (A holds the last iterates).
 */
gvt_status gvt_krr_cg_solve_multishift(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                                       const gvt_matrix* M, const gvt_matrix* N, const double* y,
                                       const double* lambdas, int32_t n_lambda, double* A,
                                       double rel_tol, int64_t max_iter, double* rel_residuals,
                                       gvt_solve_info* info, void* stream);

/*
 * Kernel logistic regression with a pairwise kernel, by Newton's method on the dual
 * coefficients (another loss through the same product; Sec. 7 names such extensions):
 *     J(a) = sum_i log(1 + exp(-y_i f_i)) + (lambda / 2) a^T K a,   f = K a,  y_i = +-1.
 * Each Newton step solves (W K + lambda I) d = -(g + lambda a) (g: loss gradient in f,
 * W = diag(s (1 - s)), s = sigmoid(y f)) through the SPD system
 * (W^1/2 K W^1/2 + lambda I) c = W^1/2 K b by CG to relative residual cg_tol (at most
 * max_cg_iter iterations), d = (b - W^1/2 c) / lambda, then a backtracking line search
 * halves the step until J decreases.  FP64 products; M, N FP64 and symmetric; a training
 * plan.  y, a: device FP64 (a out; starts from zero).  Stops when ||g + lambda a|| <=
 * grad_tol ||y|| or after newton_iters steps.  info (may be NULL): refinements = Newton
 * steps, iterations = CG iterations in total, rel_residual = ||g + lambda a|| / ||y||.
 * Returns GVT_ERR_NOT_CONVERGED when newton_iters (or an inner max_cg_iter) ends the run.
 */
gvt_status gvt_klr_newton_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                                const gvt_matrix* M, const gvt_matrix* N, const double* y,
                                double lambda, double* a, int32_t newton_iters, double cg_tol,
                                double grad_tol, int64_t max_cg_iter, gvt_solve_info* info,
                                void* stream);

/*
 * Support vector machine with the squared hinge loss and a pairwise kernel (Sec. 7 names
 * support vector machines among the kernel methods the product speeds up), trained in the
 * primal by Newton's method over active sets (Chapelle 2007):
 *     J(a) = lambda a^T K a + sum_i max(0, 1 - y_i f_i)^2,   f = K a,  y_i = +-1.
 * With S = {i : y_i f_i < 1}, each Newton point solves (K_SS + lambda I) a_S = y_S with a = 0
 * outside S: kernel ridge regression (Eq. 1) on the active pairs, by FP64 CG to relative
 * residual cg_tol (at most max_cg_iter iterations) on a plan of those pairs.  A backtracking
 * line search halves the step toward it until J does not increase.  Stops when a full step
 * leaves S unchanged (the optimum) or after newton_iters steps.  FP64 products; M, N FP64 and
 * symmetric; a training plan.  y, a: device FP64 (a out; starts from zero).  info (may be
 * NULL): refinements = Newton steps, iterations = CG iterations in total, rel_residual =
 * ||lambda a + [y f < 1](f - y)|| / ||y|| (the gradient of J is 2 K times that vector).
 * Returns GVT_ERR_NOT_CONVERGED when newton_iters (or an inner max_cg_iter) ends the run,
 * with a holding the last iterate.
 */
gvt_status gvt_svm_newton_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                                const gvt_matrix* M, const gvt_matrix* N, const double* y,
                                double lambda, double* a, int32_t newton_iters, double cg_tol,
                                int64_t max_cg_iter, gvt_solve_info* info, void* stream);

/*
 * Support vector machine with the hinge loss by sub-gradient steps (Sec. 7 names
 * sub-gradient computations for support vector machines among the uses of the product):
 *     J(a) = (lambda / 2) a^T K a + (1 / n) sum_i max(0, 1 - y_i f_i),   f = K a,  y_i = +-1,
 * minimised by the kernelised Pegasos update (Shalev-Shwartz et al. 2011, every pair in every
 * step):  a <- (1 - 1/t) a + (1 / (lambda t n)) y [y f < 1],  then f = K a,  t = 1 .. iters.
 * One FP64 product per step.  M, N FP64 and symmetric; a training plan.  y, a: device FP64
 * (a out; starts from zero).  objective (host, may be NULL) receives J at the returned a.
 * info (may be NULL): iterations = iters.  The step count is the caller's choice: the
 * method converges as O(log t / (lambda t)) in J and has no exact stopping rule.
 */
gvt_status gvt_svm_subgradient_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                                     const gvt_matrix* M, const gvt_matrix* N, const double* y,
                                     double lambda, double* a, int64_t iters, double* objective,
                                     gvt_solve_info* info, void* stream);

/*
 * MINRES on the same system (the solver of Sec. 6, which stops it early):
 * Lanczos on K + lambda I from y with Givens rotations, so that the k-th iterate
 * minimises ||y - (K + lambda I) a|| over span{y, A y, ..., A^{k-1} y}.  One FP64
 * product per iteration; M, N FP64; the plan must be a training plan.
 * a (device, n FP64): out only -- MINRES starts from zero.  Stops when the
 * recursive residual norm reaches rel_tol * ||y|| or after max_iter steps.
 * record_every > 0: the iterate after step record_every * (j + 1) is copied to
 * column j of `records` (device, n x n_records FP64, column-major, caller-owned)
 * for j < n_records -- the candidates of early stopping on a validation set.
 * info (may be NULL): iterations, status, and rel_residual recomputed in FP64
 * from the returned a.  Synchronises `stream` once per iteration.  Returns
 * GVT_ERR_NOT_CONVERGED when max_iter ends the run (a holds the last iterate),
 * GVT_ERR_BREAKDOWN on a zero rotation norm.
 */
gvt_status gvt_krr_minres_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc,
                                const gvt_matrix* M, const gvt_matrix* N,
                                const double* y, double lambda, double* a, double rel_tol,
                                int64_t max_iter, int64_t record_every, int64_t n_records,
                                double* records, gvt_solve_info* info, void* stream);

/* ------------------------------------------------------------ learned preconditioner */

/*
 * A learned symmetric positive definite preconditioner P ~ (K + lambda I)^{-1}
 * for the training pairs of a plan.  A small MLP (6 -> 128 -> 128 -> 33, ReLU)
 * maps per-pair features -- the kernel diagonals M[d,d], N[t,t], log(1 + degree)
 * of the pair's drug and target, and the signed logs sign(x) log(1 + |x|) of the
 * kernel-graph degrees g1 = K 1 and g2 = K (g1 / mean g1) (two power-iteration
 * steps of the pairwise kernel matrix K), each normalised to zero mean and unit
 * deviation over the pairs -- to D_i = c softplus(o_0) and V_i = o_{1..32}
 * (c: a fixed output scale, see gvt_precond_scale);
 *     P r = S (I + V V^T)^{-1} S r,   S = diag(sqrt(D)),
 * a diagonal matrix minus a rank-32 term (Woodbury form), SPD for any network
 * output.  The paper solves with an unpreconditioned method (Sec. 6); this is
 * an addition used with flexible CG; the true FP64 residual still decides convergence.
 * Parameters: gvt_precond_num_params() floats, layout W1[128x6] b1[128]
 * W2[128x128] b2[128] W3[33x128] b3[33] (row-major), held in FP32.
 */
int64_t gvt_precond_num_params(void);

/* Arithmetic of the network's forward and backward passes: GVT_BF16 (the default: every layer
 * and backward product a tcgen05 GEMM on BF16 operands with FP32 accumulation; gradients
 * reproducible to rounding) or GVT_F32 (SIMT, FP32 throughout; bitwise reproducible).  The
 * low-rank algebra, the loss and the application of P are FP32/FP64 in both. */
gvt_status gvt_precond_set_dtype(gvt_precond* p, int32_t dtype);

/* Create for a training plan, the pairwise kernel `desc` and its FP64 kernel
 * matrices (the features need two products with K), with initial parameters
 * theta_host.  Synchronises. */
gvt_status gvt_precond_create(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                              const gvt_matrix* N, const float* theta_host, void* stream, gvt_precond** out);
gvt_status gvt_precond_destroy(gvt_precond* p);

/* Copy parameters to (set = 0) or from (set != 0) host memory.  Synchronises. */
gvt_status gvt_precond_params(gvt_precond* p, float* theta_host, int32_t set, void* stream);

/* Normalisation (host, 12 floats: mean[6], deviation[6]) and normalised
 * features (device, n x 6 row-major); either pointer may be NULL. */
gvt_status gvt_precond_features(gvt_precond* p, float* mu_sd_host, float* X_dev, void* stream);

/* Network outputs o (device, n x 33 row-major) for the current parameters. */
gvt_status gvt_precond_outputs(gvt_precond* p, float* O_dev, void* stream);

/* z = P r for device vectors of n elements, dtype GVT_F32 or GVT_F64. */
gvt_status gvt_precond_apply(gvt_precond* p, const void* r, void* z, int32_t dtype, void* stream);

/* Loss  L = (1/K) sum_k ||P r_k - e_k||^2 / ||e_k||^2  over K <= 16 pairs
 * (R, E: device FP32, n x K column-major) and its gradient with respect to the
 * parameters (host, num_params floats), by the library's forward and backward
 * kernels.  Either output may be NULL.  Synchronises. */
gvt_status gvt_precond_loss_grad(gvt_precond* p, const float* R, const float* E, int64_t K, double* loss_host,
                                 float* grad_host, void* stream);

/* Output scale c of D = c softplus(o_0): read into *get and/or set from *set
 * (either may be NULL).  The first gvt_precond_train call sets
 * c = sum e.e / sum r.e over its training pairs (the least-squares fit of
 * r ~ e / c, close to 1 / lambda). */
gvt_status gvt_precond_scale(gvt_precond* p, double* get, const double* set);

/* `steps` Adam steps (learning rate lr) on minibatches of `batch` <= 16
 * consecutive columns of the K_total pairs (R, E: device, n x K_total column-major,
 * stored as data_dtype GVT_F32 or GVT_BF16), cycling.
 * loss_history (host, may be NULL) receives each step's minibatch loss. */
gvt_status gvt_precond_train(gvt_precond* p, const void* R, const void* E, int32_t data_dtype, int64_t K_total,
                             int32_t steps, int32_t batch, double lr, double* loss_history, void* stream);

/*
 * Training data for the preconditioner from the exact solver: plain CG from a = 0 on
 * (K_desc + lambda I) a = y with the exact GVT product, in FP64 (op_dtype GVT_F64, M and N
 * FP64) or in FP32 (op_dtype GVT_F32, M and N FP32, the handle's engine: for problems where an
 * FP64 product costs too much); at the iterations listed in iters (host, ascending, `count` of
 * them) the residual r_k and the correction e_k = a_star - a_k (a_star: device FP64, the
 * converged solution) are stored as columns of R and E (device, n x count, store_dtype GVT_F32
 * or GVT_BF16).  Synchronises.
 */
gvt_status gvt_cg_record_pairs(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                               const gvt_matrix* N, const double* y, double lambda, const double* a_star,
                               const int64_t* iters, int64_t count, int32_t op_dtype, void* R, void* E,
                               int32_t store_dtype, void* stream);

/* ------------------------------------------------------------ batched solves */

/* One problem of a batched solve or product.  All pointers are device memory. */
typedef struct gvt_problem {
    int64_t m, q, n;          /* drugs, targets, training pairs; m * kc <= 25600 where kc is
                                 n_lambda rounded up to 4 (8, 16), q <= 65535 */
    const double* M;          /* m x m FP64 drug kernel, row-major (ld = m), symmetric */
    const double* N;          /* q x q FP64 target kernel, row-major (ld = q), symmetric */
    const int32_t* d;         /* n drug ids in [0, m) */
    const int32_t* t;         /* n target ids in [0, q) */
    const double* y;          /* n labels (solve only; may be NULL for the product) */
    double* a;                /* out: n x n_lambda dual coefficients, column c at a + c * n (solve
                                 only) */
} gvt_problem;

/*
 * Kernel ridge regression (Eq. 1) for many independent problems and
 * several regularisation values at once: for every problem b and every
 * lambda_c, (R_b (M_b kron N_b) R_b^T + lambda_c I) a_bc = y_b.
 * One persistent launch per stage covers the whole batch; each loaded kernel
 * entry serves all lambda columns.  Inner CG in FP32 (dot products summed in
 * FP32 over 8 elements per thread, then in FP64; step lengths in FP64), one
 * iteration captured as a CUDA graph; the outer loop
 * refines with FP64 residuals until every system reaches
 * ||y_b - (K_b + lambda_c I) a_bc|| / ||y_b|| <= opts->rel_tol.  The tile shape
 * of stage 1 is autotuned on the first call for a batch shape and cached in
 * the handle.  n_lambda in [1, 16].  rel_residuals (host, may be NULL)
 * receives the final FP64 relative residual of system (b, c) at
 * [b * n_lambda + c].  Synchronises `stream`.
 * The FP32 operator follows the handle's engine (gvt_set_stage1_engine):
 *  GVT_STAGE1_SIMT, GVT_STAGE1_TC_BF16X3 : SIMT stages for every problem.
 *  GVT_STAGES_AUTO, GVT_STAGES_TC_F16X1  : a problem whose K' (q and m rounded up to 64) is at most
 *      1536 runs both stages as tcgen05 GEMMs on FP16 hi/lo splits (FP32-class products) when a
 *      cost model at measured GB300 rates favours it: stage 1 S_b = N_b Vd_b^T with the lambda
 *      columns of the densified pair vectors as rows of Vd_b, stage 2 C_b = M_b S_b'^T with the
 *      (target, lambda) rows of S_b, and the sampled entries read out of C_b (multi-RHS: the
 *      kc columns share every left tile).  All such problems run in one grouped launch per stage,
 *      beside the SIMT stages of the others.  Needs the split operands and outputs in at most half
 *      of the free device memory, else every problem stays on the SIMT stages.
 *  GVT_STAGES_TC_F16X3 : as AUTO, but every problem that fits runs on the tensor cores.
 * The FP64 operator of the outer residuals always runs the SIMT stages.  Returns GVT_ERR_TIMEOUT
 * when a bounded wait of a tensor-core stage expired.
 */
gvt_status gvt_krr_cg_solve_batched(gvt_handle* h, const gvt_problem* probs, int64_t n_probs,
                                    const double* lambdas, int64_t n_lambda, const gvt_solve_opts* opts,
                                    double* rel_residuals, gvt_solve_info* info, void* stream);

/*
 * The FP32 operator of the batched solve on its own (Theorem 1 per problem, several vectors at
 * once): for every problem b and column c < n_cols,
 *   w_b[:, c] = R_b (M_b kron N_b) R_b^T v_b[:, c] + shifts[c] v_b[:, c].
 * v[b], w[b] (host arrays of device pointers): FP32, n_b x n_cols column-major (column c at
 * + c * n_b); may be NULL for a problem with n_b = 0.  shifts (host, finite; 0 for the plain
 * product).  The problems' y and a are not used.  n_cols in [1, 16].  Engines as for
 * gvt_krr_cg_solve_batched.  Prepares the batch on every call (packing, pair sorts, splits):
 * the solve amortises that set-up, this call does not.  Synchronises `stream`; GVT_ERR_TIMEOUT
 * as for the solve.
 */
gvt_status gvt_matvec_batched(gvt_handle* h, const gvt_problem* probs, int64_t n_probs, const double* shifts,
                              int64_t n_cols, const float* const* v, float* const* w, void* stream);

/* ------------------------------------------------------------ instrumentation */

/* Per-stage device time and algorithmic work of the products made with a
 * handle while statistics are enabled.  Each stage launch is bracketed by
 * CUDA events on its own stream. */
typedef enum gvt_stat_kind {
    GVT_STAT_STAGE1 = 0,     /* stage 1 as a whole, S = B W, whichever engine runs it */
    GVT_STAT_STAGE2 = 1,     /* stage 2 as a whole: the sampled dots */
    GVT_STAT_ONE_SIDED = 2,  /* one-sided terms: segment sums, GEMV, gather */
    GVT_STAT_TC_GEMM = 3,    /* the tcgen05 GEMM launches of the dense engines alone (also counted
                                inside their stage's record); flops = 2 M N K of the split GEMM */
    GVT_STAT_SPARSE_STAGE1 = 4,  /* the sparse scatter-accumulate kernel launches alone (also
                                    counted inside GVT_STAT_STAGE1) */
    GVT_STAT_SPARSE_STAGE2 = 5,  /* the sampled gather-dot kernel launches alone (also counted
                                    inside GVT_STAT_STAGE2) */
    GVT_STAT_COUNT = 6
} gvt_stat_kind;

typedef struct gvt_kernel_stats {
    int64_t launches;        /* launches recorded */
    double ms;               /* summed device time of those launches */
    double flops;            /* algorithmic flops (2 per multiply-add of the definition); for
                                GVT_STAT_TC_GEMM the executed flops 2 M N K of the GEMM */
    double bytes;            /* algorithmic bytes: each operand read once, each result written once */
    double useful_flops;     /* the method's own flops the launches carry: 2 qbar n (stage 1) or
                                2 m nhat (stage 2) per Kronecker term, counting only the pairs the
                                launch serves.  Equal to `flops` except for GVT_STAT_TC_GEMM, whose
                                dense GEMM does more than the sparse work it stands in for */
} gvt_kernel_stats;

/* Start (on != 0) or stop recording; starting clears the counters. */
gvt_status gvt_stats_enable(gvt_handle* h, int32_t on);
/* Fill out[0 .. GVT_STAT_COUNT-1].  Synchronises the recorded events. */
gvt_status gvt_stats_read(gvt_handle* h, gvt_kernel_stats* out);

/* Number of CUDA kernels this library has launched in this process. */
int64_t gvt_launch_count(void);

/* ------------------------------------------------------- allocation-free product */

/* Bytes of the fixed device scratch array behind gvt_matvec_static. */
#define GVT_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/*
 * u = R(dhat,that) (M kron N) R(d,t)^T v, like gvt_matvec, with no device
 * allocation, for callers that cannot allocate device memory: programs whose
 * framework owns all device memory through its own pool, or latency-bound
 * loops that may not call cudaMalloc / cudaFree (they can synchronise the
 * device).  The paper has no counterpart.
 *
 * It needs no handle and no plan and calls no allocating routine.  Its only
 * scratch (one error word and the q_rows x m_cols intermediate S of the
 * two-stage product) lives in a static __device__ array of
 * GVT_STATIC_SCRATCH_BYTES bytes, which every device that loads the library
 * holds until the process exits.  Requests with
 * q_rows * m_cols * element size > GVT_STATIC_SCRATCH_BYTES - 256 return
 * GVT_ERR_INVALID_ARG without launching anything (the check divides rather
 * than multiplies, so no declared size can wrap it).
 *
 *  - Arguments as for gvt_plan_create + gvt_matvec (device index arrays,
 *    d_out = t_out = NULL for the training operator), one column, dtype
 *    GVT_F64 or GVT_F32.  A symmetric N lets stage 1 read rows instead of
 *    columns.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it.  That first use may also load the
 *    library's device code on the device, which is when the driver reserves
 *    the array.
 *  - Every call synchronises `stream` (below), so no call can be captured
 *    into a CUDA graph.
 *  - Every call clears the parts of the array it uses; the array keeps the
 *    last call's contents otherwise.  All calls share the one array, so calls
 *    whose work overlaps on the GPU (different streams, other host threads)
 *    race and give wrong results: serialise them.
 *  - Stage 1 accumulates with atomic adds, so the summation order (and the
 *    last bits of u) can differ from gvt_matvec and between calls.
 *  - Indices are checked inside the kernels; pairs outside the kernel
 *    matrices are skipped and reported as GVT_ERR_INDEX_OOB.  The call
 *    synchronises `stream` to read that check.
 */
gvt_status gvt_matvec_static(int64_t m_rows, int64_t m_cols, int64_t q_rows, int64_t q_cols,
                             const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                             const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                             const gvt_matrix* M, const gvt_matrix* N, const void* v, void* u,
                             int32_t dtype, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GVT_H_ */
