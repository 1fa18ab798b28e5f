/*
 * Plain FP64 CPU oracle for pairwise-kernel matrix-vector products.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (the definition, not the fast algorithm):
 *   u_i = sum_j k((dhat_i, that_i), (d_j, t_j)) * v_j
 * with k evaluated entry by entry from the kernel-function table of the
 * paper (Table 4b, Sec. 4), on the entries of the base kernel matrices
 * M (drug kernel, the paper's D) and N (target kernel, the paper's T).
 * This is the "explicit kernel matrix" way of the product (Sec. 4.9,
 * approach 1), O(n * nhat); it never uses the sum-of-Kronecker
 * decomposition (Corollary 1), so every decomposition the GPU path uses is
 * checked against an independent derivation.
 *
 * Readings of the paper fixed here:
 *  - Anti-symmetric kernel: Table 4b's sign,
 *      k(d,dbar)k(d',dbar') - k(d,dbar')k(d',dbar),
 *    i.e. (I - P)(D x D); Corollary 1 prints (P - I), the negative.
 *  - Symmetric kernel: Table 4b, no 1/2 factor.
 *  - Gaussian base kernel: squared norm exp(-gamma*||x - x'||^2) (Sec. 5.2);
 *    Table 4b prints the unsquared norm, which would not factorise into the
 *    drug x target product that Sec. 4.3 asserts.
 *  - Homogeneous kernels (symmetric, anti-symmetric, ranking, MLPK) read
 *    both pair components through M: M[out_id, in_id].
 *  - Cartesian compares output and input ids directly (Setting 1 only).
 *
 * Sums use Neumaier's compensated summation.  Build with
 * -ffp-contract=off so that x86 and Arm give identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Kernel kinds, in the order of Table 4b. */
enum {
    ORC_KRONECKER = 0,
    ORC_GAUSSIAN = 1, /* Kronecker product of two Gaussian base kernels */
    ORC_LINEAR = 2,
    ORC_POLY2D = 3,
    ORC_CARTESIAN = 4,
    ORC_SYMMETRIC = 5,
    ORC_ANTISYMMETRIC = 6,
    ORC_RANKING = 7,
    ORC_MLPK = 8
};

typedef struct {
    const double* M; int64_t ldm;
    const double* N; int64_t ldn;
} orc_mats;

/* One pairwise kernel value k((a,b),(c,e)), Table 4b.
 * (a,b) is the output (row) pair, (c,e) the input (column) pair. */
static double orc_k_pair(int kind, const orc_mats* km,
                         int64_t a, int64_t b, int64_t c, int64_t e)
{
    const double* M = km->M;
    const double* N = km->N;
    const int64_t lm = km->ldm, ln = km->ldn;
    switch (kind) {
    case ORC_KRONECKER:
    case ORC_GAUSSIAN:
        /* k_D(d,dbar) k_T(t,tbar) */
        return M[a * lm + c] * N[b * ln + e];
    case ORC_LINEAR:
        /* k_D(d,dbar) + k_T(t,tbar) */
        return M[a * lm + c] + N[b * ln + e];
    case ORC_POLY2D: {
        /* (k_D(d,dbar) + k_T(t,tbar))^2, no bias */
        double s = M[a * lm + c] + N[b * ln + e];
        return s * s;
    }
    case ORC_CARTESIAN:
        /* k_D(d,dbar) delta(t = tbar) + delta(d = dbar) k_T(t,tbar) */
        return (b == e ? M[a * lm + c] : 0.0) + (a == c ? N[b * ln + e] : 0.0);
    case ORC_SYMMETRIC:
        /* k(d,dbar)k(d',dbar') + k(d,dbar')k(d',dbar) */
        return M[a * lm + c] * M[b * lm + e] + M[a * lm + e] * M[b * lm + c];
    case ORC_ANTISYMMETRIC:
        /* k(d,dbar)k(d',dbar') - k(d,dbar')k(d',dbar) */
        return M[a * lm + c] * M[b * lm + e] - M[a * lm + e] * M[b * lm + c];
    case ORC_RANKING:
        /* k(d,dbar) - k(d,dbar') - k(d',dbar) + k(d',dbar') */
        return M[a * lm + c] - M[a * lm + e] - M[b * lm + c] + M[b * lm + e];
    case ORC_MLPK: {
        /* ranking kernel squared */
        double r = M[a * lm + c] - M[a * lm + e] - M[b * lm + c] + M[b * lm + e];
        return r * r;
    }
    default:
        return NAN;
    }
}

/* Neumaier compensated accumulation: (*s, *comp) += x. */
static void orc_neumaier_add(double* s, double* comp, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x))
        *comp += (*s - t) + x;
    else
        *comp += (x - t) + *s;
    *s = t;
}

int orc_kernel_value(int kind, const double* M, int64_t ldm,
                     const double* N, int64_t ldn,
                     int64_t a, int64_t b, int64_t c, int64_t e, double* out)
{
    orc_mats km = {M, ldm, N, ldn};
    if (kind < ORC_KRONECKER || kind > ORC_MLPK) return 1;
    *out = orc_k_pair(kind, &km, a, b, c, e);
    return 0;
}

/*
 * Explicit kernel block  K[i, j] = k((dout_i, tout_i), (din_j, tin_j)),
 * row-major n_out x n_in:  R(dhat,that) K_op R(d,t)^T  (Sec. 2, Sec. 4.9).
 */
int orc_kernel_matrix(int kind, const double* M, int64_t ldm,
                      const double* N, int64_t ldn,
                      const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                      const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                      double* K)
{
    orc_mats km = {M, ldm, N, ldn};
    if (kind < ORC_KRONECKER || kind > ORC_MLPK) return 1;
    for (int64_t i = 0; i < n_out; ++i)
        for (int64_t j = 0; j < n_in; ++j)
            K[i * n_in + j] = orc_k_pair(kind, &km, d_out[i], t_out[i], d_in[j], t_in[j]);
    return 0;
}

/*
 * u = R(dhat,that) K_op R(d,t)^T v  for k_cols right-hand sides
 * (v: n_in x k_cols column-major, u: n_out x k_cols column-major).
 * The prediction product of Sec. 3 / Eq. (1) written out as the double sum.
 * nthreads <= 0 uses the OpenMP default.
 */
int orc_pairwise_matvec(int kind, const double* M, int64_t ldm,
                        const double* N, int64_t ldn,
                        const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                        const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                        const double* v, int64_t k_cols, double* u, int nthreads)
{
    orc_mats km = {M, ldm, N, ldn};
    if (kind < ORC_KRONECKER || kind > ORC_MLPK) return 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t i = 0; i < n_out; ++i) {
        for (int64_t c = 0; c < k_cols; ++c) {
            double s = 0.0, comp = 0.0;
            const double* vc = v + c * n_in;
            for (int64_t j = 0; j < n_in; ++j) {
                double kv = orc_k_pair(kind, &km, d_out[i], t_out[i], d_in[j], t_in[j]);
                orc_neumaier_add(&s, &comp, kv * vc[j]);
            }
            u[c * n_out + i] = s + comp;
        }
    }
    return 0;
}

/*
 * Gaussian base kernel  K[a, b] = exp(-gamma * ||X_a - Y_b||^2)
 * (Sec. 5.2, squared norm), X: rows_x x dim, Y: rows_y x dim, row-major.
 * The squared distance is the plain sum of squared differences.
 */
int orc_gaussian_kernel(const double* X, int64_t rows_x,
                        const double* Y, int64_t rows_y, int64_t dim,
                        double gamma, double* K, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t a = 0; a < rows_x; ++a) {
        for (int64_t b = 0; b < rows_y; ++b) {
            double s = 0.0, comp = 0.0;
            for (int64_t k = 0; k < dim; ++k) {
                double diff = X[a * dim + k] - Y[b * dim + k];
                orc_neumaier_add(&s, &comp, diff * diff);
            }
            K[a * rows_y + b] = exp(-gamma * (s + comp));
        }
    }
    return 0;
}

/* Neumaier sum of a vector, exposed so that tests can pin it. */
double orc_compensated_sum(const double* x, int64_t n)
{
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; ++i) orc_neumaier_add(&s, &comp, x[i]);
    return s + comp;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
