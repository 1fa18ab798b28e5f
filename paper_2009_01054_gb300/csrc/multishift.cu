// Multi-shift CG: (K + lambda_s I) a_s = y for a whole lambda sweep from one Krylov space.
//
// CG runs on the base system A = K + lambda_0 I (lambda_0 = min lambda_s), one FP64
// pairwise product per iteration.  For the shift sigma_s = lambda_s - lambda_0 the
// residual stays collinear with the base residual, r_s = zeta_s r, so every shift
// advances with scalar recurrences and two vector updates:
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} alpha_{k-1} (1 + sigma alpha_k))
//   alpha^s_k = alpha_k zeta_{k+1} / zeta_k,  beta^s_k = (zeta_{k+1} / zeta_k)^2 beta_k
//   a_s += alpha^s_k p_s,  p_s = zeta_{k+1} r_{k+1} + beta^s_k p_s
// A shift stops once |zeta_s| ||r|| <= rel_tol ||y||.  The scalar recurrences run on
// the host from block partial sums added in a fixed order (reproducible runs).
#include <chrono>
#include <cmath>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kMsBlocks = kRedGrid;
constexpr int kMsThreads = kRedBlock;
constexpr int kMaxShifts = 32;

struct ShiftCoefs {
    double alpha[kMaxShifts];
    double zeta[kMaxShifts];
    double beta[kMaxShifts];
    uint32_t active;   // bit s: shift s still updates
    int count;
};

__global__ void __launch_bounds__(kMsThreads)
ms_dot(const double* __restrict__ x, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * x[i];
    block_sum_slot(acc, part, 0);
}

// w += lambda_0 p; part = block sums of p . w
__global__ void __launch_bounds__(kMsThreads)
ms_shift_dot(double* __restrict__ w, const double* __restrict__ p, double lam0, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] + lam0 * p[i];
        w[i] = x;
        acc += p[i] * x;
    }
    block_sum_slot(acc, part, 0);
}

// r -= alpha w; part = block sums of r . r
__global__ void __launch_bounds__(kMsThreads)
ms_residual_update(double* __restrict__ r, const double* __restrict__ w, double alpha, int64_t n,
                   double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = r[i] - alpha * w[i];
        r[i] = x;
        acc += x * x;
    }
    block_sum_slot(acc, part, 0);
}

// every active shift: a_s += alpha_s p_s, p_s = zeta_s r + beta_s p_s; base p = r + beta p
__global__ void __launch_bounds__(kMsThreads)
ms_shift_update(ShiftCoefs c, const double* __restrict__ r, double beta, double* __restrict__ p,
                double* __restrict__ X, double* __restrict__ P, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = r[i];
        for (int s = 0; s < c.count; ++s) {
            if (!((c.active >> s) & 1u)) continue;
            const int64_t k = (int64_t)s * n + i;
            const double ps = P[k];
            X[k] += c.alpha[s] * ps;
            P[k] = c.zeta[s] * ri + c.beta[s] * ps;
        }
        p[i] = ri + beta * p[i];
    }
}

__global__ void ms_init(const double* __restrict__ y, int64_t n, int S, double* __restrict__ r,
                        double* __restrict__ p, double* __restrict__ X, double* __restrict__ P)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double yi = y[i];
        r[i] = yi;
        p[i] = yi;
        for (int s = 0; s < S; ++s) {
            X[(int64_t)s * n + i] = 0.0;
            P[(int64_t)s * n + i] = yi;
        }
    }
}

// part = block sums of ||y - w - lambda a||^2
__global__ void __launch_bounds__(kMsThreads)
ms_true_residual(const double* __restrict__ y, const double* __restrict__ w, const double* __restrict__ a,
                 double lam, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = y[i] - w[i] - lam * a[i];
        acc += e * e;
    }
    block_sum_slot(acc, part, 0);
}

gvt_status ms_sum(const double* part_dev, std::vector<double>& host, double* out, cudaStream_t s)
{
    return host_reduce(part_dev, 1, host, out, s);
}

}  // namespace
}  // namespace gvt

using namespace gvt;

extern "C" {

gvt_status gvt_krr_cg_solve_multishift(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                       const gvt_matrix* N, const double* y, const double* lambdas,
                                       int32_t n_lambda, double* A, double rel_tol, int64_t max_iter,
                                       double* rel_residuals, gvt_solve_info* info_out, void* stream)
{
    gvt_solve_info local{};
    gvt_solve_info* info = info_out ? info_out : &local;
    *info = gvt_solve_info{};
    const auto t0 = std::chrono::steady_clock::now();
    auto ret = [&](gvt_status st) {
        info->status = st;
        info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return st;
    };
    if (!h || !plan || !desc || !M || !M->data || (!desc->homogeneous && (!N || !N->data)) || !lambdas) {
        set_error("gvt_krr_cg_solve_multishift: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in) {
        set_error("gvt_krr_cg_solve_multishift: the plan must be a training plan");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n_lambda < 1 || n_lambda > kMaxShifts || !(rel_tol >= 0.0) || max_iter < 0) {
        set_error("gvt_krr_cg_solve_multishift: 1 <= n_lambda <= 32, rel_tol >= 0, max_iter >= 0");
        return ret(GVT_ERR_INVALID_ARG);
    }
    double lam0 = lambdas[0];
    for (int s = 0; s < n_lambda; ++s) {
        if (!(lambdas[s] > 0.0) || !std::isfinite(lambdas[s])) {
            set_error("gvt_krr_cg_solve_multishift: every lambda must be > 0");
            return ret(GVT_ERR_INVALID_ARG);
        }
        lam0 = std::min(lam0, lambdas[s]);
    }
    if (M->dtype != GVT_F64 || (!desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_krr_cg_solve_multishift: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    const int64_t n = plan->n_in;
    if (n > 0 && (!y || !A)) {
        set_error("gvt_krr_cg_solve_multishift: y or A is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n == 0) return ret(GVT_OK);
    const int S = n_lambda;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gvt_matrix* Nn = desc->homogeneous ? M : N;

    Arena& ws = h->solve_ws;
    ws.reset();
    const size_t o_r = ws.take(8 * n), o_p = ws.take(8 * n), o_w = ws.take(8 * n),
                 o_P = ws.take(8 * (size_t)n * S), o_part = ws.take(8 * kMsBlocks);
    gvt_status st = ws.commit(s);
    if (st != GVT_OK) return ret(st);
    char* base = ws.base();
    double* r = reinterpret_cast<double*>(base + o_r);
    double* p = reinterpret_cast<double*>(base + o_p);
    double* w = reinterpret_cast<double*>(base + o_w);
    double* P = reinterpret_cast<double*>(base + o_P);
    double* part = reinterpret_cast<double*>(base + o_part);
    std::vector<double> ph(kMsBlocks);
    const unsigned g = kMsBlocks;

    ms_init<<<g, kMsThreads, 0, s>>>(y, n, S, r, p, A, P);
    ms_dot<<<g, kMsThreads, 0, s>>>(y, n, part);
    GVT_LAUNCHED(2, "multishift init");
    double rr = 0.0;
    if ((st = ms_sum(part, ph, &rr, s)) != GVT_OK) return ret(st);
    const double ynorm = std::sqrt(rr);
    std::vector<double> sig(S), z_prev(S, 1.0), z(S, 1.0), res(S, 0.0);
    std::vector<bool> done(S, false);
    for (int k = 0; k < S; ++k) sig[k] = lambdas[k] - lam0;
    double alpha_prev = 1.0, beta_prev = 0.0;
    int64_t it = 0;
    gvt_status result = GVT_OK;
    while (ynorm > 0.0) {
        bool all = true;
        for (int k = 0; k < S; ++k) {
            const double e = std::fabs(z[k]) * std::sqrt(rr) / ynorm;
            if (!done[k] && (e <= rel_tol || it >= max_iter)) {
                done[k] = true;
                res[k] = e;
                if (e > rel_tol) result = GVT_ERR_NOT_CONVERGED;
            }
            all = all && done[k];
        }
        if (all) break;
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, p, w, s)) != GVT_OK) return ret(st);
        double pw = 0.0, rr_new = 0.0;
        ms_shift_dot<<<g, kMsThreads, 0, s>>>(w, p, lam0, n, part);
        GVT_LAUNCHED(1, "multishift step");
        if ((st = ms_sum(part, ph, &pw, s)) != GVT_OK) return ret(st);
        if (!(pw > 0.0) || !std::isfinite(pw)) {
            set_error("multi-shift CG breakdown: p^T (K + lambda I) p <= 0 or not finite");
            result = GVT_ERR_BREAKDOWN;
            break;
        }
        const double alpha = rr / pw;
        ms_residual_update<<<g, kMsThreads, 0, s>>>(r, w, alpha, n, part);
        GVT_LAUNCHED(1, "multishift step");
        if ((st = ms_sum(part, ph, &rr_new, s)) != GVT_OK) return ret(st);
        const double beta = rr_new / rr;
        ShiftCoefs c{};
        c.count = S;
        c.active = 0;
        std::vector<double> z_next(S);
        for (int k = 0; k < S; ++k) {
            if (done[k]) continue;
            const double den = alpha * beta_prev * (z_prev[k] - z[k]) + z_prev[k] * alpha_prev * (1.0 + sig[k] * alpha);
            z_next[k] = z[k] * z_prev[k] * alpha_prev / den;
            const double ratio = z_next[k] / z[k];
            c.alpha[k] = alpha * ratio;
            c.zeta[k] = z_next[k];
            c.beta[k] = ratio * ratio * beta;
            c.active |= 1u << k;
        }
        ms_shift_update<<<g, kMsThreads, 0, s>>>(c, r, beta, p, A, P, n);
        GVT_LAUNCHED(1, "multishift step");
        for (int k = 0; k < S; ++k)
            if (!done[k]) {
                z_prev[k] = z[k];
                z[k] = z_next[k];
            }
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta;
        ++it;
    }
    info->iterations = it;
    // FP64 residual of every returned solution, recomputed
    double worst = 0.0;
    for (int k = 0; k < S; ++k) {
        const double* a = A + (int64_t)k * n;
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, a, w, s)) != GVT_OK) return ret(st);
        ms_true_residual<<<g, kMsThreads, 0, s>>>(y, w, a, lambdas[k], n, part);
        GVT_LAUNCHED(1, "multishift residual");
        double e2 = 0.0;
        if ((st = ms_sum(part, ph, &e2, s)) != GVT_OK) return ret(st);
        const double e = ynorm > 0.0 ? std::sqrt(e2) / ynorm : 0.0;
        if (rel_residuals) rel_residuals[k] = e;
        worst = std::max(worst, e);
    }
    info->rel_residual = worst;
    if (result == GVT_ERR_NOT_CONVERGED) set_error("multi-shift CG: max_iter reached before rel_tol");
    return ret(result);
}

}  // extern "C"
