// Kernel logistic regression on pairwise kernels by Newton's method: another loss driven by
// the same GVT product (the paper's closing discussion, Sec. 7).
//
// Dual coefficients a, f = K a, labels y in {-1, +1}:
//   J(a) = sum_i log(1 + exp(-y_i f_i)) + (lambda / 2) a^T K a,
//   gradient K (g + lambda a), g_i = -y_i sigmoid(-y_i f_i),
//   Hessian  K (W K + lambda I), W = diag(s_i (1 - s_i)), s_i = sigmoid(y_i f_i).
// The Newton step d solves (W K + lambda I) d = b, b = -(g + lambda a), through the SPD system
//   (W^1/2 K W^1/2 + lambda I) c = W^1/2 K b,   d = (b - W^1/2 c) / lambda,
// solved by CG (one FP64 product per iteration); a backtracking line search on J halves the
// step until J decreases (J along the step needs only dot products and one product K d).
#include <chrono>
#include <cmath>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kKlBlocks = kRedGrid;
constexpr int kKlThreads = kRedBlock;

__device__ __forceinline__ double sigmoid_pos(double x) { return 0.5 * (1.0 + tanh(0.5 * x)); }

// s = sigmoid(y f), g = -y (1 - s), b = -(g + lam a), sw = sqrt(s (1 - s)); part[0] = ||b||^2
__global__ void __launch_bounds__(kKlThreads)
kl_prep(const double* __restrict__ f, const double* __restrict__ y, const double* __restrict__ a, double lam,
        int64_t n, double* __restrict__ b, double* __restrict__ sw, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = sigmoid_pos(y[i] * f[i]);
        const double g = -y[i] * (1.0 - s);
        const double bi = -(g + lam * a[i]);
        b[i] = bi;
        sw[i] = sqrt(s * (1.0 - s));
        acc += bi * bi;
    }
    block_sum_slot(acc, part, 0);
}

__global__ void kl_mul(const double* __restrict__ x, const double* __restrict__ sw, int64_t n, double* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = sw[i] * x[i];
}

// w = sw w + lam p; part = p . w
__global__ void __launch_bounds__(kKlThreads)
kl_shift_dot(double* __restrict__ w, const double* __restrict__ sw, const double* __restrict__ p, double lam,
             int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = sw[i] * w[i] + lam * p[i];
        w[i] = x;
        acc += p[i] * x;
    }
    block_sum_slot(acc, part, 0);
}

// c += alpha p, r -= alpha w; part = r . r
__global__ void __launch_bounds__(kKlThreads)
kl_cg_update(double* __restrict__ c, double* __restrict__ r, const double* __restrict__ p,
             const double* __restrict__ w, double alpha, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        c[i] += alpha * p[i];
        const double x = r[i] - alpha * w[i];
        r[i] = x;
        acc += x * x;
    }
    block_sum_slot(acc, part, 0);
}

__global__ void kl_pupdate(double* __restrict__ p, const double* __restrict__ r, double beta, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

// r = p = rhs, c = 0; part = rhs . rhs
__global__ void __launch_bounds__(kKlThreads)
kl_cg_init(const double* __restrict__ rhs, int64_t n, double* __restrict__ c, double* __restrict__ r,
           double* __restrict__ p, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = rhs[i];
        r[i] = x;
        p[i] = x;
        c[i] = 0.0;
        acc += x * x;
    }
    block_sum_slot(acc, part, 0);
}

// d = (b - sw c) / lam; part slots: 0 = d . f, 1 = a . f
__global__ void __launch_bounds__(kKlThreads)
kl_direction(const double* __restrict__ b, const double* __restrict__ sw, const double* __restrict__ c, double lam,
             const double* __restrict__ f, const double* __restrict__ a, int64_t n, double* __restrict__ d,
             double* __restrict__ part)
{
    double df = 0.0, af = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (b[i] - sw[i] * c[i]) / lam;
        d[i] = x;
        df += x * f[i];
        af += a[i] * f[i];
    }
    block_sum_slot(df, part, 0);
    block_sum_slot(af, part, 1);
}

// part slots: 0 = d . Kd, 1 = sum log(1 + exp(-y (f + t Kd)))
__global__ void __launch_bounds__(kKlThreads)
kl_line(const double* __restrict__ f, const double* __restrict__ Kd, const double* __restrict__ d,
        const double* __restrict__ y, double t, int64_t n, double* __restrict__ part)
{
    double dkd = 0.0, loss = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        dkd += d[i] * Kd[i];
        const double z = -y[i] * (f[i] + t * Kd[i]);
        loss += z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
    }
    block_sum_slot(dkd, part, 0);
    block_sum_slot(loss, part, 1);
}

__global__ void kl_step(double* __restrict__ a, double* __restrict__ f, const double* __restrict__ d,
                        const double* __restrict__ Kd, double t, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] += t * d[i];
        f[i] += t * Kd[i];
    }
}

gvt_status kl_sums(const double* part_dev, int slots, std::vector<double>& host, double* out, cudaStream_t s)
{
    return host_reduce(part_dev, slots, host, out, s);
}

}  // namespace
}  // namespace gvt

using namespace gvt;

extern "C" {

gvt_status gvt_klr_newton_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                const gvt_matrix* N, const double* y, double lambda, double* a, int32_t newton_iters,
                                double cg_tol, double grad_tol, int64_t max_cg_iter, gvt_solve_info* info_out,
                                void* stream)
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
    if (!h || !plan || !desc || !M || !M->data || (!desc->homogeneous && (!N || !N->data))) {
        set_error("gvt_klr_newton_solve: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in || !(lambda > 0.0) || newton_iters < 0 || !(cg_tol > 0.0) || !(grad_tol >= 0.0) ||
        max_cg_iter < 1) {
        set_error("gvt_klr_newton_solve: training plan, lambda > 0, cg_tol > 0, grad_tol >= 0 and counts >= 0 "
                  "are required");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (M->dtype != GVT_F64 || (!desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_klr_newton_solve: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    const int64_t n = plan->n_in;
    if (n > 0 && (!y || !a)) {
        set_error("gvt_klr_newton_solve: y or a is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n == 0) return ret(GVT_OK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gvt_matrix* Nn = desc->homogeneous ? M : N;

    Arena& ws = h->solve_ws;
    ws.reset();
    size_t off[10];
    for (int k = 0; k < 9; ++k) off[k] = ws.take(8 * n);
    off[9] = ws.take(8 * (size_t)kKlBlocks * 2);
    gvt_status st = ws.commit(s);
    if (st != GVT_OK) return ret(st);
    auto vec = [&](int k) { return reinterpret_cast<double*>(ws.base() + off[k]); };
    double *f = vec(0), *b = vec(1), *sw = vec(2), *c = vec(3), *r = vec(4), *p = vec(5), *w = vec(6),
           *d = vec(7), *Kd = vec(8);
    double* part = reinterpret_cast<double*>(ws.base() + off[9]);
    std::vector<double> ph((size_t)kKlBlocks * 2);
    const unsigned g = kKlBlocks;
    double sums[2];

    if ((st = vec_zero<double>(a, n, s)) != GVT_OK || (st = vec_zero<double>(f, n, s)) != GVT_OK) return ret(st);
    double yy = 0.0;   // ||y||^2 (cg_init's dot; its vector outputs are overwritten later)
    {
        kl_cg_init<<<g, kKlThreads, 0, s>>>(y, n, c, r, p, part);
        GVT_LAUNCHED(1, "klr init");
        if ((st = kl_sums(part, 1, ph, &yy, s)) != GVT_OK) return ret(st);
    }
    const double ynorm = std::sqrt(yy);
    if (ynorm == 0.0) return ret(GVT_OK);

    int32_t it = 0;
    int64_t cg_total = 0;
    double rel = INFINITY;
    gvt_status result = GVT_OK;
    while (true) {
        kl_prep<<<g, kKlThreads, 0, s>>>(f, y, a, lambda, n, b, sw, part);
        GVT_LAUNCHED(1, "klr gradient");
        double bb = 0.0;
        if ((st = kl_sums(part, 1, ph, &bb, s)) != GVT_OK) return ret(st);
        rel = std::sqrt(bb) / ynorm;
        if (rel <= grad_tol || it >= newton_iters) break;
        // rhs = sw * K b
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, b, w, s)) != GVT_OK) return ret(st);
        kl_mul<<<g, kKlThreads, 0, s>>>(w, sw, n, d);   // d holds the right-hand side for a moment
        kl_cg_init<<<g, kKlThreads, 0, s>>>(d, n, c, r, p, part);
        GVT_LAUNCHED(2, "klr cg init");
        double rr = 0.0;
        if ((st = kl_sums(part, 1, ph, &rr, s)) != GVT_OK) return ret(st);
        const double rnorm0 = std::sqrt(rr);
        int64_t k = 0;
        while (rnorm0 > 0.0 && std::sqrt(rr) > cg_tol * rnorm0 && k < max_cg_iter) {
            kl_mul<<<g, kKlThreads, 0, s>>>(p, sw, n, Kd);   // Kd as scratch: sw * p
            GVT_LAUNCHED(1, "klr cg");
            if ((st = pairwise_apply<double>(plan, desc, M, Nn, Kd, w, s)) != GVT_OK) return ret(st);
            kl_shift_dot<<<g, kKlThreads, 0, s>>>(w, sw, p, lambda, n, part);
            GVT_LAUNCHED(1, "klr cg");
            double pw = 0.0;
            if ((st = kl_sums(part, 1, ph, &pw, s)) != GVT_OK) return ret(st);
            if (!(pw > 0.0) || !std::isfinite(pw)) {
                set_error("klr: CG breakdown in the Newton system");
                return ret(GVT_ERR_BREAKDOWN);
            }
            const double alpha = rr / pw;
            kl_cg_update<<<g, kKlThreads, 0, s>>>(c, r, p, w, alpha, n, part);
            GVT_LAUNCHED(1, "klr cg");
            double rr_new = 0.0;
            if ((st = kl_sums(part, 1, ph, &rr_new, s)) != GVT_OK) return ret(st);
            kl_pupdate<<<g, kKlThreads, 0, s>>>(p, r, rr_new / rr, n);
            GVT_LAUNCHED(1, "klr cg");
            rr = rr_new;
            ++k;
        }
        cg_total += k;
        if (rnorm0 > 0.0 && std::sqrt(rr) > cg_tol * rnorm0) result = GVT_ERR_NOT_CONVERGED;
        // d = (b - sw c) / lambda, Kd = K d, then the line search on J
        kl_direction<<<g, kKlThreads, 0, s>>>(b, sw, c, lambda, f, a, n, d, part);
        GVT_LAUNCHED(1, "klr direction");
        if ((st = kl_sums(part, 2, ph, sums, s)) != GVT_OK) return ret(st);
        const double df = sums[0], af = sums[1];
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, d, Kd, s)) != GVT_OK) return ret(st);
        kl_line<<<g, kKlThreads, 0, s>>>(f, Kd, d, y, 0.0, n, part);
        GVT_LAUNCHED(1, "klr line search");
        if ((st = kl_sums(part, 2, ph, sums, s)) != GVT_OK) return ret(st);
        const double dkd = sums[0];
        const double J0 = sums[1] + 0.5 * lambda * af;
        double t = 1.0;
        while (t > 1e-12) {
            kl_line<<<g, kKlThreads, 0, s>>>(f, Kd, d, y, t, n, part);
            GVT_LAUNCHED(1, "klr line search");
            if ((st = kl_sums(part, 2, ph, sums, s)) != GVT_OK) return ret(st);
            const double Jt = sums[1] + 0.5 * lambda * (af + 2.0 * t * df + t * t * dkd);
            if (Jt <= J0) break;
            t *= 0.5;
        }
        kl_step<<<g, kKlThreads, 0, s>>>(a, f, d, Kd, t, n);
        GVT_LAUNCHED(1, "klr step");
        ++it;
    }
    info->refinements = it;
    info->iterations = cg_total;
    info->rel_residual = rel;
    if (result == GVT_OK && rel > grad_tol) {
        set_error("klr: newton_iters reached before grad_tol");
        result = GVT_ERR_NOT_CONVERGED;
    }
    return ret(result);
}

}  // extern "C"
