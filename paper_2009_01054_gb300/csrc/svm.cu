// Support vector machine with the squared hinge loss on pairwise kernels, by Newton's method over
// active sets: another regularised kernel method driven by the same GVT product (the paper's
// closing discussion, Sec. 7), following Chapelle's primal training ("Training a support vector
// machine in the primal", 2007) in the coefficients a of the representer theorem:
//   J(a) = lambda a^T K a + sum_i max(0, 1 - y_i f_i)^2,   f = K a,  y_i in {-1, +1}.
// On the active set S = {i : y_i f_i < 1} the loss is (y_i - f_i)^2, so the Newton point a+ solves
//   (K_SS + lambda I) a+_S = y_S,   a+ = 0 outside S,
// a kernel ridge regression (Eq. 1) on the active pairs, solved by FP64 CG on a plan of those
// pairs.  A backtracking line search halves the step from a toward a+ until J does not increase
// (along the step f moves linearly, so J needs only dot products).  The solution is reached when
// a full step leaves S unchanged.
//
// The hinge loss is served by sub-gradient steps instead (the kernelised Pegasos update of
// Shalev-Shwartz et al., 2011, without sampling):
//   J(a) = (lambda / 2) a^T K a + (1 / n) sum_i max(0, 1 - y_i f_i),
//   a <- (1 - 1/t) a + (1 / (lambda t n)) y [y f < 1],   f = K a,   t = 1, 2, ...
// one product per step.
#include <chrono>
#include <cmath>
#include <cstdint>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kSvBlocks = kRedGrid;
constexpr int kSvThreads = kRedBlock;

unsigned sv_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// flag_i = y_i f_i < 1
__global__ void sv_flags(const double* __restrict__ f, const double* __restrict__ y, int64_t n,
                         uint8_t* __restrict__ flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = y[i] * f[i] < 1.0 ? 1 : 0;
}

// the active pairs and their labels: dS = d[idx], tS = t[idx], yS = y[idx], bS = 0
__global__ void sv_gather(const int32_t* __restrict__ idx, int64_t ns, const int32_t* __restrict__ d,
                          const int32_t* __restrict__ t, const double* __restrict__ y, int32_t* __restrict__ dS,
                          int32_t* __restrict__ tS, double* __restrict__ yS, double* __restrict__ bS)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = idx[k];
        dS[k] = d[i];
        tS[k] = t[i];
        yS[k] = y[i];
        bS[k] = 0.0;
    }
}

__global__ void sv_zero(double* __restrict__ x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.0;
}

// a+[idx[k]] = bS[k]
__global__ void sv_scatter(const int32_t* __restrict__ idx, int64_t ns, const double* __restrict__ bS,
                           double* __restrict__ ap)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += (int64_t)gridDim.x * blockDim.x)
        ap[idx[k]] = bS[k];
}

// slots: 0 = a . f, 1 = a . (f+ - f), 2 = (a+ - a) . f, 3 = (a+ - a) . (f+ - f),
//        4 = sum_i max(0, 1 - y_i f_i)^2 (the loss at the current point)
__global__ void __launch_bounds__(kSvThreads)
sv_dots(const double* __restrict__ a, const double* __restrict__ f, const double* __restrict__ ap,
        const double* __restrict__ fp, const double* __restrict__ y, int64_t n, double* __restrict__ part)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = ap[i] - a[i], df = fp[i] - f[i];
        s0 += a[i] * f[i];
        s1 += a[i] * df;
        s2 += d * f[i];
        s3 += d * df;
        const double m = 1.0 - y[i] * f[i];
        if (m > 0.0) s4 += m * m;
    }
    block_sum_slot(s0, part, 0);
    block_sum_slot(s1, part, 1);
    block_sum_slot(s2, part, 2);
    block_sum_slot(s3, part, 3);
    block_sum_slot(s4, part, 4);
}

// slot 0 = sum_i max(0, 1 - y_i (f_i + t (f+_i - f_i)))^2
__global__ void __launch_bounds__(kSvThreads)
sv_loss(const double* __restrict__ f, const double* __restrict__ fp, const double* __restrict__ y, double t,
        int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = 1.0 - y[i] * (f[i] + t * (fp[i] - f[i]));
        if (m > 0.0) acc += m * m;
    }
    block_sum_slot(acc, part, 0);
}

// a += t (a+ - a), f += t (f+ - f)
__global__ void sv_step(double* __restrict__ a, double* __restrict__ f, const double* __restrict__ ap,
                        const double* __restrict__ fp, double t, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] += t * (ap[i] - a[i]);
        f[i] += t * (fp[i] - f[i]);
    }
}

// slot 0 = ||lambda a + [y f < 1] (f - y)||^2, the coefficient-space gradient of J (up to 2 K);
// slot 1 = ||y||^2
__global__ void __launch_bounds__(kSvThreads)
sv_grad(const double* __restrict__ a, const double* __restrict__ f, const double* __restrict__ y, double lam,
        int64_t n, double* __restrict__ part)
{
    double acc = 0.0, yy = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double g = lam * a[i] + (y[i] * f[i] < 1.0 ? f[i] - y[i] : 0.0);
        acc += g * g;
        yy += y[i] * y[i];
    }
    block_sum_slot(acc, part, 0);
    block_sum_slot(yy, part, 1);
}

// one sub-gradient step of the hinge SVM: a = (1 - 1/t) a + c y [y f < 1], c = 1 / (lambda t n)
__global__ void sg_step(double* __restrict__ a, const double* __restrict__ f, const double* __restrict__ y,
                        double keep, double c, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = keep * a[i] + (y[i] * f[i] < 1.0 ? c * y[i] : 0.0);
}

// slot 0 = a . f, slot 1 = sum_i max(0, 1 - y_i f_i)
__global__ void __launch_bounds__(kSvThreads)
sg_objective(const double* __restrict__ a, const double* __restrict__ f, const double* __restrict__ y, int64_t n,
             double* __restrict__ part)
{
    double af = 0.0, loss = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        af += a[i] * f[i];
        loss += fmax(0.0, 1.0 - y[i] * f[i]);
    }
    block_sum_slot(af, part, 0);
    block_sum_slot(loss, part, 1);
}

}  // namespace
}  // namespace gvt

using namespace gvt;

extern "C" {

gvt_status gvt_svm_newton_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                const gvt_matrix* N, const double* y, double lambda, double* a, int32_t newton_iters,
                                double cg_tol, int64_t max_cg_iter, gvt_solve_info* info_out, void* stream)
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
        set_error("gvt_svm_newton_solve: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in || !(lambda > 0.0) || newton_iters < 0 || !(cg_tol > 0.0) || max_cg_iter < 1) {
        set_error("gvt_svm_newton_solve: training plan, lambda > 0, cg_tol > 0 and counts >= 0 are required");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (M->dtype != GVT_F64 || (!desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_svm_newton_solve: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    const int64_t n = plan->n_in;
    if (n > 0 && (!y || !a)) {
        set_error("gvt_svm_newton_solve: y or a is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n == 0) return ret(GVT_OK);
    if (n > INT32_MAX) {
        set_error("gvt_svm_newton_solve: more than 2^31 - 1 pairs");
        return ret(GVT_ERR_UNSUPPORTED);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gvt_matrix* Nn = desc->homogeneous ? M : N;

    // device vectors: f, a+, f+, y_S, b_S (FP64); d_S, t_S, idx (int32); flags; partial sums
    DevBuf bf, bap, bfp, byS, bbS, bdS, btS, bidx, bflag, bpart;
    gvt_status st;
    if ((st = bf.reserve(8 * (size_t)n, s)) != GVT_OK || (st = bap.reserve(8 * (size_t)n, s)) != GVT_OK ||
        (st = bfp.reserve(8 * (size_t)n, s)) != GVT_OK || (st = byS.reserve(8 * (size_t)n, s)) != GVT_OK ||
        (st = bbS.reserve(8 * (size_t)n, s)) != GVT_OK || (st = bdS.reserve(4 * (size_t)n, s)) != GVT_OK ||
        (st = btS.reserve(4 * (size_t)n, s)) != GVT_OK || (st = bidx.reserve(4 * (size_t)n, s)) != GVT_OK ||
        (st = bflag.reserve((size_t)n, s)) != GVT_OK || (st = bpart.reserve(8 * (size_t)kSvBlocks * 5, s)) != GVT_OK)
        return ret(st);
    double *f = static_cast<double*>(bf.ptr), *ap = static_cast<double*>(bap.ptr), *fp = static_cast<double*>(bfp.ptr);
    double *yS = static_cast<double*>(byS.ptr), *bS = static_cast<double*>(bbS.ptr);
    int32_t *dS = static_cast<int32_t*>(bdS.ptr), *tS = static_cast<int32_t*>(btS.ptr);
    int32_t* idx = static_cast<int32_t*>(bidx.ptr);
    uint8_t* flag = static_cast<uint8_t*>(bflag.ptr);
    double* part = static_cast<double*>(bpart.ptr);
    const unsigned g = sv_grid(n);
    std::vector<double> ph((size_t)kSvBlocks * 5);
    double sums[5];

    sv_zero<<<g, 256, 0, s>>>(a, n);
    sv_zero<<<g, 256, 0, s>>>(f, n);
    GVT_LAUNCHED(2, "svm init");

    gvt_solve_opts opts;
    gvt_solve_opts_default(&opts);
    opts.mode = GVT_SOLVE_FP64_CG;
    opts.rel_tol = cg_tol;
    opts.max_iter = max_cg_iter;

    std::vector<uint8_t> S(n), S_prev;
    std::vector<int32_t> hidx;
    bool full_prev = false, converged = false;
    int32_t it = 0;
    int64_t cg_total = 0;
    gvt_status result = GVT_OK;
    for (;; ++it) {
        sv_flags<<<g, 256, 0, s>>>(f, y, n, flag);
        GVT_LAUNCHED(1, "svm active set");
        if (cudaMemcpyAsync(S.data(), flag, (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "svm active set"));
        if (!S_prev.empty() && full_prev && S == S_prev) {
            converged = true;
            break;
        }
        if (it >= newton_iters) break;
        hidx.clear();
        for (int64_t i = 0; i < n; ++i)
            if (S[i]) hidx.push_back((int32_t)i);
        const int64_t ns = (int64_t)hidx.size();
        sv_zero<<<g, 256, 0, s>>>(ap, n);
        GVT_LAUNCHED(1, "svm newton point");
        if (ns > 0) {
            if (cudaMemcpyAsync(idx, hidx.data(), 4 * (size_t)ns, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return ret(cuda_fail(cudaGetLastError(), "svm active pairs"));
            sv_gather<<<sv_grid(ns), 256, 0, s>>>(idx, ns, plan->d_in, plan->t_in, y, dS, tS, yS, bS);
            GVT_LAUNCHED(1, "svm active pairs");
            // the Newton point: kernel ridge regression on the active pairs
            gvt_plan* sp = nullptr;
            if ((st = gvt_plan_create(h, plan->m_rows, plan->m_cols, plan->q_rows, plan->q_cols, dS, tS, ns, nullptr,
                                      nullptr, 0, stream, &sp)) != GVT_OK)
                return ret(st);
            gvt_solve_info si{};
            st = gvt_krr_cg_solve(h, sp, desc, M, N, yS, lambda, bS, &opts, &si, stream);
            gvt_plan_destroy(sp);
            cg_total += si.iterations;
            if (st == GVT_ERR_NOT_CONVERGED) result = GVT_ERR_NOT_CONVERGED;
            else if (st != GVT_OK) return ret(st);
            sv_scatter<<<sv_grid(ns), 256, 0, s>>>(idx, ns, bS, ap);
            GVT_LAUNCHED(1, "svm newton point");
        }
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, ap, fp, s)) != GVT_OK) return ret(st);
        // line search: J(t) = lambda (a + t d).(f + t df) + loss(t), d = a+ - a, df = f+ - f
        sv_dots<<<kSvBlocks, kSvThreads, 0, s>>>(a, f, ap, fp, y, n, part);
        GVT_LAUNCHED(1, "svm line search");
        if ((st = host_reduce(part, 5, ph, sums, s)) != GVT_OK) return ret(st);
        const double af = sums[0], adf = sums[1], dfv = sums[2], ddf = sums[3];
        const double J0 = lambda * af + sums[4];
        double t = 1.0;
        while (t > 1e-12) {
            sv_loss<<<kSvBlocks, kSvThreads, 0, s>>>(f, fp, y, t, n, part);
            GVT_LAUNCHED(1, "svm line search");
            double loss = 0.0;
            if ((st = host_reduce(part, 1, ph, &loss, s)) != GVT_OK) return ret(st);
            const double Jt = lambda * (af + t * (adf + dfv) + t * t * ddf) + loss;
            if (Jt <= J0) break;
            t *= 0.5;
        }
        sv_step<<<g, 256, 0, s>>>(a, f, ap, fp, t, n);
        GVT_LAUNCHED(1, "svm step");
        S_prev = S;
        full_prev = t == 1.0;
    }
    sv_grad<<<kSvBlocks, kSvThreads, 0, s>>>(a, f, y, lambda, n, part);
    GVT_LAUNCHED(1, "svm gradient");
    double gs[2];
    if ((st = host_reduce(part, 2, ph, gs, s)) != GVT_OK) return ret(st);
    const double ynorm = std::sqrt(gs[1]);
    info->refinements = it;
    info->iterations = cg_total;
    info->rel_residual = ynorm > 0.0 ? std::sqrt(gs[0]) / ynorm : 0.0;
    if (result == GVT_OK && !converged) {
        set_error("svm: newton_iters reached before the active set settled");
        result = GVT_ERR_NOT_CONVERGED;
    }
    return ret(result);
}

gvt_status gvt_svm_subgradient_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                     const gvt_matrix* N, const double* y, double lambda, double* a, int64_t iters,
                                     double* objective, gvt_solve_info* info_out, void* stream)
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
        set_error("gvt_svm_subgradient_solve: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in || !(lambda > 0.0) || iters < 0) {
        set_error("gvt_svm_subgradient_solve: training plan, lambda > 0 and iters >= 0 are required");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (M->dtype != GVT_F64 || (!desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_svm_subgradient_solve: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    const int64_t n = plan->n_in;
    if (n > 0 && (!y || !a)) {
        set_error("gvt_svm_subgradient_solve: y or a is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (objective) *objective = 0.0;
    if (n == 0) return ret(GVT_OK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gvt_matrix* Nn = desc->homogeneous ? M : N;
    DevBuf bf, bpart;
    gvt_status st;
    if ((st = bf.reserve(8 * (size_t)n, s)) != GVT_OK || (st = bpart.reserve(8 * (size_t)kSvBlocks * 2, s)) != GVT_OK)
        return ret(st);
    double* f = static_cast<double*>(bf.ptr);
    double* part = static_cast<double*>(bpart.ptr);
    const unsigned g = sv_grid(n);
    sv_zero<<<g, 256, 0, s>>>(a, n);
    sv_zero<<<g, 256, 0, s>>>(f, n);
    GVT_LAUNCHED(2, "hinge svm init");
    for (int64_t t = 1; t <= iters; ++t) {
        sg_step<<<g, 256, 0, s>>>(a, f, y, 1.0 - 1.0 / (double)t, 1.0 / (lambda * (double)t * (double)n), n);
        GVT_LAUNCHED(1, "hinge svm step");
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, a, f, s)) != GVT_OK) return ret(st);
    }
    sg_objective<<<kSvBlocks, kSvThreads, 0, s>>>(a, f, y, n, part);
    GVT_LAUNCHED(1, "hinge svm objective");
    std::vector<double> ph((size_t)kSvBlocks * 2);
    double sums[2];
    if ((st = host_reduce(part, 2, ph, sums, s)) != GVT_OK) return ret(st);
    if (objective) *objective = 0.5 * lambda * sums[0] + sums[1] / (double)n;
    info->iterations = iters;
    return ret(GVT_OK);
}

}  // extern "C"
