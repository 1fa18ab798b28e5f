// MINRES for the kernel ridge system (K + lambda I) a = y: the solver of Sec. 6.
//
// Lanczos on A = K + lambda I started from y (each step one FP64 pairwise product),
// with the tridiagonal T_k reduced by Givens rotations; a_k minimises ||y - A a||
// over the Krylov space K_k(A, y), and |phibar_k| = ||y - A a_k||.  The device
// holds the vectors; the O(1) rotation recurrences run on the host from two dot
// products per step (block partial sums added on the host in a fixed order, so
// runs are reproducible).  Iterates can be written out every `record_every`
// steps, for early stopping on a validation set (the paper stops MINRES early).
#include <chrono>
#include <cmath>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kMrBlocks = kRedGrid;
constexpr int kMrThreads = kRedBlock;

// w = w + lambda v - beta v_prev; part = block sums of v . w
__global__ void __launch_bounds__(kMrThreads)
mr_shift_dot(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ v_prev, double lam,
             double beta, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] + lam * v[i] - beta * v_prev[i];
        w[i] = x;
        acc += v[i] * x;
    }
    block_sum_slot(acc, part, 0);
}

// w -= alpha v; part = block sums of w . w
__global__ void __launch_bounds__(kMrThreads)
mr_axpy_norm(double* __restrict__ w, const double* __restrict__ v, double alpha, int64_t n,
             double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] - alpha * v[i];
        w[i] = x;
        acc += x * x;
    }
    block_sum_slot(acc, part, 0);
}

// d_k = (v - delta d1 - eps d2) / gamma into d2; a += tau d_k; w *= 1 / beta_next (v_{k+1})
__global__ void __launch_bounds__(kMrThreads)
mr_update(const double* __restrict__ v, double* __restrict__ w, const double* __restrict__ d1,
          double* __restrict__ d2, double* __restrict__ a, double delta, double eps, double inv_gamma, double tau,
          double inv_beta_next, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (v[i] - delta * d1[i] - eps * d2[i]) * inv_gamma;
        d2[i] = d;
        a[i] += tau * d;
        w[i] *= inv_beta_next;
    }
}

// r = y - w - lambda a; part = block sums of r . r
__global__ void __launch_bounds__(kMrThreads)
mr_residual(const double* __restrict__ y, const double* __restrict__ w, const double* __restrict__ a, double lam,
            int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = y[i] - w[i] - lam * a[i];
        acc += r * r;
    }
    block_sum_slot(acc, part, 0);
}

__global__ void mr_scale(const double* __restrict__ x, double s, int64_t n, double* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = s * x[i];
}

__global__ void mr_dot(const double* __restrict__ x, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * x[i];
    block_sum_slot(acc, part, 0);
}

gvt_status host_sum(const double* part_dev, std::vector<double>& part_host, double* out, cudaStream_t s)
{
    return host_reduce(part_dev, 1, part_host, out, s);
}

}  // namespace

gvt_status host_reduce(const double* part_dev, int slots, std::vector<double>& host, double* out, cudaStream_t s)
{
    if (host.size() < (size_t)kRedGrid * slots) host.resize((size_t)kRedGrid * slots);
    GVT_CUDA(cudaMemcpyAsync(host.data(), part_dev, sizeof(double) * kRedGrid * slots, cudaMemcpyDeviceToHost, s));
    GVT_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < slots; ++k) {
        double t = 0.0;
        for (int b = 0; b < kRedGrid; ++b) t += host[(size_t)k * kRedGrid + b];
        out[k] = t;
    }
    return GVT_OK;
}

}  // namespace gvt

using namespace gvt;

extern "C" {

gvt_status gvt_krr_minres_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                const gvt_matrix* N, const double* y, double lambda, double* a, double rel_tol,
                                int64_t max_iter, int64_t record_every, int64_t n_records, double* records,
                                gvt_solve_info* info_out, void* stream)
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
        set_error("gvt_krr_minres_solve: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in) {
        set_error("gvt_krr_minres_solve: the plan must be a training plan (output pairs = input pairs)");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!(lambda > 0.0) || !(rel_tol >= 0.0) || max_iter < 0 || record_every < 0 || n_records < 0 ||
        (record_every > 0 && n_records > 0 && !records)) {
        set_error("gvt_krr_minres_solve: lambda > 0, rel_tol >= 0, counts >= 0 and a records buffer are required");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (M->dtype != GVT_F64 || (!desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_krr_minres_solve: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    const int64_t n = plan->n_in;
    if (n > 0 && (!y || !a)) {
        set_error("gvt_krr_minres_solve: y or a is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n == 0) return ret(GVT_OK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gvt_matrix* Nn = desc->homogeneous ? M : N;

    Arena& ws = h->solve_ws;
    ws.reset();
    const size_t o_vp = ws.take(8 * n), o_v = ws.take(8 * n), o_w = ws.take(8 * n), o_d1 = ws.take(8 * n),
                 o_d2 = ws.take(8 * n), o_part = ws.take(8 * kMrBlocks);
    gvt_status st = ws.commit(s);
    if (st != GVT_OK) return ret(st);
    char* base = ws.base();
    double* vp = reinterpret_cast<double*>(base + o_vp);
    double* v = reinterpret_cast<double*>(base + o_v);
    double* w = reinterpret_cast<double*>(base + o_w);
    double* d1 = reinterpret_cast<double*>(base + o_d1);
    double* d2 = reinterpret_cast<double*>(base + o_d2);
    double* part = reinterpret_cast<double*>(base + o_part);
    std::vector<double> ph(kMrBlocks);
    const unsigned g = kMrBlocks;

    // beta_1 = ||y||, v_1 = y / beta_1, a = 0
    double yy = 0.0;
    mr_dot<<<g, kMrThreads, 0, s>>>(y, n, part);
    GVT_LAUNCHED(1, "minres init");
    if ((st = host_sum(part, ph, &yy, s)) != GVT_OK) return ret(st);
    const double beta1 = std::sqrt(yy);
    if ((st = vec_zero<double>(a, n, s)) != GVT_OK || (st = vec_zero<double>(vp, n, s)) != GVT_OK ||
        (st = vec_zero<double>(d1, n, s)) != GVT_OK || (st = vec_zero<double>(d2, n, s)) != GVT_OK)
        return ret(st);
    if (beta1 == 0.0) return ret(GVT_OK);
    mr_scale<<<g, kMrThreads, 0, s>>>(y, 1.0 / beta1, n, v);
    GVT_LAUNCHED(1, "minres init");

    double beta = 0.0, phibar = beta1;
    double c2 = 1.0, s2 = 0.0, c1 = 1.0, s1 = 0.0;
    int64_t k = 0, rec = 0;
    gvt_status result = GVT_OK;
    while (k < max_iter && std::fabs(phibar) / beta1 > rel_tol) {
        ++k;
        if ((st = pairwise_apply<double>(plan, desc, M, Nn, v, w, s)) != GVT_OK) return ret(st);
        double alpha = 0.0, bb = 0.0;
        mr_shift_dot<<<g, kMrThreads, 0, s>>>(w, v, vp, lambda, beta, n, part);
        GVT_LAUNCHED(1, "minres lanczos");
        if ((st = host_sum(part, ph, &alpha, s)) != GVT_OK) return ret(st);
        mr_axpy_norm<<<g, kMrThreads, 0, s>>>(w, v, alpha, n, part);
        GVT_LAUNCHED(1, "minres lanczos");
        if ((st = host_sum(part, ph, &bb, s)) != GVT_OK) return ret(st);
        const double beta_next = std::sqrt(bb);
        // rotations k-2 and k-1 on column k of T, then rotation k removes beta_{k+1}
        const double eps = s2 * beta, dprime = c2 * beta;
        const double delta = c1 * dprime + s1 * alpha;
        const double gbar = -s1 * dprime + c1 * alpha;
        const double gamma = std::hypot(gbar, beta_next);
        if (!(gamma > 0.0) || !std::isfinite(gamma)) {
            set_error("MINRES breakdown: zero or non-finite rotation norm");
            result = GVT_ERR_BREAKDOWN;
            break;
        }
        const double c = gbar / gamma, sn = beta_next / gamma;
        const double tau = c * phibar;
        phibar = -sn * phibar;
        mr_update<<<g, kMrThreads, 0, s>>>(v, w, d1, d2, a, delta, eps, 1.0 / gamma, tau,
                                            beta_next > 0.0 ? 1.0 / beta_next : 0.0, n);
        GVT_LAUNCHED(1, "minres update");
        if (record_every > 0 && k % record_every == 0 && rec < n_records) {
            GVT_CUDA(cudaMemcpyAsync(records + rec * n, a, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            ++rec;
        }
        std::swap(d1, d2);            // d_{k-1} <- d_k, d_{k-2} <- d_{k-1}
        c2 = c1; s2 = s1; c1 = c; s1 = sn;
        if (beta_next == 0.0) break;  // invariant Krylov space: a_k is exact
        double* t = vp;               // v_{k-1} <- v_k, v_k <- v_{k+1} (in w), w <- free
        vp = v;
        v = w;
        w = t;
        beta = beta_next;
    }
    info->iterations = k;
    // true FP64 residual of the returned iterate
    if ((st = pairwise_apply<double>(plan, desc, M, Nn, a, w, s)) != GVT_OK) return ret(st);
    mr_residual<<<g, kMrThreads, 0, s>>>(y, w, a, lambda, n, part);
    GVT_LAUNCHED(1, "minres residual");
    double rr = 0.0;
    if ((st = host_sum(part, ph, &rr, s)) != GVT_OK) return ret(st);
    info->rel_residual = std::sqrt(rr) / beta1;
    if (result == GVT_OK && std::fabs(phibar) / beta1 > rel_tol) {
        set_error("MINRES: max_iter reached before rel_tol");
        result = GVT_ERR_NOT_CONVERGED;
    }
    return ret(result);
}

}  // extern "C"
