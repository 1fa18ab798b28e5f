// Kernel ridge regression (Eq. 1) by conjugate gradients on
// top of the GVT products: plain FP64 CG, and mixed-precision iterative
// refinement (FP64 residual and correction, FP32 operator and vectors inside,
// FP64 dot products and step lengths everywhere).
//
// Scalars live on the device; a CG iteration is
//   w = K p (GVT), w += lambda p, pw = p.w        (fused shift + dot)
//   alpha = rr / pw                               (one block)
//   a += alpha p, r -= alpha w, rr' = r.r         (fused update + dot)
//   beta = rr' / rr                               (one block)
//   p = r + beta p
// Dot products reduce in FP64 in a fixed order (per-block partials, then one
// block), so a run is bitwise reproducible.  The iterations run on a stream the
// handle owns, joined to the caller's by events; in steady state blocks of
// iterations replay from a CUDA graph (the launches of small problems are then
// no longer separated by the host's launch gaps).
#include <cuda_bf16.h>

#include <chrono>
#include <cmath>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

enum Scal { SC_RR = 0, SC_PW, SC_ALPHA, SC_BETA, SC_FLAG, SC_RR0, SC_TMP, SC_RZ, SC_ZW, SC_COUNT };

__device__ double block_sum(double x)
{
    __shared__ double sh[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kRedThreads / 32; ++i) r += sh[i];
    __syncthreads();
    return r;   // valid in thread 0
}

template <class X, class Y>
__global__ void __launch_bounds__(kRedThreads)
dot_kernel(const X* __restrict__ x, const Y* __restrict__ y, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// w += lambda p ; part = p.w
template <class T>
__global__ void __launch_bounds__(kRedThreads)
shift_dot_kernel(T* __restrict__ w, const T* __restrict__ p, double lam, int64_t n, double* __restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T wi = w[i] + (T)lam * p[i];
        w[i] = wi;
        acc += (double)p[i] * (double)wi;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// sc[dst] = sum(part); optionally alpha / beta / breakdown logic
__global__ void __launch_bounds__(kRedThreads)
finalize_kernel(const double* __restrict__ part, int nb, double* __restrict__ sc, int what)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
    acc = block_sum(acc);
    if (threadIdx.x != 0) return;
    if (what == 0) {            // alpha = rr / pw; after a breakdown the iteration stays frozen
        sc[SC_PW] = acc;
        if (sc[SC_FLAG] != 0.0 || !(acc > 0.0) || !isfinite(acc)) {
            sc[SC_FLAG] = 1.0;
            sc[SC_ALPHA] = 0.0;
        } else {
            sc[SC_ALPHA] = sc[SC_RR] / acc;
        }
    } else if (what == 1) {     // beta = rr' / rr, rr = rr'
        const double rr = sc[SC_RR];
        sc[SC_BETA] = (rr > 0.0) ? acc / rr : 0.0;
        sc[SC_RR] = acc;
        if (!isfinite(acc)) sc[SC_FLAG] = 1.0;
    } else if (what == 2) {     // rr = sum, start of a CG run
        sc[SC_RR] = acc;
        sc[SC_RR0] = acc;
        sc[SC_FLAG] = 0.0;
    } else if (what == 3) {     // plain dot into SC_TMP
        sc[SC_TMP] = acc;
    } else if (what == 4) {     // flexible CG start: rz = r.z
        sc[SC_RZ] = acc;
        if (!isfinite(acc) || !(acc > 0.0)) sc[SC_FLAG] = 1.0;
    } else if (what == 5) {     // flexible CG: alpha = rz / pw (frozen after a breakdown)
        sc[SC_PW] = acc;
        if (sc[SC_FLAG] != 0.0 || !(acc > 0.0) || !isfinite(acc)) {
            sc[SC_FLAG] = 1.0;
            sc[SC_ALPHA] = 0.0;
        } else {
            sc[SC_ALPHA] = sc[SC_RZ] / acc;
        }
    } else if (what == 6) {     // rr only
        sc[SC_RR] = acc;
        if (!isfinite(acc)) sc[SC_FLAG] = 1.0;
    } else if (what == 7) {     // z.w
        sc[SC_ZW] = acc;
    } else {                    // what == 8: Polak-Ribiere beta = z'.(r' - r) / rz = -alpha z'.w / rz
        const double rz = sc[SC_RZ];
        sc[SC_BETA] = rz != 0.0 ? -sc[SC_ALPHA] * sc[SC_ZW] / rz : 0.0;
        sc[SC_RZ] = acc;
        if (!isfinite(acc) || !(acc > 0.0)) sc[SC_FLAG] = 1.0;
    }
}

// a += alpha p ; r -= alpha w ; part = r.r
template <class T, class TA>
__global__ void __launch_bounds__(kRedThreads)
update_kernel(TA* __restrict__ a, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ w,
              int64_t n, const double* __restrict__ sc, double* __restrict__ part)
{
    const double alpha = sc[SC_ALPHA];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] = (TA)((double)a[i] + alpha * (double)p[i]);
        const T ri = (T)((double)r[i] - alpha * (double)w[i]);
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// p = r + beta p
template <class T>
__global__ void pupdate_kernel(T* __restrict__ p, const T* __restrict__ r, int64_t n, const double* __restrict__ sc)
{
    const double beta = sc[SC_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (T)((double)r[i] + beta * (double)p[i]);
}

// r = y - (Ka + lambda a), with Ka given
__global__ void residual_kernel(const double* __restrict__ y, const double* __restrict__ Ka,
                                const double* __restrict__ a, double lam, int64_t n, double* __restrict__ r)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = y[i] - (Ka[i] + lam * a[i]);
}

// dst = (float)(src * scale)
__global__ void scale_to_f32_kernel(const double* __restrict__ src, double scale, int64_t n, float* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)(src[i] * scale);
}

// a += scale * c
__global__ void axpy_f32_kernel(double* __restrict__ a, const float* __restrict__ c, double scale, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += scale * (double)c[i];
}

// R = r ; E = a_star - x, stored as FP32 or BF16
__device__ __forceinline__ void store_as(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void store_as(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
template <class T, class TS>
__global__ void record_kernel(const T* __restrict__ r, const T* __restrict__ x,
                              const double* __restrict__ a_star, int64_t n, TS* __restrict__ R, TS* __restrict__ E)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        store_as(R + i, (double)r[i]);
        store_as(E + i, a_star[i] - (double)x[i]);
    }
}

template <class T>
__global__ void copy_kernel(T* __restrict__ dst, const T* __restrict__ src, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Residual history of a solve (gvt_solve_opts.history): (iteration, relative residual) pairs.
struct History {
    double* buf = nullptr;
    int32_t cap = 0;
    int32_t* len = nullptr;
    double scale = 1.0;      // converts a run's residual (relative to its own b) to ||.|| / ||y||
    int64_t offset = 0;      // iterations done before the run
    void add(int64_t it, double rel) const
    {
        if (!buf || !len || *len >= cap) return;
        buf[2 * *len] = (double)(offset + it);
        buf[2 * *len + 1] = rel * scale;
        ++*len;
    }
};

unsigned vgrid(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)g;
}

// CG on (K + lambda I) x = b with operator dtype T; x has type TA and starts
// at zero.  With a preconditioner P this is flexible CG (Polak-Ribiere beta,
// z = P r; z is a scratch vector).  Returns iterations used through *iters and
// the final recursive relative residual through *rel.
template <class T, class TA>
gvt_status cg_run(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* N,
                  const T* b, double bnorm, double lam, TA* x, T* r, T* p, T* w, double* part, double* sc,
                  double* hsc, double tol, int64_t max_iter, int check_every, int64_t* iters, double* rel,
                  cudaStream_t s_caller, gvt_precond* P = nullptr, T* z = nullptr, const History* hist = nullptr)
{
    const int64_t n = plan->n_in;
    *iters = 0;
    *rel = 1.0;
    if (bnorm == 0.0) {
        *rel = 0.0;
        return GVT_OK;
    }
    // The iterations run on the handle's CG stream (a capture cannot start on the legacy default
    // stream), after everything queued on the caller's stream so far; on every return the caller's
    // stream waits for them.
    cudaStream_t s = s_caller;
    gvt_handle* h = plan->h;
    if (h) {
        if (!h->cg_stream) {
            GVT_CUDA(cudaStreamCreateWithFlags(&h->cg_stream, cudaStreamNonBlocking));
            GVT_CUDA(cudaEventCreateWithFlags(&h->cg_fork, cudaEventDisableTiming));
            GVT_CUDA(cudaEventCreateWithFlags(&h->cg_join, cudaEventDisableTiming));
        }
        GVT_CUDA(cudaEventRecord(h->cg_fork, s_caller));
        GVT_CUDA(cudaStreamWaitEvent(h->cg_stream, h->cg_fork, 0));
        s = h->cg_stream;
    }
    struct JoinGuard {
        gvt_handle* h;
        cudaStream_t caller;
        ~JoinGuard()
        {
            if (!h) return;
            cudaEventRecord(h->cg_join, h->cg_stream);
            cudaStreamWaitEvent(caller, h->cg_join, 0);
        }
    } join_guard{h, s_caller};
    copy_kernel<T><<<vgrid(n), 256, 0, s>>>(r, b, n);
    dot_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(r, r, n, part);
    finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 2);
    GVT_LAUNCHED(3, "cg init");
    if (P) {
        GVT_CHECK(precond_apply<T>(P, r, z, s));
        copy_kernel<T><<<vgrid(n), 256, 0, s>>>(p, z, n);
        dot_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(r, z, n, part);
        finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 4);
        GVT_LAUNCHED(3, "fcg init");
    } else {
        copy_kernel<T><<<vgrid(n), 256, 0, s>>>(p, b, n);
        GVT_LAUNCH_CHECK("cg init");
    }
    if (check_every < 1) check_every = 1;
    // The convergence checks lag one check behind, so that the GPU never idles waiting for the
    // host: each check copies the scalars asynchronously into one of two pinned slots and records
    // an event; the host reads a check only after the next check's iterations are queued.  At most
    // check_every iterations run past the one that met the tolerance (a breakdown in them leaves
    // x unchanged: alpha is set to zero).
    cudaEvent_t ev[2] = {nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard()
        {
            for (int i = 0; i < 2; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } ev_guard{ev};
    for (auto& e : ev) GVT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    double* ring[2] = {hsc + 16, hsc + 32};   // SC_COUNT doubles each, clear of hsc[0, SC_COUNT)
    int64_t ring_it[2] = {0, 0};              // iteration of the check held in each slot
    int pending = -1, next_slot = 0;
    // 1 = stop with GVT_OK, 2 = stop with a breakdown, 0 = go on
    auto read_check = [&](int slot) -> int {
        const double* h = ring[slot];
        if (h[SC_FLAG] != 0.0) {
            *rel = std::sqrt(std::fabs(h[SC_RR])) / bnorm;
            return 2;
        }
        *rel = std::sqrt(h[SC_RR]) / bnorm;
        if (hist) hist->add(ring_it[slot], *rel);
        return *rel <= tol ? 1 : 0;
    };
    // Steady-state iterations of plain CG replay from a CUDA graph: after the first block of
    // check_every iterations (the workspace grown, per-tile forms and split factors built), one
    // block is captured and replayed while at least check_every iterations remain.  A product that
    // cannot be captured (or statistics, whose events are read per launch) keeps the loop eager.
    auto cg_iteration = [&]() -> gvt_status {
        GVT_CHECK(pairwise_apply<T>(plan, desc, M, N, p, w, s));
        shift_dot_kernel<T><<<kRedBlocks, kRedThreads, 0, s>>>(w, p, lam, n, part);
        finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 0);
        update_kernel<T, TA><<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, w, n, sc, part);
        finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 1);
        pupdate_kernel<T><<<vgrid(n), 256, 0, s>>>(p, r, n, sc);
        GVT_LAUNCHED(5, "cg iteration");
        return GVT_OK;
    };
    struct GraphGuard {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        ~GraphGuard()
        {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } graph;
    bool try_graph = !P && !(plan->h && plan->h->stats_on);
    long long graph_launches = 0;   // kernels in one replayed block
    int64_t it = 0;
    while (it < max_iter) {
        if (graph.e && it % check_every == 0 && it + check_every <= max_iter) {
            GVT_CUDA(cudaGraphLaunch(graph.e, s));
            count_launches((int)graph_launches);
            it += check_every;
        } else if (!P) {
            GVT_CHECK(cg_iteration());
            ++it;
        } else {
            GVT_CHECK(pairwise_apply<T>(plan, desc, M, N, p, w, s));
            shift_dot_kernel<T><<<kRedBlocks, kRedThreads, 0, s>>>(w, p, lam, n, part);
            finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 5);
            update_kernel<T, TA><<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, w, n, sc, part);
            finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 6);
            GVT_LAUNCHED(4, "fcg iteration");
            GVT_CHECK(precond_apply<T>(P, r, z, s));
            dot_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(z, w, n, part);
            finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 7);
            dot_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(r, z, n, part);
            finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 8);
            pupdate_kernel<T><<<vgrid(n), 256, 0, s>>>(p, z, n, sc);
            GVT_LAUNCHED(5, "fcg iteration");
            ++it;
        }
        if (it % check_every == 0 || it == max_iter) {
            const int slot = next_slot;
            next_slot ^= 1;
            GVT_CUDA(cudaMemcpyAsync(ring[slot], sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
            GVT_CUDA(cudaEventRecord(ev[slot], s));
            ring_it[slot] = it;
            if (pending >= 0) {
                GVT_CUDA(cudaEventSynchronize(ev[pending]));
                const int verdict = read_check(pending);
                pending = -1;
                if (verdict == 2) {
                    GVT_CUDA(cudaStreamSynchronize(s));
                    *iters = it;
                    set_error("CG breakdown: p^T (K + lambda I) p <= 0 or not finite");
                    return GVT_ERR_BREAKDOWN;
                }
                if (verdict == 1) {
                    // the returned x is the latest iterate: accept it if it meets the tolerance too
                    // (a breakdown after convergence left x as it was); CG residuals need not
                    // decrease monotonically, so otherwise iterate on
                    GVT_CUDA(cudaStreamSynchronize(s));
                    const double kept = *rel;
                    const int latest = read_check(slot);
                    if (latest != 0) {
                        if (latest == 2) *rel = kept;
                        *iters = it;
                        return GVT_OK;
                    }
                }
            }
            pending = slot;
        }
        if (try_graph && it == check_every) {
            try_graph = false;
            const long long before = gvt_launch_count_internal();
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                gvt_status gst = GVT_OK;
                for (int k = 0; k < check_every && gst == GVT_OK; ++k) gst = cg_iteration();
                cudaGraph_t g = nullptr;
                const cudaError_t ce = cudaStreamEndCapture(s, &g);
                if (gst == GVT_OK && ce == cudaSuccess && g && cudaGraphInstantiate(&graph.e, g, 0) == cudaSuccess) {
                    graph.g = g;
                } else {
                    if (g) cudaGraphDestroy(g);
                    graph.e = nullptr;
                }
            }
            cudaGetLastError();   // a capture that failed leaves the loop eager
            // the captured kernels ran nowhere yet: they are counted when a block replays
            graph_launches = gvt_launch_count_internal() - before;
            count_launches(-(int)graph_launches);
        }
    }
    *iters = it;
    if (pending >= 0) {
        GVT_CUDA(cudaEventSynchronize(ev[pending]));
        const int verdict = read_check(pending);
        if (verdict == 2) {
            set_error("CG breakdown: p^T (K + lambda I) p <= 0 or not finite");
            return GVT_ERR_BREAKDOWN;
        }
        if (verdict == 1) return GVT_OK;
    }
    return GVT_ERR_NOT_CONVERGED;
}

// ||y - (K64 a + lambda a)|| into r (FP64) and its norm on the host.
gvt_status fp64_residual(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* N,
                         const double* y, const double* a, double lam, double* Ka, double* r, double* part,
                         double* sc, double* hsc, double* rnorm, cudaStream_t s)
{
    const int64_t n = plan->n_in;
    GVT_CHECK(pairwise_apply<double>(plan, desc, M, N, a, Ka, s));
    residual_kernel<<<vgrid(n), 256, 0, s>>>(y, Ka, a, lam, n, r);
    dot_kernel<double, double><<<kRedBlocks, kRedThreads, 0, s>>>(r, r, n, part);
    finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 3);
    GVT_LAUNCHED(3, "residual");
    GVT_CUDA(cudaMemcpyAsync(hsc, sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    GVT_CUDA(cudaStreamSynchronize(s));
    *rnorm = std::sqrt(hsc[SC_TMP]);
    return GVT_OK;
}

// CG from zero on (K + lambda I) x = y in operator precision T; at the listed iterations the
// residual and a_star - x go to columns of R and E (storage TS).
template <class T, class TS>
gvt_status record_run(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* Nn,
                      const double* y, double lambda, const double* a_star, const int64_t* iters, int64_t count,
                      TS* R, TS* E, cudaStream_t s)
{
    const int64_t n = plan->n_in;
    Arena& ws = h->solve_ws;
    ws.reset();
    const size_t o_x = ws.take(sizeof(T) * n), o_r = ws.take(sizeof(T) * n), o_p = ws.take(sizeof(T) * n),
                 o_w = ws.take(sizeof(T) * n), o_y = ws.take(sizeof(T) * n);
    const size_t o_part = ws.take(8 * kRedBlocks), o_sc = ws.take(8 * SC_COUNT);
    GVT_CHECK(ws.commit(s));
    char* base = ws.base();
    T* x = (T*)(base + o_x);
    T* r = (T*)(base + o_r);
    T* p = (T*)(base + o_p);
    T* w = (T*)(base + o_w);
    T* yy = (T*)(base + o_y);
    double* part = (double*)(base + o_part);
    double* sc = (double*)(base + o_sc);
    if (sizeof(T) == 8) {
        copy_kernel<double><<<vgrid(n), 256, 0, s>>>(reinterpret_cast<double*>(yy), y, n);
        GVT_LAUNCH_CHECK("record init");
    } else {
        GVT_CHECK(convert(y, GVT_F64, yy, GVT_F32, n, s));
    }
    GVT_CHECK(vec_zero<T>(x, n, s));
    copy_kernel<T><<<vgrid(n), 256, 0, s>>>(r, yy, n);
    copy_kernel<T><<<vgrid(n), 256, 0, s>>>(p, yy, n);
    dot_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(r, r, n, part);
    finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 2);
    GVT_LAUNCHED(4, "record init");
    int64_t j = 0;
    for (int64_t it = 0; j < count; ++it) {
        if (it == iters[j]) {
            record_kernel<T, TS><<<vgrid(n), 256, 0, s>>>(r, x, a_star, n, R + j * n, E + j * n);
            GVT_LAUNCH_CHECK("record");
            ++j;
            if (j == count) break;
        }
        GVT_CHECK(pairwise_apply<T>(plan, desc, M, Nn, p, w, s));
        shift_dot_kernel<T><<<kRedBlocks, kRedThreads, 0, s>>>(w, p, lambda, n, part);
        finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 0);
        update_kernel<T, T><<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, w, n, sc, part);
        finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 1);
        pupdate_kernel<T><<<vgrid(n), 256, 0, s>>>(p, r, n, sc);
        GVT_LAUNCHED(5, "record iteration");
    }
    GVT_CUDA(cudaStreamSynchronize(s));
    return GVT_OK;
}

}  // namespace
}  // namespace gvt

extern "C" gvt_status gvt_cg_record_pairs(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                          const gvt_matrix* N, const double* y, double lambda, const double* a_star,
                                          const int64_t* iters, int64_t count, int32_t op_dtype, void* R, void* E,
                                          int32_t store_dtype, void* stream)
{
    using namespace gvt;
    if (!h || !plan || !desc || !M || !y || !a_star || !iters || count < 1 || !R || !E || !plan->out_is_in ||
        !(lambda > 0.0) || (op_dtype != GVT_F64 && op_dtype != GVT_F32) ||
        (store_dtype != GVT_F32 && store_dtype != GVT_BF16)) {
        set_error("gvt_cg_record_pairs: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    const gvt_matrix* Nn = desc->homogeneous ? M : N;
    if (!Nn || M->dtype != op_dtype || Nn->dtype != op_dtype) {
        set_error("gvt_cg_record_pairs: M and N must have the operator dtype");
        return GVT_ERR_INVALID_ARG;
    }
    for (int64_t j = 1; j < count; ++j)
        if (iters[j] <= iters[j - 1] || iters[0] < 0) {
            set_error("gvt_cg_record_pairs: iterations must be ascending and >= 0");
            return GVT_ERR_INVALID_ARG;
        }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op_dtype == GVT_F64) {
        if (store_dtype == GVT_BF16)
            return record_run<double, __nv_bfloat16>(h, plan, desc, M, Nn, y, lambda, a_star, iters, count,
                                                     static_cast<__nv_bfloat16*>(R), static_cast<__nv_bfloat16*>(E), s);
        return record_run<double, float>(h, plan, desc, M, Nn, y, lambda, a_star, iters, count,
                                         static_cast<float*>(R), static_cast<float*>(E), s);
    }
    if (store_dtype == GVT_BF16)
        return record_run<float, __nv_bfloat16>(h, plan, desc, M, Nn, y, lambda, a_star, iters, count,
                                                static_cast<__nv_bfloat16*>(R), static_cast<__nv_bfloat16*>(E), s);
    return record_run<float, float>(h, plan, desc, M, Nn, y, lambda, a_star, iters, count, static_cast<float*>(R),
                                    static_cast<float*>(E), s);
}


using namespace gvt;

extern "C" {

gvt_status gvt_solve_opts_default(gvt_solve_opts* o)
{
    if (!o) {
        set_error("gvt_solve_opts_default: NULL");
        return GVT_ERR_INVALID_ARG;
    }
    o->rel_tol = 1e-6;
    o->max_iter = 10000;
    o->mode = GVT_SOLVE_FP64_CG;
    o->inner_dtype = GVT_F32;
    o->inner_tol = 1e-3;
    o->max_refine = 30;
    o->check_every = 1;
    o->precond_budget = 0;
    o->precond = nullptr;
    o->history = nullptr;
    o->history_cap = 0;
    o->reserved_opts = 0;
    return GVT_OK;
}

gvt_status gvt_krr_cg_solve(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                            const gvt_matrix* N, const double* y, double lambda, double* a,
                            const gvt_solve_opts* opts_in, gvt_solve_info* info, void* stream)
{
    auto t0 = std::chrono::steady_clock::now();
    gvt_solve_opts opts;
    if (opts_in) opts = *opts_in; else gvt_solve_opts_default(&opts);
    gvt_solve_info loc{};
    if (!info) info = &loc;
    *info = gvt_solve_info{};
    auto ret = [&](gvt_status st_) {
        info->status = st_;
        return st_;
    };
    if (!h || !plan || !desc || !M || (!N && !desc->homogeneous)) {
        set_error("gvt_krr_cg_solve: NULL argument");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!plan->out_is_in) {
        set_error("gvt_krr_cg_solve: the plan must be a training plan (output pairs = input pairs)");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (!(lambda > 0.0) || !(opts.rel_tol > 0.0) || opts.max_iter < 0) {
        set_error("gvt_krr_cg_solve: lambda and rel_tol must be > 0");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (opts.mode != GVT_SOLVE_FP64_CG && opts.mode != GVT_SOLVE_MIXED_IR) {
        set_error("gvt_krr_cg_solve: unknown mode");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (opts.mode == GVT_SOLVE_MIXED_IR && opts.inner_dtype != GVT_F32 && opts.inner_dtype != GVT_BF16 &&
        opts.inner_dtype != GVT_F16) {
        set_error("gvt_krr_cg_solve: MIXED_IR inner operator must be GVT_F32, GVT_BF16 or GVT_F16");
        return ret(GVT_ERR_UNSUPPORTED);
    }
    const int64_t n = plan->n_in;
    gvt_precond* P = const_cast<gvt_precond*>(opts.precond);
    if (P && precond_size(P) != n) {
        set_error("gvt_krr_cg_solve: the preconditioner was built for a different number of pairs");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n > 0 && (!y || !a)) {
        set_error("gvt_krr_cg_solve: y or a is NULL");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (M->dtype != GVT_F64 || (N && !desc->homogeneous && N->dtype != GVT_F64)) {
        set_error("gvt_krr_cg_solve: M and N must be FP64");
        return ret(GVT_ERR_INVALID_ARG);
    }
    if (n == 0) {
        info->time_ms = 0.0;
        return ret(GVT_OK);
    }
    if (opts.history && opts.history_cap < 0) {
        set_error("gvt_krr_cg_solve: history_cap < 0");
        return ret(GVT_ERR_INVALID_ARG);
    }
    History hist;
    hist.buf = opts.history;
    hist.cap = opts.history ? opts.history_cap : 0;
    hist.len = &info->history_len;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool homo = desc->homogeneous != 0;
    const gvt_matrix* Nn = homo ? M : N;
    FactorCacheScope keep_splits(h);   // M and N stay fixed for the whole solve
    // flexible-CG iterations before the plain-CG fallback
    const int64_t pbudget = opts.precond_budget > 0 ? std::min<int64_t>(opts.precond_budget, opts.max_iter)
                                                    : std::max<int64_t>(1, opts.max_iter / 2);

    // ---- solver workspace
    Arena& ws = h->solve_ws;
    ws.reset();
    const size_t o_r = ws.take(8 * n), o_p = ws.take(8 * n), o_w = ws.take(8 * n), o_y = ws.take(8 * n);
    const size_t o_part = ws.take(8 * kRedBlocks), o_sc = ws.take(8 * SC_COUNT);
    size_t o_z = (P && opts.mode == GVT_SOLVE_FP64_CG) ? ws.take(8 * n) : 0;
    size_t o_m32 = 0, o_n32 = 0, o_r32 = 0, o_p32 = 0, o_w32 = 0, o_c32 = 0, o_q32 = 0;
    const bool mixed = opts.mode == GVT_SOLVE_MIXED_IR;
    if (mixed) {
        o_m32 = ws.take(4 * (size_t)M->rows * M->ld);
        if (!homo) o_n32 = ws.take(4 * (size_t)Nn->rows * Nn->ld);
        o_r32 = ws.take(4 * n); o_p32 = ws.take(4 * n); o_w32 = ws.take(4 * n); o_c32 = ws.take(4 * n);
        o_q32 = ws.take(4 * n);
        if (P) o_z = ws.take(4 * n);
    }
    gvt_status st = ws.commit(s);
    if (st != GVT_OK) return ret(st);
    char* base = ws.base();
    double* r = (double*)(base + o_r);
    double* p = (double*)(base + o_p);
    double* w = (double*)(base + o_w);
    double* ytmp = (double*)(base + o_y);
    double* part = (double*)(base + o_part);
    double* sc = (double*)(base + o_sc);
    double* hsc = h->host_scalars;

    // ||y||
    dot_kernel<double, double><<<kRedBlocks, kRedThreads, 0, s>>>(y, y, n, part);
    finalize_kernel<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, sc, 3);
    count_launches(2);
    if (cudaMemcpyAsync(hsc, sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "solve init"));
    const double ynorm = std::sqrt(hsc[SC_TMP]);

    auto finish = [&](gvt_status status) {
        double rn = 0.0;
        gvt_status s2 = fp64_residual(plan, desc, M, Nn, y, a, lambda, w, r, part, sc, hsc, &rn, s);
        info->rel_residual = ynorm > 0 ? rn / ynorm : 0.0;
        info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (s2 != GVT_OK) status = s2;
        return ret(status);
    };

    if (!mixed) {
        // b = y - (K a + lambda a) for a warm start; x accumulates the correction into a.
        double rn;
        st = fp64_residual(plan, desc, M, Nn, y, a, lambda, w, ytmp, part, sc, hsc, &rn, s);
        if (st != GVT_OK) return ret(st);
        if (ynorm == 0.0 || rn / ynorm <= opts.rel_tol) return finish(GVT_OK);
        int64_t its = 0;
        double rel = 1.0;
        hist.add(0, rn / ynorm);
        hist.scale = rn / ynorm;
        // CG on the correction: stop when ||r|| <= rel_tol * ||y||
        st = cg_run<double, double>(plan, desc, M, Nn, ytmp, rn, lambda, a, r, p, w, part, sc, hsc,
                                    opts.rel_tol * ynorm / rn, P ? pbudget : opts.max_iter, opts.check_every,
                                    &its, &rel, s, P, P ? (double*)(base + o_z) : nullptr, &hist);
        info->iterations = its;
        if (P && (st == GVT_ERR_NOT_CONVERGED || st == GVT_ERR_BREAKDOWN)) {
            // fallback: plain CG from the current iterate with the remaining iterations
            info->precond_fallback = 1;
            st = fp64_residual(plan, desc, M, Nn, y, a, lambda, w, ytmp, part, sc, hsc, &rn, s);
            if (st != GVT_OK) return ret(st);
            if (rn / ynorm <= opts.rel_tol) return finish(GVT_OK);
            int64_t its2 = 0;
            hist.scale = rn / ynorm;
            hist.offset = its;
            st = cg_run<double, double>(plan, desc, M, Nn, ytmp, rn, lambda, a, r, p, w, part, sc, hsc,
                                        opts.rel_tol * ynorm / rn, opts.max_iter - its, opts.check_every, &its2,
                                        &rel, s, nullptr, nullptr, &hist);
            info->iterations = its + its2;
        }
        return finish(st);
    }

    // ---- mixed precision: FP32 copies of the kernel matrices
    float* m32 = (float*)(base + o_m32);
    float* n32 = homo ? m32 : (float*)(base + o_n32);
    float* r32 = (float*)(base + o_r32);
    float* p32 = (float*)(base + o_p32);
    float* w32 = (float*)(base + o_w32);
    float* c32 = (float*)(base + o_c32);
    float* q32 = (float*)(base + o_q32);
    // element count up to the end of the last row (a view's ld may run past its allocation)
    auto span = [](const gvt_matrix* A) { return A->rows > 0 ? (A->rows - 1) * A->ld + A->cols : 0; };
    st = convert(M->data, GVT_F64, m32, GVT_F32, span(M), s);
    if (st == GVT_OK && !homo) st = convert(Nn->data, GVT_F64, n32, GVT_F32, span(Nn), s);
    if (st != GVT_OK) return ret(st);
    gvt_matrix M32 = *M, N32 = *Nn;
    M32.data = m32; M32.dtype = GVT_F32;
    N32.data = n32; N32.dtype = GVT_F32;

    int64_t total = 0;
    for (int k = 0; k <= opts.max_refine; ++k) {
        double rn;
        st = fp64_residual(plan, desc, M, Nn, y, a, lambda, w, r, part, sc, hsc, &rn, s);
        if (st != GVT_OK) return ret(st);
        info->refinements = k;
        hist.add(total, ynorm > 0 ? rn / ynorm : 0.0);
        if (ynorm == 0.0 || rn / ynorm <= opts.rel_tol) {
            info->iterations = total;
            return finish(GVT_OK);
        }
        if (total >= opts.max_iter || k == opts.max_refine) break;
        scale_to_f32_kernel<<<vgrid(n), 256, 0, s>>>(r, 1.0 / rn, n, r32);
        count_launches(1);
        vec_zero<float>(c32, n, s);
        int64_t its = 0;
        double rel = 1.0;
        // the inner solve only needs to reach the outer target relative to ||r||
        const double inner_tol = std::max(opts.inner_tol, 0.5 * opts.rel_tol * ynorm / rn);
        const int saved_engine = plan->h->stage1_engine;
        if (opts.inner_dtype == GVT_BF16) plan->h->stage1_engine = GVT_STAGE1_TC_BF16X3;
        if (opts.inner_dtype == GVT_F16) plan->h->stage1_engine = GVT_STAGES_TC_F16X1;
        const int64_t inner_budget = P ? std::min(pbudget, opts.max_iter - total) : opts.max_iter - total;
        st = cg_run<float, float>(plan, desc, &M32, &N32, r32, 1.0, lambda, c32, q32, p32, w32, part, sc,
                                  hsc, inner_tol, inner_budget, opts.check_every, &its, &rel, s,
                                  P, P ? (float*)(base + o_z) : nullptr);
        plan->h->stage1_engine = saved_engine;
        if (opts.inner_dtype != GVT_F32 || saved_engine != GVT_STAGE1_SIMT) {
            int word = 0;
            if (cudaMemcpyAsync(&word, handle_err_word(plan->h), sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return ret(cuda_fail(cudaGetLastError(), "device error word"));
            if (word) {
                cudaMemsetAsync(handle_err_word(plan->h), 0, sizeof(int), s);
                set_error("a bounded wait in a tensor-core stage expired");
                info->iterations = total + its;
                return ret(GVT_ERR_TIMEOUT);
            }
        }
        total += its;
        if (P && (st == GVT_ERR_NOT_CONVERGED || st == GVT_ERR_BREAKDOWN)) {
            // fallback: the remaining inner solves run plain CG; a broken-down correction is dropped
            info->precond_fallback = 1;
            P = nullptr;
            if (st == GVT_ERR_BREAKDOWN) continue;
        } else if (st == GVT_ERR_BREAKDOWN) {
            info->iterations = total;
            return finish(st);
        }
        axpy_f32_kernel<<<vgrid(n), 256, 0, s>>>(a, c32, rn, n);
        count_launches(1);
    }
    info->iterations = total;
    return finish(GVT_ERR_NOT_CONVERGED);
}

}  // extern "C"
