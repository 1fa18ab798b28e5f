// Batched kernel ridge regression: many independent problems, each with
// several regularisation values lambda_c, solved together (Eq. linsystem for
// every (problem, lambda) system).
//
// All problems live in packed device buffers.  The Kronecker operator of
// every problem is applied to k = n_lambda right-hand sides at once, so that
// each kernel-matrix element loaded serves k multiply-adds:
//   stage 1:  S_b[y, x, c] = sum_{j: d_j = x} N_b[y, t_j] V[j, c]
//   stage 2:  W[i, c]      = sum_x M_b[d_i, x] S_b[t_i, x, c]   (+ lambda_c V[i, c])
// Both stages are persistent kernels that walk a work list of
// (problem, tile) items sorted by cost, one launch for the whole batch.  The
// FP32 CG iteration (operator, FP64 dot products, per-system step lengths,
// updates) is captured once into a CUDA graph and replayed; the FP64 operator
// gives the true residuals of an iterative-refinement loop around it.  The
// stage tile shapes are chosen by timing the candidates on the first call.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>

#include "gvt_internal.h"

namespace gvt {
namespace {

struct BProb {
    int64_t n_off;   // first packed row
    int32_t n, m, q;
    int32_t pad;
    int64_t m_off;   // packed M_b (m x m)
    int64_t q_off;   // packed N_b (q x q)
    int64_t seg_off; // packed seg_b (m + 1)
    int64_t s_off;   // packed S_b (q x m x kc)
};

constexpr int KC_MAX = 16;

// ------------------------------------------------------------------ stage 1
// item = (problem, first column x0, first row y0); a CTA of NT threads owns
// 4*NT/ (kc/4) rows ... concretely: thread = (row quad, column quad).
template <class T, int NT>
__global__ void __launch_bounds__(NT)
b_stage1_kernel(const int4* __restrict__ items, int n_items, const BProb* __restrict__ probs,
                const T* __restrict__ Npk, const int32_t* __restrict__ seg, const int32_t* __restrict__ tcol,
                const int32_t* __restrict__ perm, const T* __restrict__ V, T* __restrict__ S, int kc, int tx)
{
    const int cq_n = kc / 4;                 // column quads; NT / cq_n row quads per item
    const int cq = threadIdx.x % cq_n, rq = threadIdx.x / cq_n;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const BProb P = probs[w.x];
        const int y = w.z + rq * 4;
        const bool row_ok = y < P.q;
        const T* Nb = Npk + P.q_off;
        const int32_t* sg = seg + P.seg_off;
        const int xe = min(w.y + tx, P.m);
        for (int x = w.y; x < xe; ++x) {
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
            const int j1 = sg[x + 1];
            for (int j = sg[x]; j < j1; ++j) {
                const int64_t g = P.n_off + j;
                const int32_t t = tcol[g];
                const T* vr = V + (P.n_off + perm[g]) * kc + cq * 4;
                T vv[4], nb[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) vv[c] = vr[c];
                const T* nr = Nb + (int64_t)t * P.q + y;   // row t of the symmetric N_b
#pragma unroll
                for (int a = 0; a < 4; ++a) nb[a] = (row_ok && y + a < P.q) ? nr[a] : T(0);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = fma(nb[a], vv[c], acc[a][c]);
            }
            if (row_ok) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (y + a >= P.q) break;
                    T* sr = S + P.s_off + ((int64_t)(y + a) * P.m + x) * kc + cq * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) sr[c] = acc[a][c];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ stage 2
// item = (problem, first output, end output) in drug-sorted order; one warp
// per output: 8 lanes along x times 4 lanes along column quads (kc = 16).
template <class T>
__global__ void __launch_bounds__(256)
b_stage2_kernel(const int4* __restrict__ items, int n_items, const BProb* __restrict__ probs,
                const T* __restrict__ Mpk, const int32_t* __restrict__ key, const int32_t* __restrict__ tcol,
                const int32_t* __restrict__ perm, const T* __restrict__ S, const T* __restrict__ V,
                const double* __restrict__ lam, T* __restrict__ Wout, int kc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cq_n = kc / 4;
    const int xl_n = 32 / cq_n;
    const int cq = lane % cq_n, xl = lane / cq_n;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const BProb P = probs[w.x];
        const T* Mb = Mpk + P.m_off;
        for (int i = w.y + warp; i < w.z; i += 8) {
            const int64_t g = P.n_off + i;
            const int32_t r = key[g], s = tcol[g];
            const T* mr = Mb + (int64_t)r * P.m;
            const T* sr = S + P.s_off + (int64_t)s * P.m * kc + cq * 4;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            for (int x = xl; x < P.m; x += xl_n) {
                const T mv = mr[x];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fma(mv, sr[(int64_t)x * kc + c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                for (int o = cq_n; o < 32; o <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
            if (xl == 0) {
                const int64_t row = (P.n_off + perm[g]) * kc + cq * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int cc = cq * 4 + c;
                    Wout[row + c] = acc[c] + (T)lam[cc] * V[row + c];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ batched CG vector kernels
// One block per problem; thread (jl, c) with c = tid % kc.  Systems: b * kc + c.
constexpr int kBT = 256;

__device__ double bsum_col(double x, double* sh, int kc)
{
    // reduce over the (kBT / kc) row lanes that share column c = tid % kc
    sh[threadIdx.x] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < kc)
        for (int l = threadIdx.x; l < kBT; l += kc) r += sh[l];
    __syncthreads();
    return r;
}

template <class T>
__global__ void __launch_bounds__(kBT)
b_dot_kernel(const BProb* __restrict__ probs, const T* __restrict__ X, const T* __restrict__ Y, int kc,
             double* __restrict__ out)
{
    __shared__ double sh[kBT];
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    double acc = 0.0;
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        acc += (double)X[e] * (double)Y[e];
    }
    const double r = bsum_col(acc, sh, kc);
    if (threadIdx.x < kc) out[(int64_t)blockIdx.x * kc + threadIdx.x] = r;
}

// per-system scalars
enum BS { B_RR = 0, B_PW, B_ALPHA, B_BETA, B_ACT, B_TOL2, B_N };

// alpha = rr / pw for active systems (breakdown freezes the system and flags it)
__global__ void b_alpha_kernel(const double* __restrict__ pw, double* __restrict__ sc, int nsys, int* flag)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    double* x = sc + (int64_t)s * B_N;
    x[B_PW] = pw[s];
    if (x[B_ACT] == 0.0) {
        x[B_ALPHA] = 0.0;
        return;
    }
    if (!(pw[s] > 0.0) || !isfinite(pw[s])) {
        x[B_ALPHA] = 0.0;
        x[B_ACT] = 0.0;
        atomicExch(flag, 1);
        return;
    }
    x[B_ALPHA] = x[B_RR] / pw[s];
}

// beta = rr'/rr; deactivate converged systems; count the active ones
__global__ void b_beta_kernel(const double* __restrict__ rr_new, double* __restrict__ sc, int nsys,
                              int* __restrict__ n_active)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    double* x = sc + (int64_t)s * B_N;
    if (x[B_ACT] == 0.0) {
        x[B_BETA] = 0.0;
        return;
    }
    const double rn = rr_new[s];
    x[B_BETA] = x[B_RR] > 0.0 ? rn / x[B_RR] : 0.0;
    x[B_RR] = rn;
    if (rn <= x[B_TOL2] || !isfinite(rn)) {
        x[B_ACT] = 0.0;
        x[B_BETA] = 0.0;
    } else {
        atomicAdd(n_active, 1);
    }
}

// x += alpha p; r -= alpha w; part rr (per problem block)
template <class T>
__global__ void __launch_bounds__(kBT)
b_update_kernel(const BProb* __restrict__ probs, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                const T* __restrict__ w, const double* __restrict__ sc, int kc, double* __restrict__ rr_out)
{
    __shared__ double sh[kBT];
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double alpha = sc[((int64_t)blockIdx.x * kc + c) * B_N + B_ALPHA];
    double acc = 0.0;
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        x[e] = (T)((double)x[e] + alpha * (double)p[e]);
        const T ri = (T)((double)r[e] - alpha * (double)w[e]);
        r[e] = ri;
        acc += (double)ri * (double)ri;
    }
    const double s = bsum_col(acc, sh, kc);
    if (threadIdx.x < kc) rr_out[(int64_t)blockIdx.x * kc + threadIdx.x] = s;
}

// p = r + beta p
template <class T>
__global__ void __launch_bounds__(kBT)
b_pupdate_kernel(const BProb* __restrict__ probs, T* __restrict__ p, const T* __restrict__ r,
                 const double* __restrict__ sc, int kc)
{
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double beta = sc[((int64_t)blockIdx.x * kc + c) * B_N + B_BETA];
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        p[e] = (T)((double)r[e] + beta * (double)p[e]);
    }
}

// start of an inner solve: r = p = b (FP32 copies of the scaled residual), x = 0, per-system tolerance
__global__ void b_init_scal_kernel(const double* __restrict__ rr0, double* __restrict__ sc, int nsys, int k, int kc,
                                   double inner_tol, const double* __restrict__ skip)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    double* x = sc + (int64_t)s * B_N;
    const int c = s % kc;
    x[B_RR] = rr0[s];
    x[B_TOL2] = inner_tol * inner_tol * rr0[s];
    x[B_ACT] = (c < k && rr0[s] > 0.0 && skip[s] == 0.0) ? 1.0 : 0.0;
    x[B_ALPHA] = x[B_BETA] = 0.0;
}

// r64 = Y (broadcast over columns < k) - W64 ; W64 already holds K a + lambda a
__global__ void b_residual_kernel(const BProb* __restrict__ probs, const double* __restrict__ y,
                                  const double* __restrict__ W, double* __restrict__ r, int k, int kc)
{
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        r[e] = (c < k) ? y[P.n_off + j] - W[e] : 0.0;
    }
}

// r32 = r64 / ||r||_sys ; c32 = 0
__global__ void b_scale_kernel(const BProb* __restrict__ probs, const double* __restrict__ r64,
                               const double* __restrict__ rn, float* __restrict__ b32, float* __restrict__ rr32,
                               float* __restrict__ p32, float* __restrict__ c32, int kc)
{
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double n = rn[(int64_t)blockIdx.x * kc + c];
    const double inv = n > 0.0 ? 1.0 / n : 0.0;
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        const float v = (float)(r64[e] * inv);
        b32[e] = v;
        rr32[e] = v;
        p32[e] = v;
        c32[e] = 0.f;
    }
}

// a64 += ||r|| * c32
__global__ void b_correct_kernel(const BProb* __restrict__ probs, double* __restrict__ a, const float* __restrict__ c32,
                                 const double* __restrict__ rn, int kc)
{
    const BProb P = probs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double n = rn[(int64_t)blockIdx.x * kc + c];
    for (int64_t j = jl; j < P.n; j += nl) {
        const int64_t e = (P.n_off + j) * kc + c;
        a[e] += n * (double)c32[e];
    }
}

// out_b[c * n_b + j] = a[(n_off + j) * kc + c]
__global__ void b_unpack_kernel(const BProb* __restrict__ probs, const double* __restrict__ a,
                                double* const* __restrict__ outs, int k, int kc)
{
    const BProb P = probs[blockIdx.x];
    double* o = outs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    if (c >= k || o == nullptr) return;
    for (int64_t j = jl; j < P.n; j += nl) o[(int64_t)c * P.n + j] = a[(P.n_off + j) * kc + c];
}

__global__ void b_pack_kernel(const double* __restrict__ src, int64_t n, double* __restrict__ d64, float* __restrict__ d32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        d64[i] = src[i];
        d32[i] = (float)src[i];
    }
}

template <class T>
__global__ void b_fill_kernel(T* __restrict__ x, int64_t n, T v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

unsigned gs(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// ------------------------------------------------------------------ operator object
struct Batch {
    int P = 0, k = 0, kc = 0;
    int64_t n_total = 0, mm = 0, qq = 0, segs = 0, s_elems = 0;
    std::vector<BProb> hp;
    BProb* probs = nullptr;
    double* M64 = nullptr; float* M32 = nullptr;
    double* N64 = nullptr; float* N32 = nullptr;
    int32_t *key = nullptr, *tcol = nullptr, *perm = nullptr, *seg = nullptr;
    int4 *it1 = nullptr, *it2 = nullptr;
    int n1 = 0, n2 = 0;
    int tx = 2, nt1 = 128;        // autotuned stage-1 shape
    std::vector<void*> allocs;
    ~Batch() { for (void* p : allocs) cudaFree(p); }
    template <class P_>
    gvt_status alloc(P_** out, size_t count)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(P_)) != cudaSuccess) {
            cudaGetLastError();
            set_error("batched solve: device allocation failed");
            return GVT_ERR_ALLOC;
        }
        allocs.push_back(p);
        *out = static_cast<P_*>(p);
        return GVT_OK;
    }
};

gvt_status build_items(Batch& B, int tx, int nt1, std::vector<int4>& i1)
{
    const int rows_per = 4 * (nt1 / (B.kc / 4));
    std::vector<std::pair<double, int4>> w;
    for (int b = 0; b < B.P; ++b) {
        const BProb& p = B.hp[b];
        const double dens = p.m > 0 ? (double)p.n / p.m : 0.0;
        for (int x0 = 0; x0 < p.m; x0 += tx)
            for (int y0 = 0; y0 < p.q; y0 += rows_per)
                w.push_back({dens * std::min(tx, p.m - x0), make_int4(b, x0, y0, 0)});
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    i1.clear();
    for (auto& e : w) i1.push_back(e.second);
    return GVT_OK;
}

template <class T>
gvt_status apply(const Batch& B, const T* Mpk, const T* Npk, const T* V, T* S, T* W, const double* lam, int grid1,
                 cudaStream_t s)
{
    if (B.nt1 == 128)
        b_stage1_kernel<T, 128><<<grid1, 128, 0, s>>>(B.it1, B.n1, B.probs, Npk, B.seg, B.tcol, B.perm, V, S, B.kc, B.tx);
    else
        b_stage1_kernel<T, 64><<<grid1, 64, 0, s>>>(B.it1, B.n1, B.probs, Npk, B.seg, B.tcol, B.perm, V, S, B.kc, B.tx);
    b_stage2_kernel<T><<<152 * 8, 256, 0, s>>>(B.it2, B.n2, B.probs, Mpk, B.key, B.tcol, B.perm, S, V, lam, W, B.kc);
    GVT_LAUNCHED(2, "batched operator");
    return GVT_OK;
}

}  // namespace
}  // namespace gvt

using namespace gvt;

extern "C" gvt_status gvt_krr_cg_solve_batched(gvt_handle* h, const gvt_problem* probs, int64_t n_probs,
                                               const double* lambdas_host, int64_t n_lambda,
                                               const gvt_solve_opts* opts_in, double* rel_residuals,
                                               gvt_solve_info* info, void* stream)
{
    auto t0 = std::chrono::steady_clock::now();
    gvt_solve_opts opts;
    if (opts_in) opts = *opts_in; else gvt_solve_opts_default(&opts);
    gvt_solve_info loc{};
    if (!info) info = &loc;
    *info = gvt_solve_info{};
    auto ret = [&](gvt_status st) {
        info->status = st;
        info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return st;
    };
    if (!h || !probs || n_probs <= 0 || n_probs > 65535 || !lambdas_host || n_lambda < 1 || n_lambda > KC_MAX ||
        !(opts.rel_tol > 0.0)) {
        set_error("gvt_krr_cg_solve_batched: bad argument (1..65535 problems, 1..16 lambdas)");
        return ret(GVT_ERR_INVALID_ARG);
    }
    for (int64_t l = 0; l < n_lambda; ++l)
        if (!(lambdas_host[l] > 0.0)) {
            set_error("gvt_krr_cg_solve_batched: lambdas must be > 0");
            return ret(GVT_ERR_INVALID_ARG);
        }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Batch B;
    B.P = (int)n_probs;
    B.k = (int)n_lambda;
    B.kc = (B.k + 3) / 4 * 4;
    if (B.kc == 12) B.kc = 16;   // column quads must divide the 32 lanes of a warp
    B.hp.resize(B.P);
    int64_t maxn = 0;
    for (int b = 0; b < B.P; ++b) {
        const gvt_problem& p = probs[b];
        if (p.m <= 0 || p.q <= 0 || p.m > 65535 || p.q > 65535 || p.n < 0 || p.n > INT32_MAX ||
            (p.n > 0 && (!p.d || !p.t || !p.y || !p.a)) || !p.M || !p.N) {
            set_error("gvt_krr_cg_solve_batched: bad problem " + std::to_string(b));
            return ret(GVT_ERR_INVALID_ARG);
        }
        BProb& q = B.hp[b];
        q.n_off = B.n_total; q.n = (int32_t)p.n; q.m = (int32_t)p.m; q.q = (int32_t)p.q; q.pad = 0;
        q.m_off = B.mm; q.q_off = B.qq; q.seg_off = B.segs; q.s_off = B.s_elems;
        B.n_total += p.n; B.mm += p.m * p.m; B.qq += p.q * p.q; B.segs += p.m + 1;
        B.s_elems += p.q * p.m * B.kc;
        maxn = std::max<int64_t>(maxn, p.n);
    }
    const int kc = B.kc, k = B.k;
    const int nsys = B.P * kc;
    gvt_status st;
#define BCHK(x) do { if ((st = (x)) != GVT_OK) return ret(st); } while (0)
    BCHK(B.alloc(&B.probs, B.P));
    BCHK(B.alloc(&B.M64, B.mm)); BCHK(B.alloc(&B.M32, B.mm));
    BCHK(B.alloc(&B.N64, B.qq)); BCHK(B.alloc(&B.N32, B.qq));
    BCHK(B.alloc(&B.key, B.n_total)); BCHK(B.alloc(&B.tcol, B.n_total)); BCHK(B.alloc(&B.perm, B.n_total));
    BCHK(B.alloc(&B.seg, B.segs));
    void* sort_ws = nullptr;
    BCHK(B.alloc(reinterpret_cast<char**>(&sort_ws), sort_workspace_bytes(maxn)));
    int32_t* mm = h->status.as<int32_t>();
    for (int b = 0; b < B.P; ++b) {
        const gvt_problem& p = probs[b];
        const BProb& q = B.hp[b];
        b_pack_kernel<<<gs(q.m * (int64_t)q.m), 256, 0, s>>>(p.M, (int64_t)q.m * q.m, B.M64 + q.m_off, B.M32 + q.m_off);
        b_pack_kernel<<<gs(q.q * (int64_t)q.q), 256, 0, s>>>(p.N, (int64_t)q.q * q.q, B.N64 + q.q_off, B.N32 + q.q_off);
        count_launches(2);
        if (q.n == 0) {
            BCHK(segment_offsets(B.key + q.n_off, 0, q.m, B.seg + q.seg_off, s));
            continue;
        }
        // validate ids, then sort this problem's pairs by drug id
        int32_t hm[4];
        BCHK(minmax_i32(p.d, q.n, mm, s));
        if (cudaMemcpyAsync(hm, mm, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ret(cuda_fail(cudaGetLastError(), "batched validation"));
        BCHK(minmax_i32(p.t, q.n, mm + 2, s));
        if (cudaMemcpyAsync(hm + 2, mm + 2, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched validation"));
        if (hm[0] < 0 || hm[1] >= q.m || hm[2] < 0 || hm[3] >= q.q) {
            set_error("gvt_krr_cg_solve_batched: problem " + std::to_string(b) + " has a pair index outside its kernels");
            return ret(GVT_ERR_INDEX_OOB);
        }
        BCHK(radix_sort_by_key(p.d, q.n, q.m, B.key + q.n_off, B.perm + q.n_off, sort_ws, s));
        BCHK(gather_i32(p.t, B.perm + q.n_off, q.n, B.tcol + q.n_off, s));
        BCHK(segment_offsets(B.key + q.n_off, q.n, q.m, B.seg + q.seg_off, s));
    }
    if (cudaMemcpyAsync(B.probs, B.hp.data(), sizeof(BProb) * B.P, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched upload"));

    // stage-2 items: chunks of 64 outputs
    std::vector<int4> i2;
    {
        std::vector<std::pair<double, int4>> w;
        for (int b = 0; b < B.P; ++b)
            for (int i0 = 0; i0 < B.hp[b].n; i0 += 64)
                w.push_back({(double)B.hp[b].m * std::min(64, B.hp[b].n - i0),
                             make_int4(b, i0, std::min(i0 + 64, B.hp[b].n), 0)});
        std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
        for (auto& e : w) i2.push_back(e.second);
    }
    B.n2 = (int)i2.size();
    BCHK(B.alloc(&B.it2, i2.size()));

    // ---- vectors
    const int64_t NE = B.n_total * kc;
    double *lam = nullptr, *a64 = nullptr, *r64 = nullptr, *w64 = nullptr, *S64 = nullptr, *ynorm = nullptr;
    double *rn = nullptr, *part = nullptr, *sc = nullptr, *skip = nullptr;
    float *S32 = nullptr, *b32 = nullptr, *r32 = nullptr, *p32 = nullptr, *w32 = nullptr, *c32 = nullptr;
    int* flags = nullptr;
    BCHK(B.alloc(&lam, kc)); BCHK(B.alloc(&a64, NE)); BCHK(B.alloc(&r64, NE)); BCHK(B.alloc(&w64, NE));
    BCHK(B.alloc(&S64, B.s_elems)); BCHK(B.alloc(&S32, B.s_elems));
    BCHK(B.alloc(&b32, NE)); BCHK(B.alloc(&r32, NE)); BCHK(B.alloc(&p32, NE)); BCHK(B.alloc(&w32, NE));
    BCHK(B.alloc(&c32, NE)); BCHK(B.alloc(&ynorm, nsys)); BCHK(B.alloc(&rn, nsys)); BCHK(B.alloc(&part, nsys));
    BCHK(B.alloc(&sc, (size_t)nsys * B_N)); BCHK(B.alloc(&skip, nsys)); BCHK(B.alloc(&flags, 4));
    std::vector<double> hl(kc, 1.0);
    for (int c = 0; c < k; ++c) hl[c] = lambdas_host[c];
    if (cudaMemcpyAsync(lam, hl.data(), sizeof(double) * kc, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B.it2, i2.data(), sizeof(int4) * i2.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(a64, 0, sizeof(double) * NE, s) != cudaSuccess ||
        cudaMemsetAsync(flags, 0, 16, s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched init"));

    // ||y|| per system: pack y, broadcast it over the columns with W = 0
    std::vector<double> hyn(nsys, 0.0);
    double* ypk = nullptr;
    BCHK(B.alloc(&ypk, B.n_total));
    for (int b = 0; b < B.P; ++b)
        if (B.hp[b].n > 0 &&
            cudaMemcpyAsync(ypk + B.hp[b].n_off, probs[b].y, 8 * (size_t)B.hp[b].n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched y"));
    b_fill_kernel<double><<<gs(NE), 256, 0, s>>>(w64, NE, 0.0);
    b_residual_kernel<<<B.P, kBT, 0, s>>>(B.probs, ypk, w64, r64, k, kc);
    b_dot_kernel<double><<<B.P, kBT, 0, s>>>(B.probs, r64, r64, kc, ynorm);
    count_launches(3);
    if (cudaMemcpyAsync(hyn.data(), ynorm, 8 * (size_t)nsys, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched norms"));
    for (auto& v : hyn) v = std::sqrt(v);

    // ---- autotune the stage-1 tile shape (column tile tx, threads per item); cached per handle
    const int grid1 = 152 * 8;
    {
        struct Cand { int tx, nt; };
        const Cand cands[] = {{1, 128}, {2, 128}, {4, 128}, {2, 64}, {4, 64}};
        const int ncand = 5;
        std::vector<int4> i1;
        auto key = std::make_tuple(B.P, B.n_total, kc);
        auto itc = h->batch_tune.find(key);
        int best = 0;
        if (itc != h->batch_tune.end()) {
            best = itc->second;
        } else {
            b_fill_kernel<float><<<gs(NE), 256, 0, s>>>(p32, NE, 0.f);
            count_launches(1);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best_ms = 1e30f;
            for (int ci = 0; ci < ncand; ++ci) {
                B.tx = cands[ci].tx;
                B.nt1 = cands[ci].nt;
                build_items(B, B.tx, B.nt1, i1);
                BCHK(B.alloc(&B.it1, i1.size()));
                B.n1 = (int)i1.size();
                if (cudaMemcpyAsync(B.it1, i1.data(), sizeof(int4) * i1.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
                    return ret(cuda_fail(cudaGetLastError(), "batched items"));
                BCHK(apply<float>(B, B.M32, B.N32, p32, S32, w32, lam, grid1, s));   // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) BCHK(apply<float>(B, B.M32, B.N32, p32, S32, w32, lam, grid1, s));
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = ci;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->batch_tune[key] = best;
        }
        B.tx = cands[best].tx;
        B.nt1 = cands[best].nt;
        build_items(B, B.tx, B.nt1, i1);
        BCHK(B.alloc(&B.it1, i1.size()));
        B.n1 = (int)i1.size();
        if (cudaMemcpyAsync(B.it1, i1.data(), sizeof(int4) * i1.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched items"));
        info->refinements = 0;
    }

    // ---- one inner CG iteration (FP32 operator, FP64 scalars), captured as a CUDA graph
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const unsigned sg = (unsigned)((nsys + 255) / 256);
    auto record_iter = [&](cudaStream_t cs) -> gvt_status {
        GVT_CHECK(apply<float>(B, B.M32, B.N32, p32, S32, w32, lam, grid1, cs));
        b_dot_kernel<float><<<B.P, kBT, 0, cs>>>(B.probs, p32, w32, kc, part);
        b_alpha_kernel<<<sg, 256, 0, cs>>>(part, sc, nsys, flags);
        b_update_kernel<float><<<B.P, kBT, 0, cs>>>(B.probs, c32, r32, p32, w32, sc, kc, part);
        b_beta_kernel<<<sg, 256, 0, cs>>>(part, sc, nsys, flags + 1);
        b_pupdate_kernel<float><<<B.P, kBT, 0, cs>>>(B.probs, p32, r32, sc, kc);
        GVT_LAUNCHED(5, "batched CG iteration");
        return GVT_OK;
    };
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "capture stream"));
    if (cudaStreamSynchronize(s) != cudaSuccess) return ret(cuda_fail(cudaGetLastError(), "sync"));
    cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    gvt_status cst = record_iter(cap);
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (cst != GVT_OK || ce != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        set_error("batched solve: CUDA graph capture failed");
        return ret(cst != GVT_OK ? cst : GVT_ERR_CUDA);
    }
    cudaStreamDestroy(cap);
    struct GraphGuard {
        cudaGraph_t g; cudaGraphExec_t e;
        ~GraphGuard() { if (e) cudaGraphExecDestroy(e); if (g) cudaGraphDestroy(g); }
    } guard{graph, gexec};

    // ---- iterative refinement: FP64 residual, FP32 inner CG on the correction
    std::vector<double> hrn(nsys), hskip(nsys, 0.0);
    int64_t total_it = 0;
    const int check = std::max(1, opts.check_every > 1 ? opts.check_every : 5);
    gvt_status final_st = GVT_ERR_NOT_CONVERGED;
    for (int outer = 0; outer <= opts.max_refine; ++outer) {
        // r64 = y - (K a + lambda a)
        BCHK(apply<double>(B, B.M64, B.N64, a64, S64, w64, lam, grid1, s));
        b_residual_kernel<<<B.P, kBT, 0, s>>>(B.probs, ypk, w64, r64, k, kc);
        b_dot_kernel<double><<<B.P, kBT, 0, s>>>(B.probs, r64, r64, kc, rn);
        count_launches(2);
        if (cudaMemcpyAsync(hrn.data(), rn, 8 * (size_t)nsys, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched residual"));
        double worst = 0.0;
        int open = 0;
        for (int b = 0; b < B.P; ++b)
            for (int c = 0; c < k; ++c) {
                const int sy = b * kc + c;
                hrn[sy] = std::sqrt(hrn[sy]);
                const double rel = hyn[sy] > 0 ? hrn[sy] / hyn[sy] : 0.0;
                worst = std::max(worst, rel);
                hskip[sy] = rel <= opts.rel_tol ? 1.0 : 0.0;
                open += hskip[sy] == 0.0;
                if (rel_residuals) rel_residuals[(int64_t)b * k + c] = rel;
            }
        info->rel_residual = worst;
        info->refinements = outer;
        if (open == 0) {
            final_st = GVT_OK;
            break;
        }
        if (outer == opts.max_refine || total_it >= opts.max_iter) break;
        if (cudaMemcpyAsync(rn, hrn.data(), 8 * (size_t)nsys, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(skip, hskip.data(), 8 * (size_t)nsys, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched upload"));
        b_scale_kernel<<<B.P, kBT, 0, s>>>(B.probs, r64, rn, b32, r32, p32, c32, kc);
        b_dot_kernel<float><<<B.P, kBT, 0, s>>>(B.probs, r32, r32, kc, part);
        const double itol = std::max(opts.inner_tol, 1e-6);
        b_init_scal_kernel<<<sg, 256, 0, s>>>(part, sc, nsys, k, kc, itol, skip);
        count_launches(3);
        int64_t it = 0;
        while (total_it + it < opts.max_iter) {
            if (cudaMemsetAsync(flags + 1, 0, 4, s) != cudaSuccess ||
                cudaGraphLaunch(gexec, s) != cudaSuccess)
                return ret(cuda_fail(cudaGetLastError(), "graph launch"));
            count_launches(7);
            ++it;
            if (it % check == 0) {
                int hf[2];
                if (cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return ret(cuda_fail(cudaGetLastError(), "batched check"));
                if (hf[1] == 0) break;   // no system still active
            }
        }
        total_it += it;
        b_correct_kernel<<<B.P, kBT, 0, s>>>(B.probs, a64, c32, rn, kc);
        count_launches(1);
    }
    info->iterations = total_it;
    // scatter the solutions back: a_b[:, c] (column-major per problem)
    {
        std::vector<double*> outs(B.P);
        for (int b = 0; b < B.P; ++b) outs[b] = probs[b].a;
        double** douts = nullptr;
        BCHK(B.alloc(&douts, B.P));
        if (cudaMemcpyAsync(douts, outs.data(), sizeof(double*) * B.P, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched output"));
        b_unpack_kernel<<<B.P, kBT, 0, s>>>(B.probs, a64, douts, k, kc);
        count_launches(1);
    }
    int hf[2];
    if (cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched finish"));
    if (hf[0] && final_st != GVT_OK) {
        set_error("batched CG breakdown in at least one system");
        return ret(GVT_ERR_BREAKDOWN);
    }
    if (final_st != GVT_OK) set_error("batched solve: iteration limit reached before every system converged");
#undef BCHK
    return ret(final_st);
}
