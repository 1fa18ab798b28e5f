// Batched kernel ridge regression: many independent problems, each with
// several regularisation values lambda_c, solved together (Eq. 1 for
// every (problem, lambda) system).
//
// All problems live in packed device buffers.  The Kronecker operator of
// every problem is applied to k = n_lambda right-hand sides at once, so that
// each kernel-matrix element loaded serves k multiply-adds:
//   stage 1:  S_b[y, x, c] = sum_{j: d_j = x} N_b[y, t_j] V[j, c]
//   stage 2:  W[i, c]      = sum_x M_b[d_i, x] S_b[t_i, x, c]   (+ lambda_c V[i, c])
// Both stages are persistent kernels that walk a work list of
// (problem, tile) items sorted by cost, one launch for the whole batch.  The
// FP32 CG iteration (operator, dot products summed in FP32 per thread and in
// FP64 across threads, per-system FP64 step lengths, FP32 updates) is captured
// once into a CUDA graph and replayed; the FP64 operator
// gives the true residuals of an iterative-refinement loop around it.  The
// stage tile shapes are chosen by timing the candidates on the first call.
//
// Tensor-core operator (engines GVT_STAGES_AUTO, _TC_F16X3, _TC_F16X1).  With
// the lambda columns as extra rows of the right operands, both stages of a
// problem are small dense GEMMs whose kc right-hand sides share every left
// tile (multi-RHS):
//   stage 1:  S_b[t, (c, x)] = sum_k N_b[t, k] Vd_b[(c, x), k],
//             Vd_b[(c, x), t_j] = sum of V[j, c] over the pairs j with d_j = x
//   stage 2:  C_b[d, (t, c)] = sum_x M_b[d, x] S_b[t, (c, x)],
//             W[i, c] = C_b[d_i, (t_i, c)] + lambda_c V[i, c]
// on FP16 hi/lo splits (FP32-class products; the split format of the dense
// stages), all problems in one grouped tcgen05 launch per stage.  A cost model
// per problem (dense GEMM and pass time against the sparse stages' time at
// rates measured on GB300) keeps the sparse problems on the SIMT stages, which
// then run beside the GEMMs on a second stream of the captured graph.  The
// FP64 operator of the outer residuals stays on the SIMT stages.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>

#include "gvt_internal.h"
#include "split16.cuh"

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
    int64_t seg2_off;// packed target-order segments (q + 1)
};

constexpr int KC_MAX = 16;

// Packed kernel matrices use a row pitch rounded up to 4 elements (zero
// padding), so 4 consecutive rows of a column tile load as one 16-byte vector.
__host__ __device__ inline int pitch4(int x) { return (x + 3) & ~3; }

template <class T> struct V4;
template <> struct V4<float> {
    __device__ static void ld(const float* p, float (&o)[4])
    {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
    __device__ static void ld_shared(const float* p, float (&o)[4])
    {
        const float4 q = *reinterpret_cast<const float4*>(p);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
};
template <> struct V4<double> {
    __device__ static void ld(const double* p, double (&o)[4])
    {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    __device__ static void ld_shared(const double* p, double (&o)[4])
    {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};

// ------------------------------------------------------------------ stage 1
// item = (problem, first column x0, first row y0).  Thread = (row quad rq,
// column quad cq); the item's entries are staged in shared memory as
// (target id, pair) records and consumed 4 at a time (8 vector loads in flight).
constexpr int kB1Chunk = 256;
constexpr int kB1MaxTx = 2;      // columns per stage-1 item (register tile)

template <class T, int NT>
__global__ void __launch_bounds__(NT)
b_stage1_kernel(const int4* __restrict__ items, int n_items, const BProb* __restrict__ probs,
                const T* __restrict__ Npk, const int32_t* __restrict__ seg, const int32_t* __restrict__ tcol,
                const int32_t* __restrict__ perm, const T* __restrict__ V, T* __restrict__ S, int kc, int tx)
{
    __shared__ int2 ent[kB1Chunk];
    const int cq_n = kc / 4;                 // column quads; NT / cq_n row quads per item
    const int cq = threadIdx.x % cq_n, rq = threadIdx.x / cq_n;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const BProb P = probs[w.x];
        const int qp = pitch4(P.q);
        const int y = w.z + rq * 4;
        const bool row_ok = y < P.q;
        const T* Nb = Npk + P.q_off + (row_ok ? y : 0);
        const T* Vb = V + P.n_off * kc + cq * 4;
        const int32_t* sg = seg + P.seg_off;
        const int xe = min(w.y + tx, P.m);
        const int jb = sg[w.y], je = sg[xe];
        T acc[kB1MaxTx][4][4];   // [column in tile][row][lambda]
#pragma unroll
        for (int u = 0; u < kB1MaxTx; ++u)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[u][a][c] = T(0);
        for (int j0 = jb; j0 < je; j0 += kB1Chunk) {
            __syncthreads();
            for (int e = threadIdx.x; e < kB1Chunk && j0 + e < je; e += NT) {
                const int64_t g = P.n_off + j0 + e;
                ent[e] = make_int2(tcol[g], perm[g]);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kB1MaxTx; ++u) {
                if (w.y + u >= xe) break;
                const int lo = max(sg[w.y + u], j0) - j0;
                const int hi = min(sg[w.y + u + 1], j0 + kB1Chunk) - j0;
                int e = lo;
                for (; e + 4 <= hi; e += 4) {
                    T nb[4][4], vv[4][4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int2 en = ent[e + r];
                        V4<T>::ld(Nb + (int64_t)en.x * qp, nb[r]);
                        V4<T>::ld(Vb + (int64_t)en.y * kc, vv[r]);
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int c = 0; c < 4; ++c) acc[u][a][c] = fma(nb[r][a], vv[r][c], acc[u][a][c]);
                }
                for (; e < hi; ++e) {
                    T nb[4], vv[4];
                    const int2 en = ent[e];
                    V4<T>::ld(Nb + (int64_t)en.x * qp, nb);
                    V4<T>::ld(Vb + (int64_t)en.y * kc, vv);
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[u][a][c] = fma(nb[a], vv[c], acc[u][a][c]);
                }
            }
        }
        if (row_ok) {
#pragma unroll
            for (int u = 0; u < kB1MaxTx; ++u) {
                if (w.y + u >= xe) break;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (y + a >= P.q) break;
                    T* sr = S + P.s_off + ((int64_t)(y + a) * P.m + w.y + u) * kc + cq * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) sr[c] = acc[u][a][c];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ stage 2
// item = (problem, target t): the outputs with target t (pairs sorted by
// target) all read row t of S_b, which is staged once in shared memory
// (padded to pitch4(m) rows of kc with zeros).  A warp takes 4 outputs of the
// group at a time; lane = (x quad xl, lambda quad cq): per x quad it loads
// the 4 x 4 block of S from shared memory and one 4-vector of each output's
// M row, then does 64 multiply-adds.
constexpr int kB2G = 4;

template <class T>
__global__ void __launch_bounds__(256)
b_stage2_kernel(const int4* __restrict__ items, int n_items, const BProb* __restrict__ probs,
                const T* __restrict__ Mpk, const int32_t* __restrict__ seg2, const int32_t* __restrict__ dcol2,
                const int32_t* __restrict__ perm2, const T* __restrict__ S, const T* __restrict__ V,
                const double* __restrict__ lam, T* __restrict__ Wout, int kc)
{
    extern __shared__ __align__(16) unsigned char s2_raw[];
    T* srow = reinterpret_cast<T*>(s2_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cq_n = kc / 4;
    const int xl_n = 32 / cq_n;
    const int cq = lane % cq_n, xl = lane / cq_n;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const BProb P = probs[w.x];
        const int t = w.y;
        const int32_t* sg = seg2 + P.seg2_off;
        const int i0 = sg[t], i1 = sg[t + 1];
        const int mp = pitch4(P.m);
        const T* src = S + P.s_off + (int64_t)t * P.m * kc;
        __syncthreads();
        for (int e = threadIdx.x; e < mp * kc; e += blockDim.x) srow[e] = e < P.m * kc ? src[e] : T(0);
        __syncthreads();
        const T* Mb = Mpk + P.m_off;
        for (int ib = i0 + warp * kB2G; ib < i1; ib += 8 * kB2G) {
            const int ng = min(kB2G, i1 - ib);
            const T* mr[kB2G];
#pragma unroll
            for (int g = 0; g < kB2G; ++g) {
                const int gi = ib + (g < ng ? g : ng - 1);
                mr[g] = Mb + (int64_t)dcol2[P.n_off + gi] * mp;
            }
            T acc[kB2G][4];
#pragma unroll
            for (int g = 0; g < kB2G; ++g)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[g][c] = T(0);
            for (int x = xl * 4; x < mp; x += xl_n * 4) {
                T sv[4][4], mv[kB2G][4];
#pragma unroll
                for (int xx = 0; xx < 4; ++xx) V4<T>::ld_shared(srow + (x + xx) * kc + cq * 4, sv[xx]);
#pragma unroll
                for (int g = 0; g < kB2G; ++g) V4<T>::ld(mr[g] + x, mv[g]);
#pragma unroll
                for (int g = 0; g < kB2G; ++g)
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[g][c] = fma(mv[g][xx], sv[xx][c], acc[g][c]);
            }
#pragma unroll
            for (int g = 0; g < kB2G; ++g)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    for (int o = cq_n; o < 32; o <<= 1) acc[g][c] += __shfl_xor_sync(0xffffffffu, acc[g][c], o);
            if (xl == 0) {
#pragma unroll
                for (int g = 0; g < kB2G; ++g) {
                    if (g >= ng) break;
                    const int64_t row = (P.n_off + perm2[P.n_off + ib + g]) * kc + cq * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) Wout[row + c] = acc[g][c] + (T)lam[cq * 4 + c] * V[row + c];
                }
            }
        }
    }
}

// ------------------------------------------------------------------ batched CG vector kernels
// Work unit: a chunk of kRows consecutive rows of one problem (chunk = (b, r0, r1));
// thread (jl, c) with c = tid % kc.  Dot products produce one partial sum per
// (chunk, column); b_sys_sum adds a problem's chunks in a fixed order.
constexpr int kBT = 256;
constexpr int kRows = 128;

__device__ double bsum_col(double x, double* sh, int kc)
{
    sh[threadIdx.x] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < kc)
        for (int l = threadIdx.x; l < kBT; l += kc) r += sh[l];
    __syncthreads();
    return r;
}

// Each thread sums its (at most kRows / (kBT / kc) = 8) products in T, the working precision
// of the vectors (FP32 products on the GPU run at 64 times the FP64 rate), and the block adds the
// threads' partial sums in FP64 in a fixed order.
template <class T>
__global__ void __launch_bounds__(kBT)
b_dot_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs, const T* __restrict__ X,
             const T* __restrict__ Y, int kc, double* __restrict__ part)
{
    __shared__ double sh[kBT];
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    T acc = T(0);
#pragma unroll 4
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
        acc = fma(X[e], Y[e], acc);
    }
    const double r = bsum_col((double)acc, sh, kc);
    if (threadIdx.x < kc) part[(int64_t)blockIdx.x * kc + threadIdx.x] = r;
}

// out[b * kc + c] = sum of part over problem b's chunks [cfirst[b], cfirst[b+1]): one warp per
// system, lanes striding the chunks, then a shuffle tree (a fixed order)
__global__ void b_sys_sum_kernel(const double* __restrict__ part, const int32_t* __restrict__ cfirst, int P, int kc,
                                 double* __restrict__ out)
{
    const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= P * kc) return;
    const int b = s / kc, c = s % kc;
    double acc = 0.0;
    for (int q = cfirst[b] + lane; q < cfirst[b + 1]; q += 32) acc += part[(int64_t)q * kc + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) out[s] = acc;
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

// x += alpha p; r -= alpha w; partial r.r per chunk
template <class T>
__global__ void __launch_bounds__(kBT)
b_update_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs, T* __restrict__ x,
                T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ w, const double* __restrict__ sc,
                int kc, double* __restrict__ part)
{
    __shared__ double sh[kBT];
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const T alpha = (T)sc[((int64_t)ch.x * kc + c) * B_N + B_ALPHA];
    T acc = T(0);
#pragma unroll 4
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
        x[e] = fma(alpha, p[e], x[e]);
        const T ri = fma(-alpha, w[e], r[e]);
        r[e] = ri;
        acc = fma(ri, ri, acc);
    }
    const double sres = bsum_col((double)acc, sh, kc);
    if (threadIdx.x < kc) part[(int64_t)blockIdx.x * kc + threadIdx.x] = sres;
}

// p = r + beta p
template <class T>
__global__ void __launch_bounds__(kBT)
b_pupdate_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs, T* __restrict__ p,
                 const T* __restrict__ r, const double* __restrict__ sc, int kc)
{
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const T beta = (T)sc[((int64_t)ch.x * kc + c) * B_N + B_BETA];
#pragma unroll 4
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
        p[e] = fma(beta, p[e], r[e]);
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
__global__ void b_residual_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs,
                                  const double* __restrict__ y, const double* __restrict__ W, double* __restrict__ r,
                                  int k, int kc)
{
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
        r[e] = (c < k) ? y[base + j] - W[e] : 0.0;
    }
}

// b32 = r32 = p32 = r64 / ||r||_sys ; c32 = 0
__global__ void b_scale_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs,
                               const double* __restrict__ r64, const double* __restrict__ rn, float* __restrict__ b32,
                               float* __restrict__ rr32, float* __restrict__ p32, float* __restrict__ c32, int kc)
{
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double n = rn[(int64_t)ch.x * kc + c];
    const double inv = n > 0.0 ? 1.0 / n : 0.0;
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
        const float v = (float)(r64[e] * inv);
        b32[e] = v;
        rr32[e] = v;
        p32[e] = v;
        c32[e] = 0.f;
    }
}

// a64 += ||r|| * c32
__global__ void b_correct_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs,
                                 double* __restrict__ a, const float* __restrict__ c32, const double* __restrict__ rn,
                                 int kc)
{
    const int4 ch = chunks[blockIdx.x];
    const int64_t base = probs[ch.x].n_off;
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const double n = rn[(int64_t)ch.x * kc + c];
    for (int j = ch.y + jl; j < ch.z; j += nl) {
        const int64_t e = (base + j) * kc + c;
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

// dst[r * pitch4(n) + c] = src[r * n + c] (zero padding), FP64 and FP32 copies
__global__ void b_pack_kernel(const double* __restrict__ src, int n, double* __restrict__ d64, float* __restrict__ d32)
{
    const int np = pitch4(n);
    const int64_t total = (int64_t)n * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / np, c = i % np;
        const double v = c < n ? src[r * n + c] : 0.0;
        d64[i] = v;
        d32[i] = (float)v;
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
    int P = 0, k = 0, kc = 0, m_max = 0;
    int64_t n_total = 0, mm = 0, qq = 0, segs = 0, segs2 = 0, s_elems = 0;
    std::vector<BProb> hp;
    BProb* probs = nullptr;
    double* M64 = nullptr; float* M32 = nullptr;
    double* N64 = nullptr; float* N32 = nullptr;
    int32_t *key = nullptr, *tcol = nullptr, *perm = nullptr, *seg = nullptr;        // drug order
    int32_t *key2 = nullptr, *dcol2 = nullptr, *perm2 = nullptr, *seg2 = nullptr;    // target order
    int4 *it1 = nullptr, *it2 = nullptr, *chunks = nullptr;   // stage items of every problem (FP64 operator)
    int4 *it1s = nullptr, *it2s = nullptr;                      // of the SIMT problems (FP32 operator)
    int32_t* cfirst = nullptr;
    int n1 = 0, n2 = 0, nch = 0, n1s = 0, n2s = 0;
    std::vector<char> on_tc;                                    // problem runs on the tensor cores (FP32)
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

void build_items(const Batch& B, int tx, int nt1, std::vector<int4>& i1, bool simt_only)
{
    const int rows_per = 4 * (nt1 / (B.kc / 4));
    std::vector<std::pair<double, int4>> w;
    for (int b = 0; b < B.P; ++b) {
        if (simt_only && B.on_tc[b]) continue;
        const BProb& p = B.hp[b];
        const double dens = p.m > 0 ? (double)p.n / p.m : 0.0;
        for (int x0 = 0; x0 < p.m; x0 += tx)
            for (int y0 = 0; y0 < p.q; y0 += rows_per)
                w.push_back({dens * std::min(tx, p.m - x0), make_int4(b, x0, y0, 0)});
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    i1.clear();
    for (auto& e : w) i1.push_back(e.second);
}

// the SIMT stages over the listed items (all problems, or the SIMT problems alone)
template <class T>
gvt_status apply(const Batch& B, const T* Mpk, const T* Npk, const T* V, T* S, T* W, const double* lam, int grid1,
                 cudaStream_t s, bool simt_only = false)
{
    const int4* it1 = simt_only ? B.it1s : B.it1;
    const int4* it2 = simt_only ? B.it2s : B.it2;
    const int n1 = simt_only ? B.n1s : B.n1, n2 = simt_only ? B.n2s : B.n2;
    if (n1 == 0 && n2 == 0) return GVT_OK;
    if (B.nt1 == 128)
        b_stage1_kernel<T, 128><<<grid1, 128, 0, s>>>(it1, n1, B.probs, Npk, B.seg, B.tcol, B.perm, V, S, B.kc, B.tx);
    else
        b_stage1_kernel<T, 64><<<grid1, 64, 0, s>>>(it1, n1, B.probs, Npk, B.seg, B.tcol, B.perm, V, S, B.kc, B.tx);
    const size_t smem = sizeof(T) * (size_t)pitch4(B.m_max) * B.kc;
    b_stage2_kernel<T><<<152 * 4, 256, smem, s>>>(it2, n2, B.probs, Mpk, B.seg2, B.dcol2, B.perm2, S, V, lam, W,
                                                  B.kc);
    GVT_LAUNCHED(2, "batched operator");
    return GVT_OK;
}

// out[sys] = X . Y per system (chunk partials, then a fixed-order sum per problem)
template <class T>
void sys_dot(const Batch& B, const T* X, const T* Y, double* part, double* out, cudaStream_t s)
{
    b_dot_kernel<T><<<B.nch, kBT, 0, s>>>(B.chunks, B.probs, X, Y, B.kc, part);
    b_sys_sum_kernel<<<(unsigned)(((int64_t)B.P * B.kc * 32 + 255) / 256), 256, 0, s>>>(part, B.cfirst, B.P, B.kc,
                                                                                         out);
    count_launches(2);
}

// ------------------------------------------------------------------ tensor-core operator
// One tensor-core problem: its split operands' first rows, K' of each stage and its outputs.
struct BTc {
    int32_t b;          // problem
    int32_t kp1, kp2;   // q and m rounded up to 64 (K' of stage 1 and stage 2)
    int32_t pad;
    int64_t a1_row;     // N_b split: q rows
    int64_t b1_row;     // Vd_b split: kc * m rows (c, x) at c * m + x
    int64_t a2_row;     // M_b split: m rows
    int64_t b2_row;     // S_b split: q * kc rows (t, c) at t * kc + c
    int64_t c1_off;     // S_b, FP32, q x (kc * m)
    int64_t c2_off;     // C_b, FP32, m x (q * kc)
};

// rows [r0, r0 + 8) of one split set (a warp per row): row r of the source at src_off + r * ld,
// `cols` values, split into dst row dst_row + r
struct BSplit {
    int64_t src_off, dst_row;
    int32_t ld, rows, cols, kp;
};

constexpr int kTcParts = 3;
constexpr int kTcMaxKp = 1536;      // widest K' of a tensor-core problem (shared-memory rows of stage 1)
constexpr int kTcSplitRows = 8;     // rows per split block (a warp each)

using split16::row_scale;
using split16::split8_f16;
using split16::store3;

// dst row = the FP16 split ([hi|hi|lo], or [hi|lo|hi] with pattern_b) of a source row, with its
// power-of-two scale; zeros from cols to kp
__global__ void __launch_bounds__(32 * kTcSplitRows)
b_tc_split_kernel(const int2* __restrict__ items, const BSplit* __restrict__ sets, const float* __restrict__ src,
                  uint4* __restrict__ dst, int64_t pitch_u4, float* __restrict__ inv_scale, int pattern_b)
{
    __shared__ float scale[kTcSplitRows];
    const int2 it = items[blockIdx.x];
    const BSplit S = sets[it.x];
    const int nr = min(kTcSplitRows, S.rows - it.y);   // rows of this block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < nr) {   // row scales, a warp per row
        const int64_t r = it.y + warp;
        const float* row = src + S.src_off + r * S.ld;
        float m = 0.f;
        for (int k = lane; k < S.cols; k += 32) m = fmaxf(m, fabsf(row[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float sc, inv;
        row_scale(m, sc, inv);
        if (lane == 0) {
            scale[warp] = sc;
            inv_scale[S.dst_row + r] = inv;
        }
    }
    __syncthreads();
    // the splits, every thread on consecutive 8-value groups of the block's rows (coalesced stores)
    const int per_row = S.kp / 8;
    for (int e = threadIdx.x; e < nr * per_row; e += blockDim.x) {
        const int rr = e / per_row, q = e % per_row;
        const int64_t r = it.y + rr;
        const float* row = src + S.src_off + r * S.ld;
        float xs[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) xs[k] = q * 8 + k < S.cols ? row[q * 8 + k] : 0.f;
        uint4 hi, lo;
        split8_f16(xs, scale[rr], hi, lo);
        store3(dst + (S.dst_row + r) * pitch_u4, q, per_row, pattern_b, kTcParts, hi, lo);
    }
}

// Vd_b rows (c, x) for one drug x of one problem (a block): the pairs of x (their segment in
// drug order) are accumulated at column t_j of each of the kc rows in shared memory (repeated
// pairs add up), then every row is split [hi|lo|hi] with its own scale
__global__ void __launch_bounds__(256)
b_tc_densify_kernel(const int2* __restrict__ items, const BTc* __restrict__ tcp, const BProb* __restrict__ probs,
                    const int32_t* __restrict__ seg, const int32_t* __restrict__ tcol,
                    const int32_t* __restrict__ perm, const float* __restrict__ V, int kc,
                    uint4* __restrict__ dst, int64_t pitch_u4, float* __restrict__ inv_scale)
{
    extern __shared__ float4 vrow4[];   // kc x kp1 floats
    float* vrow = reinterpret_cast<float*>(vrow4);
    const int2 it = items[blockIdx.x];
    const BTc T = tcp[it.x];
    const BProb P = probs[T.b];
    const int x = it.y, kp = T.kp1;
    for (int e = threadIdx.x; e < kc * kp / 4; e += blockDim.x) vrow4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int32_t* sg = seg + P.seg_off;
    const int j0 = sg[x], nj = sg[x + 1] - j0;
    for (int e = threadIdx.x; e < nj * kc; e += blockDim.x) {
        const int64_t g = P.n_off + j0 + e / kc;
        const int c = e % kc;
        atomicAdd(&vrow[c * kp + tcol[g]], V[(P.n_off + perm[g]) * kc + c]);
    }
    __syncthreads();
    __shared__ float scale[KC_MAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < kc; c += 8) {   // row scales, a warp per row
        const float* vr = vrow + c * kp;
        float m = 0.f;
        for (int k = lane; k < kp; k += 32) m = fmaxf(m, fabsf(vr[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float sc, inv;
        row_scale(m, sc, inv);
        if (lane == 0) {
            scale[c] = sc;
            inv_scale[T.b1_row + (int64_t)c * P.m + x] = inv;
        }
    }
    __syncthreads();
    // the splits, every thread on consecutive 8-value groups of the kc rows (coalesced stores)
    const int per_row = kp / 8;
    for (int e = threadIdx.x; e < kc * per_row; e += blockDim.x) {
        const int c = e / per_row, q = e % per_row;
        const float4* src = reinterpret_cast<const float4*>(vrow + c * kp + q * 8);
        const float4 a = src[0], b = src[1];
        const float xs[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint4 hi, lo;
        split8_f16(xs, scale[c], hi, lo);
        store3(dst + (T.b1_row + (int64_t)c * P.m + x) * pitch_u4, q, per_row, 1, kTcParts, hi, lo);
    }
}

// W[i, c] = C_b[d_i, t_i * kc + c] + lambda_c V[i, c] over a chunk of a problem's pairs (drug order)
__global__ void __launch_bounds__(kBT)
b_tc_gather_kernel(const int4* __restrict__ chunks, const BProb* __restrict__ probs, const int32_t* __restrict__ tc_of,
                   const BTc* __restrict__ tcp, const int32_t* __restrict__ key, const int32_t* __restrict__ tcol,
                   const int32_t* __restrict__ perm, const float* __restrict__ C2, const float* __restrict__ V,
                   const double* __restrict__ lam, float* __restrict__ W, int kc)
{
    const int4 ch = chunks[blockIdx.x];
    const BProb P = probs[ch.x];
    const BTc T = tcp[tc_of[ch.x]];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    const float lc = (float)lam[c];
    const int64_t ldc2 = (int64_t)P.q * kc;
    for (int g = ch.y + jl; g < ch.z; g += nl) {
        const int64_t gg = P.n_off + g;
        const int64_t e = (P.n_off + perm[gg]) * kc + c;
        W[e] = C2[T.c2_off + (int64_t)key[gg] * ldc2 + (int64_t)tcol[gg] * kc + c] + lc * V[e];
    }
}

// The tensor-core part of a batch: buffers, launch lists and the problems it covers.
struct BatchTc {
    int n = 0;                          // tensor-core problems
    int64_t pitch1 = 0, pitch2 = 0;     // row pitch (16-bit elements) of the stage-1 / stage-2 splits
    int64_t rows_a1 = 0, rows_b1 = 0, rows_a2 = 0, rows_b2 = 0;
    int kp1_max = 0;
    BTc* tcp = nullptr;
    int32_t* tc_of = nullptr;           // problem -> tensor-core index (-1: SIMT)
    uint16_t *A1 = nullptr, *B1 = nullptr, *A2 = nullptr, *B2 = nullptr;
    float *sA1 = nullptr, *sB1 = nullptr, *sA2 = nullptr, *sB2 = nullptr;
    float *C1 = nullptr, *C2 = nullptr;
    TcGroupTile *t1 = nullptr, *t2 = nullptr;
    int64_t n_t1 = 0, n_t2 = 0;
    int2 *dens_items = nullptr, *split_items = nullptr;
    int n_dens = 0, n_split = 0;
    BSplit* split_b2 = nullptr;
    int4* chunks = nullptr;
    int n_chunks = 0;
    double useful_flops = 0.0;
};

// time of one operator application of problem p on the SIMT stages and on the tensor cores (the
// two GEMMs' executed flops, the densify / split / gather passes' bytes), at GB300 rates measured
// on the batched stages and the grouped GEMM
constexpr double kBSimtRate = 1.1e13;   // useful flop/s of the batched SIMT stages
constexpr double kBTcRate = 1.0e15;     // executed flop/s of the grouped split GEMM (small tiles)
constexpr double kBPassBw = 4.0e12;     // bytes/s of the split, densify and gather passes

double simt_time(const BProb& p, int kc) { return 2.0 * kc * (double)p.n * (p.q + p.m) / kBSimtRate; }

double tc_time(const BProb& p, int kc)
{
    auto up = [](int64_t x, int64_t a) { return (double)((x + a - 1) / a * a); };
    const double kp1 = up(p.q, 64), kp2 = up(p.m, 64);
    const double g1 = 2.0 * kTcParts * up(p.q, 128) * up((int64_t)kc * p.m, 256) * kp1;
    const double g2 = 2.0 * kTcParts * up(p.m, 128) * up((int64_t)kc * p.q, 256) * kp2;
    const double cells = (double)kc * p.m * p.q;
    const double bytes = 2.0 * (2.0 * kTcParts * kc * p.m * kp1)   // Vd split written, read
                         + 2.0 * (4.0 * cells)                      // S written, read
                         + 2.0 * (2.0 * kTcParts * kc * p.q * kp2)  // S split written, read
                         + 4.0 * cells + 16.0 * kc * p.n;           // C written, gathered
    return (g1 + g2) / kBTcRate + bytes / kBPassBw;
}

// The FP32 operator: the tensor-core problems through the two grouped GEMMs on stream s, the
// SIMT problems' stages beside them on `side` (joined back into s); their outputs are disjoint.
gvt_status apply_f32(const Batch& B, const BatchTc& X, const float* M32, const float* N32, const float* V, float* S,
                     float* W, const double* lam, int grid1, int* err, cudaStream_t s, cudaStream_t side,
                     cudaEvent_t fork, cudaEvent_t join)
{
    if (X.n == 0) return apply<float>(B, M32, N32, V, S, W, lam, grid1, s, true);
    const bool simt = B.n1s > 0 || B.n2s > 0;
    if (simt) {
        GVT_CUDA(cudaEventRecord(fork, s));
        GVT_CUDA(cudaStreamWaitEvent(side, fork, 0));
        GVT_CHECK(apply<float>(B, M32, N32, V, S, W, lam, grid1, side, true));
    }
    const size_t smem = sizeof(float) * (size_t)B.kc * X.kp1_max;
    b_tc_densify_kernel<<<X.n_dens, 256, smem, s>>>(X.dens_items, X.tcp, B.probs, B.seg, B.tcol, B.perm, V, B.kc,
                                                     reinterpret_cast<uint4*>(X.B1), X.pitch1 / 8, X.sB1);
    GVT_LAUNCH_CHECK("batched densify");
    TcSparse g1{};
    g1.group = X.t1;
    g1.n_tiles = X.n_t1;
    g1.bn = 256;
    GVT_CHECK(tc_gemm(X.A1, X.pitch1, X.B1, X.pitch1, X.C1, 0, X.rows_a1, X.rows_b1, X.pitch1, true, X.sA1, X.sB1,
                      err, s, GVT_TC_PAIRS_OFF, 0, &g1));
    b_tc_split_kernel<<<X.n_split, 32 * kTcSplitRows, 0, s>>>(X.split_items, X.split_b2, X.C1,
                                                               reinterpret_cast<uint4*>(X.B2), X.pitch2 / 8, X.sB2, 1);
    GVT_LAUNCH_CHECK("batched split");
    TcSparse g2{};
    g2.group = X.t2;
    g2.n_tiles = X.n_t2;
    g2.bn = 256;
    GVT_CHECK(tc_gemm(X.A2, X.pitch2, X.B2, X.pitch2, X.C2, 0, X.rows_a2, X.rows_b2, X.pitch2, true, X.sA2, X.sB2,
                      err, s, GVT_TC_PAIRS_OFF, 0, &g2));
    b_tc_gather_kernel<<<X.n_chunks, kBT, 0, s>>>(X.chunks, B.probs, X.tc_of, X.tcp, B.key, B.tcol, B.perm, X.C2, V,
                                                  lam, W, B.kc);
    GVT_LAUNCH_CHECK("batched gather");
    if (simt) {
        GVT_CUDA(cudaEventRecord(join, side));
        GVT_CUDA(cudaStreamWaitEvent(s, join, 0));
    }
    return GVT_OK;
}

// V[(n_off + j) * kc + c] = in_b[c * n_b + j] for c < k, 0 for the padding columns (a block per problem)
__global__ void b_pack_cols_kernel(const BProb* __restrict__ probs, const float* const* __restrict__ ins,
                                   float* __restrict__ V, int k, int kc)
{
    const BProb P = probs[blockIdx.x];
    const float* in = ins[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    for (int64_t j = jl; j < P.n; j += nl) V[(P.n_off + j) * kc + c] = c < k ? in[(int64_t)c * P.n + j] : 0.f;
}

// out_b[c * n_b + j] = W[(n_off + j) * kc + c] for c < k
__global__ void b_unpack_cols_kernel(const BProb* __restrict__ probs, const float* __restrict__ W,
                                     float* const* __restrict__ outs, int k, int kc)
{
    const BProb P = probs[blockIdx.x];
    float* o = outs[blockIdx.x];
    const int c = threadIdx.x % kc, jl = threadIdx.x / kc, nl = kBT / kc;
    if (c >= k) return;
    for (int64_t j = jl; j < P.n; j += nl) o[(int64_t)c * P.n + j] = W[(P.n_off + j) * kc + c];
}

// ------------------------------------------------------------------ set-up shared by the solve and the product
// A prepared batch: the packed problems, the FP32 operator (SIMT stages and the tensor-core part)
// and its vectors.
struct BatchRun {
    Batch B;
    BatchTc X;
    double* lam = nullptr;                      // kc shifts
    float *S32 = nullptr, *v32 = nullptr, *w32 = nullptr;   // FP32 operator: S (SIMT), input, output
    int grid1 = 152 * 8;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~BatchRun()
    {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
    // w32 = (K_b + lambda_c I) v32 for every problem and column, FP32
    gvt_status apply32(gvt_handle* h, cudaStream_t s)
    {
        return apply_f32(B, X, B.M32, B.N32, v32, S32, w32, lam, grid1, handle_err_word(h), s, side, ev_fork, ev_join);
    }
};

// Packs the problems (kernel matrices in FP64 and FP32, pairs sorted by drug and by target),
// builds the stage items and vector chunks, picks the problems of the tensor-core operator,
// autotunes the SIMT stage-1 shape and prepares the tensor-core part.  n_cols in [1, 16]
// (validated by the caller); labels: the problems' y and a are required.
gvt_status batch_prepare(gvt_handle* h, const gvt_problem* probs, int64_t n_probs, const double* shifts,
                         int64_t n_cols, bool labels, const char* who, cudaStream_t s, BatchRun& R)
{
    Batch& B = R.B;
    B.P = (int)n_probs;
    B.k = (int)n_cols;
    B.kc = (B.k + 3) / 4 * 4;
    if (B.kc == 12) B.kc = 16;   // lambda quads must divide the 32 lanes of a warp
    B.hp.resize(B.P);
    int64_t maxn = 0;
    for (int b = 0; b < B.P; ++b) {
        const gvt_problem& p = probs[b];
        // stage 2 keeps one FP64 row of S_b (m x kc) in shared memory: m * kc * 8 <= 200 KiB
        if (p.m <= 0 || p.q <= 0 || pitch4((int)std::min<int64_t>(p.m, 1 << 20)) * B.kc * 8 > 200 * 1024 || p.q > 65535 || p.n < 0 || p.n > INT32_MAX ||
            (p.n > 0 && (!p.d || !p.t || (labels && (!p.y || !p.a)))) || !p.M || !p.N) {
            set_error(std::string(who) + ": bad problem " + std::to_string(b) +
                      " (m * padded lambda count <= 25600, q <= 65535)");
            return GVT_ERR_INVALID_ARG;
        }
        BProb& q = B.hp[b];
        q.n_off = B.n_total; q.n = (int32_t)p.n; q.m = (int32_t)p.m; q.q = (int32_t)p.q; q.pad = 0;
        q.m_off = B.mm; q.q_off = B.qq; q.seg_off = B.segs; q.s_off = B.s_elems; q.seg2_off = B.segs2;
        B.n_total += p.n; B.mm += p.m * pitch4((int)p.m); B.qq += p.q * pitch4((int)p.q);
        B.segs += p.m + 1; B.segs2 += p.q + 1;
        B.s_elems += p.q * p.m * B.kc;
        B.m_max = std::max<int>(B.m_max, (int)p.m);
        maxn = std::max<int64_t>(maxn, p.n);
    }
    const int kc = B.kc;
    GVT_CHECK(B.alloc(&B.probs, B.P));
    GVT_CHECK(B.alloc(&B.M64, B.mm)); GVT_CHECK(B.alloc(&B.M32, B.mm));
    GVT_CHECK(B.alloc(&B.N64, B.qq)); GVT_CHECK(B.alloc(&B.N32, B.qq));
    GVT_CHECK(B.alloc(&B.key, B.n_total)); GVT_CHECK(B.alloc(&B.tcol, B.n_total)); GVT_CHECK(B.alloc(&B.perm, B.n_total));
    GVT_CHECK(B.alloc(&B.seg, B.segs));
    GVT_CHECK(B.alloc(&B.key2, B.n_total)); GVT_CHECK(B.alloc(&B.dcol2, B.n_total)); GVT_CHECK(B.alloc(&B.perm2, B.n_total));
    GVT_CHECK(B.alloc(&B.seg2, B.segs2));
    char* sort_ws = nullptr;
    GVT_CHECK(B.alloc(&sort_ws, sort_workspace_bytes(maxn)));
    int32_t* mm = h->status.as<int32_t>();
    for (int b = 0; b < B.P; ++b) {
        const gvt_problem& p = probs[b];
        const BProb& q = B.hp[b];
        b_pack_kernel<<<gs(q.m * (int64_t)pitch4(q.m)), 256, 0, s>>>(p.M, q.m, B.M64 + q.m_off, B.M32 + q.m_off);
        b_pack_kernel<<<gs(q.q * (int64_t)pitch4(q.q)), 256, 0, s>>>(p.N, q.q, B.N64 + q.q_off, B.N32 + q.q_off);
        count_launches(2);
        if (q.n == 0) {
            GVT_CHECK(segment_offsets(B.key + q.n_off, 0, q.m, B.seg + q.seg_off, s));
            GVT_CHECK(segment_offsets(B.key2 + q.n_off, 0, q.q, B.seg2 + q.seg2_off, s));
            continue;
        }
        // validate ids, then sort this problem's pairs by drug id (stage 1) and by target id (stage 2)
        int32_t hm[4];
        GVT_CHECK(minmax_i32(p.d, q.n, mm, s));
        GVT_CHECK(minmax_i32(p.t, q.n, mm + 2, s));
        if (cudaMemcpyAsync(hm, mm, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batched validation");
        if (hm[0] < 0 || hm[1] >= q.m || hm[2] < 0 || hm[3] >= q.q) {
            set_error(std::string(who) + ": problem " + std::to_string(b) + " has a pair index outside its kernels");
            return GVT_ERR_INDEX_OOB;
        }
        GVT_CHECK(radix_sort_by_key(p.d, q.n, q.m, B.key + q.n_off, B.perm + q.n_off, sort_ws, s));
        GVT_CHECK(gather_i32(p.t, B.perm + q.n_off, q.n, B.tcol + q.n_off, s));
        GVT_CHECK(segment_offsets(B.key + q.n_off, q.n, q.m, B.seg + q.seg_off, s));
        GVT_CHECK(radix_sort_by_key(p.t, q.n, q.q, B.key2 + q.n_off, B.perm2 + q.n_off, sort_ws, s));
        GVT_CHECK(gather_i32(p.d, B.perm2 + q.n_off, q.n, B.dcol2 + q.n_off, s));
        GVT_CHECK(segment_offsets(B.key2 + q.n_off, q.n, q.q, B.seg2 + q.seg2_off, s));
    }
    if (cudaMemcpyAsync(B.probs, B.hp.data(), sizeof(BProb) * B.P, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "batched upload");

    // problems whose FP32 operator runs on the tensor cores (FP16x3 splits): all that fit under
    // GVT_STAGES_TC_F16X3, those the cost model favours under GVT_STAGES_AUTO / _TC_F16X1
    const int eng = h->stage1_engine;
    const bool tc_engine = eng == GVT_STAGES_AUTO || eng == GVT_STAGES_TC_F16X3 || eng == GVT_STAGES_TC_F16X1;
    B.on_tc.assign(B.P, 0);
    for (int b = 0; b < B.P; ++b) {
        const BProb& q = B.hp[b];
        const bool fits = (q.q + 63) / 64 * 64 <= kTcMaxKp && (q.m + 63) / 64 * 64 <= kTcMaxKp && q.n > 0;
        if (tc_engine && fits && (eng == GVT_STAGES_TC_F16X3 || tc_time(q, B.kc) < simt_time(q, B.kc)))
            B.on_tc[b] = 1;
    }
    {
        // the split operands and FP32 outputs must fit in half of the free device memory
        int64_t r1 = 0, r2 = 0, cells = 0, kp1 = 64, kp2 = 64;
        for (int b = 0; b < B.P; ++b)
            if (B.on_tc[b]) {
                const BProb& q = B.hp[b];
                r1 += q.q + (int64_t)B.kc * q.m;
                r2 += q.m + (int64_t)B.kc * q.q;
                cells += (int64_t)B.kc * q.m * q.q;
                kp1 = std::max<int64_t>(kp1, (q.q + 63) / 64 * 64);
                kp2 = std::max<int64_t>(kp2, (q.m + 63) / 64 * 64);
            }
        const double need = 2.0 * kTcParts * (double)(r1 * kp1 + r2 * kp2) + 4.0 * (double)(r1 + r2) + 8.0 * cells;
        size_t free_b = 0, total_b = 0;
        if (cells > 0 && (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || need > 0.5 * (double)free_b ||
                          r1 > INT32_MAX || r2 > INT32_MAX)) {
            cudaGetLastError();
            std::fill(B.on_tc.begin(), B.on_tc.end(), 0);
        }
    }
    // stage-2 items: one per (problem, target with outputs), largest first
    std::vector<int32_t> hseg2(B.segs2);
    if (cudaMemcpyAsync(hseg2.data(), B.seg2, 4 * (size_t)B.segs2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "batched segments");
    {
        std::vector<std::pair<double, int4>> w;
        for (int b = 0; b < B.P; ++b) {
            const BProb& q = B.hp[b];
            for (int t = 0; t < q.q; ++t) {
                const int ns = hseg2[q.seg2_off + t + 1] - hseg2[q.seg2_off + t];
                if (ns > 0) w.push_back({(double)ns * q.m + q.m, make_int4(b, t, 0, 0)});
            }
        }
        std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
        std::vector<int4> i2, i2s;
        for (auto& e : w) {
            i2.push_back(e.second);
            if (!B.on_tc[e.second.x]) i2s.push_back(e.second);
        }
        B.n2 = (int)i2.size();
        B.n2s = (int)i2s.size();
        GVT_CHECK(B.alloc(&B.it2, i2.size()));
        GVT_CHECK(B.alloc(&B.it2s, i2s.size()));
        if ((!i2.empty() &&
             cudaMemcpyAsync(B.it2, i2.data(), sizeof(int4) * i2.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            (!i2s.empty() &&
             cudaMemcpyAsync(B.it2s, i2s.data(), sizeof(int4) * i2s.size(), cudaMemcpyHostToDevice, s) != cudaSuccess))
            return cuda_fail(cudaGetLastError(), "batched items");
    }
    // row chunks of every problem for the vector kernels
    {
        std::vector<int4> ch;
        std::vector<int32_t> cf(B.P + 1, 0);
        for (int b = 0; b < B.P; ++b) {
            cf[b] = (int32_t)ch.size();
            for (int r0 = 0; r0 < B.hp[b].n; r0 += kRows) ch.push_back(make_int4(b, r0, std::min(r0 + kRows, B.hp[b].n), 0));
        }
        cf[B.P] = (int32_t)ch.size();
        if (ch.empty()) ch.push_back(make_int4(0, 0, 0, 0));
        B.nch = (int)ch.size();
        GVT_CHECK(B.alloc(&B.chunks, ch.size()));
        GVT_CHECK(B.alloc(&B.cfirst, cf.size()));
        if (cudaMemcpyAsync(B.chunks, ch.data(), sizeof(int4) * ch.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(B.cfirst, cf.data(), 4 * cf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batched chunks");
    }
    // stage 2 stages one S row (m x kc) in shared memory
    {
        const size_t sm64 = sizeof(double) * (size_t)pitch4(B.m_max) * kc;
        const size_t sm32 = sizeof(float) * (size_t)pitch4(B.m_max) * kc;
        if (sm64 > 48 * 1024 &&
            cudaFuncSetAttribute(b_stage2_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "stage 2 shared memory");
        if (sm32 > 48 * 1024 &&
            cudaFuncSetAttribute(b_stage2_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "stage 2 shared memory");
    }

    // shifts (lambda_c; 1 for the padding columns, whose vectors are zero), the FP32 operator's
    // vectors and its SIMT S
    const int64_t NE = B.n_total * kc;
    GVT_CHECK(B.alloc(&R.lam, kc));
    GVT_CHECK(B.alloc(&R.S32, B.s_elems));
    GVT_CHECK(B.alloc(&R.v32, NE));
    GVT_CHECK(B.alloc(&R.w32, NE));
    {
        std::vector<double> hl(kc, 1.0);
        for (int c = 0; c < B.k; ++c) hl[c] = shifts[c];
        if (cudaMemcpyAsync(R.lam, hl.data(), sizeof(double) * kc, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batched shifts");
    }

    // ---- autotune the stage-1 tile shape (column tile tx, threads per item); cached per handle
    const int grid1 = R.grid1;
    {
        struct Cand { int tx, nt; };
        const Cand cands[] = {{1, 128}, {2, 128}, {1, 64}, {2, 64}};
        const int ncand = 4;
        std::vector<int4> i1;
        int64_t n_simt = 0;
        for (int b = 0; b < B.P; ++b)
            if (!B.on_tc[b]) n_simt += B.hp[b].n;
        auto key = std::make_tuple(B.P, n_simt, kc);
        auto itc = h->batch_tune.find(key);
        int best = 1;   // (tx 2, 128 threads) when no FP32 problem runs on the SIMT stages
        if (itc != h->batch_tune.end()) {
            best = itc->second;
        } else if (n_simt > 0) {
            b_fill_kernel<float><<<gs(NE), 256, 0, s>>>(R.v32, NE, 0.f);
            count_launches(1);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best_ms = 1e30f;
            for (int ci = 0; ci < ncand; ++ci) {
                B.tx = cands[ci].tx;
                B.nt1 = cands[ci].nt;
                build_items(B, B.tx, B.nt1, i1, true);
                GVT_CHECK(B.alloc(&B.it1s, i1.size()));
                B.n1s = (int)i1.size();
                if (cudaMemcpyAsync(B.it1s, i1.data(), sizeof(int4) * i1.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
                    return cuda_fail(cudaGetLastError(), "batched items");
                GVT_CHECK(apply<float>(B, B.M32, B.N32, R.v32, R.S32, R.w32, R.lam, grid1, s, true));   // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) GVT_CHECK(apply<float>(B, B.M32, B.N32, R.v32, R.S32, R.w32, R.lam, grid1, s, true));
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
        build_items(B, B.tx, B.nt1, i1, false);
        GVT_CHECK(B.alloc(&B.it1, i1.size()));
        B.n1 = (int)i1.size();
        if (cudaMemcpyAsync(B.it1, i1.data(), sizeof(int4) * i1.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batched items");
        build_items(B, B.tx, B.nt1, i1, true);
        GVT_CHECK(B.alloc(&B.it1s, i1.size()));
        B.n1s = (int)i1.size();
        if (!i1.empty() &&
            cudaMemcpyAsync(B.it1s, i1.data(), sizeof(int4) * i1.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batched items");
    }

    // ---- tensor-core part of the FP32 operator: split kernel matrices, buffers, launch lists
    BatchTc& X = R.X;
    {
        std::vector<BTc> ht;
        std::vector<int32_t> h_tc_of(B.P, -1);
        std::vector<int> order;
        for (int b = 0; b < B.P; ++b)
            if (B.on_tc[b]) order.push_back(b);
        // longest tiles (largest K') first
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return std::max(B.hp[x].q, B.hp[x].m) > std::max(B.hp[y].q, B.hp[y].m);
        });
        int64_t kp1m = 64, kp2m = 64;
        for (int b : order) {
            const BProb& q = B.hp[b];
            BTc t{};
            t.b = b;
            t.kp1 = (q.q + 63) / 64 * 64;
            t.kp2 = (q.m + 63) / 64 * 64;
            t.a1_row = X.rows_a1; t.b1_row = X.rows_b1; t.a2_row = X.rows_a2; t.b2_row = X.rows_b2;
            t.c1_off = ht.empty() ? 0 : ht.back().c1_off + (int64_t)B.hp[ht.back().b].q * kc * B.hp[ht.back().b].m;
            t.c2_off = ht.empty() ? 0 : ht.back().c2_off + (int64_t)B.hp[ht.back().b].m * B.hp[ht.back().b].q * kc;
            X.rows_a1 += q.q; X.rows_b1 += (int64_t)kc * q.m; X.rows_a2 += q.m; X.rows_b2 += (int64_t)q.q * kc;
            kp1m = std::max<int64_t>(kp1m, t.kp1);
            kp2m = std::max<int64_t>(kp2m, t.kp2);
            h_tc_of[b] = (int32_t)ht.size();
            ht.push_back(t);
        }
        X.n = (int)ht.size();
        if (X.n > 0) {
            const int64_t c1n = ht.back().c1_off + (int64_t)B.hp[ht.back().b].q * kc * B.hp[ht.back().b].m;
            const int64_t c2n = ht.back().c2_off + (int64_t)B.hp[ht.back().b].m * B.hp[ht.back().b].q * kc;
            X.kp1_max = (int)kp1m;
            X.pitch1 = kTcParts * kp1m;
            X.pitch2 = kTcParts * kp2m;
            GVT_CHECK(B.alloc(&X.A1, X.rows_a1 * X.pitch1)); GVT_CHECK(B.alloc(&X.B1, X.rows_b1 * X.pitch1));
            GVT_CHECK(B.alloc(&X.A2, X.rows_a2 * X.pitch2)); GVT_CHECK(B.alloc(&X.B2, X.rows_b2 * X.pitch2));
            GVT_CHECK(B.alloc(&X.sA1, X.rows_a1)); GVT_CHECK(B.alloc(&X.sB1, X.rows_b1));
            GVT_CHECK(B.alloc(&X.sA2, X.rows_a2)); GVT_CHECK(B.alloc(&X.sB2, X.rows_b2));
            GVT_CHECK(B.alloc(&X.C1, c1n)); GVT_CHECK(B.alloc(&X.C2, c2n));
            // grouped GEMM tiles: per problem, n tile outer, m tile inner (the problem's A strips stay in L2)
            std::vector<TcGroupTile> t1, t2;
            for (const BTc& t : ht) {
                const BProb& q = B.hp[t.b];
                const int64_t n1c = (int64_t)kc * q.m, n2c = (int64_t)q.q * kc;
                for (int64_t nt = 0; nt * 256 < n1c; ++nt)
                    for (int64_t mt = 0; mt * 128 < q.q; ++mt) {
                        TcGroupTile g{};
                        g.a_row = (int32_t)(t.a1_row + mt * 128);
                        g.b_row = (int32_t)(t.b1_row + nt * 256);
                        g.nkb = kTcParts * t.kp1 / 64;
                        g.m_valid = (int32_t)(q.q - mt * 128);
                        g.n_valid = (int32_t)(n1c - nt * 256);
                        g.c_off = t.c1_off + mt * 128 * n1c + nt * 256;
                        g.ldc = n1c;
                        t1.push_back(g);
                    }
                for (int64_t nt = 0; nt * 256 < n2c; ++nt)
                    for (int64_t mt = 0; mt * 128 < q.m; ++mt) {
                        TcGroupTile g{};
                        g.a_row = (int32_t)(t.a2_row + mt * 128);
                        g.b_row = (int32_t)(t.b2_row + nt * 256);
                        g.nkb = kTcParts * t.kp2 / 64;
                        g.m_valid = (int32_t)(q.m - mt * 128);
                        g.n_valid = (int32_t)(n2c - nt * 256);
                        g.c_off = t.c2_off + mt * 128 * n2c + nt * 256;
                        g.ldc = n2c;
                        t2.push_back(g);
                    }
            }
            X.n_t1 = (int64_t)t1.size();
            X.n_t2 = (int64_t)t2.size();
            // split sets: N_b and M_b once here, S_b every application
            std::vector<BSplit> sa1, sa2, sb2;
            std::vector<int2> ia1, ia2, ib2, idn;
            for (int i = 0; i < X.n; ++i) {
                const BTc& t = ht[i];
                const BProb& q = B.hp[t.b];
                sa1.push_back(BSplit{q.q_off, t.a1_row, pitch4(q.q), q.q, q.q, t.kp1});
                sa2.push_back(BSplit{q.m_off, t.a2_row, pitch4(q.m), q.m, q.m, t.kp2});
                sb2.push_back(BSplit{t.c1_off, t.b2_row, q.m, q.q * kc, q.m, t.kp2});
                for (int r = 0; r < q.q; r += kTcSplitRows) ia1.push_back(make_int2(i, r));
                for (int r = 0; r < q.m; r += kTcSplitRows) ia2.push_back(make_int2(i, r));
                for (int r = 0; r < q.q * kc; r += kTcSplitRows) ib2.push_back(make_int2(i, r));
                for (int x = 0; x < q.m; ++x) idn.push_back(make_int2(i, x));
            }
            // gather chunks over each problem's pairs
            std::vector<int4> tch;
            for (int i = 0; i < X.n; ++i) {
                const int b = ht[i].b;
                for (int r0 = 0; r0 < B.hp[b].n; r0 += kRows)
                    tch.push_back(make_int4(b, r0, std::min(r0 + kRows, B.hp[b].n), 0));
            }
            BSplit *d_sa1 = nullptr, *d_sa2 = nullptr;
            int2 *d_ia1 = nullptr, *d_ia2 = nullptr;
            GVT_CHECK(B.alloc(&X.tcp, ht.size())); GVT_CHECK(B.alloc(&X.tc_of, h_tc_of.size()));
            GVT_CHECK(B.alloc(&X.t1, t1.size())); GVT_CHECK(B.alloc(&X.t2, t2.size()));
            GVT_CHECK(B.alloc(&d_sa1, sa1.size())); GVT_CHECK(B.alloc(&d_sa2, sa2.size())); GVT_CHECK(B.alloc(&X.split_b2, sb2.size()));
            GVT_CHECK(B.alloc(&d_ia1, ia1.size())); GVT_CHECK(B.alloc(&d_ia2, ia2.size()));
            GVT_CHECK(B.alloc(&X.split_items, ib2.size())); GVT_CHECK(B.alloc(&X.dens_items, idn.size()));
            GVT_CHECK(B.alloc(&X.chunks, tch.size()));
            X.n_split = (int)ib2.size();
            X.n_dens = (int)idn.size();
            X.n_chunks = (int)tch.size();
            auto up = [&](void* dst, const void* src, size_t bytes) {
                return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
            };
            if (!up(X.tcp, ht.data(), sizeof(BTc) * ht.size()) ||
                !up(X.tc_of, h_tc_of.data(), 4 * h_tc_of.size()) ||
                !up(X.t1, t1.data(), sizeof(TcGroupTile) * t1.size()) ||
                !up(X.t2, t2.data(), sizeof(TcGroupTile) * t2.size()) ||
                !up(d_sa1, sa1.data(), sizeof(BSplit) * sa1.size()) ||
                !up(d_sa2, sa2.data(), sizeof(BSplit) * sa2.size()) ||
                !up(X.split_b2, sb2.data(), sizeof(BSplit) * sb2.size()) ||
                !up(d_ia1, ia1.data(), sizeof(int2) * ia1.size()) ||
                !up(d_ia2, ia2.data(), sizeof(int2) * ia2.size()) ||
                !up(X.split_items, ib2.data(), sizeof(int2) * ib2.size()) ||
                !up(X.dens_items, idn.data(), sizeof(int2) * idn.size()) ||
                !up(X.chunks, tch.data(), sizeof(int4) * tch.size()))
                return cuda_fail(cudaGetLastError(), "batched tensor-core lists");
            b_tc_split_kernel<<<(unsigned)ia1.size(), 32 * kTcSplitRows, 0, s>>>(
                d_ia1, d_sa1, B.N32, reinterpret_cast<uint4*>(X.A1), X.pitch1 / 8, X.sA1, 0);
            b_tc_split_kernel<<<(unsigned)ia2.size(), 32 * kTcSplitRows, 0, s>>>(
                d_ia2, d_sa2, B.M32, reinterpret_cast<uint4*>(X.A2), X.pitch2 / 8, X.sA2, 0);
            GVT_LAUNCHED(2, "batched kernel-matrix splits");
            const size_t dsm = sizeof(float) * (size_t)kc * X.kp1_max;
            if (dsm > 48 * 1024 &&
                cudaFuncSetAttribute(b_tc_densify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) !=
                    cudaSuccess)
                return cuda_fail(cudaGetLastError(), "densify shared memory");
            if (B.n1s > 0 || B.n2s > 0) {
                if (cudaStreamCreateWithFlags(&R.side, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&R.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&R.ev_join, cudaEventDisableTiming) != cudaSuccess)
                    return cuda_fail(cudaGetLastError(), "batched side stream");
            }
            // one eager application before the capture (kernel attributes, tensor-map encoder)
            b_fill_kernel<float><<<gs(NE), 256, 0, s>>>(R.v32, NE, 0.f);
            count_launches(1);
            GVT_CHECK(apply_f32(B, X, B.M32, B.N32, R.v32, R.S32, R.w32, R.lam, grid1, handle_err_word(h), s, R.side, R.ev_fork,
                           R.ev_join));
        }
    }

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
    BatchRun R;
    gvt_status st;
#define BCHK(x) do { if ((st = (x)) != GVT_OK) return ret(st); } while (0)
    BCHK(batch_prepare(h, probs, n_probs, lambdas_host, n_lambda, true, "gvt_krr_cg_solve_batched", s, R));
    Batch& B = R.B;
    BatchTc& X = R.X;
    const int kc = B.kc, k = B.k;
    const int nsys = B.P * kc;
    const int grid1 = R.grid1;
    double* lam = R.lam;
    float *S32 = R.S32, *p32 = R.v32, *w32 = R.w32;
    // ---- vectors
    const int64_t NE = B.n_total * kc;
    double *a64 = nullptr, *r64 = nullptr, *w64 = nullptr, *S64 = nullptr, *ynorm = nullptr;
    double *rn = nullptr, *part = nullptr, *sysv = nullptr, *sc = nullptr, *skip = nullptr, *ypk = nullptr;
    float *b32 = nullptr, *r32 = nullptr, *c32 = nullptr;
    int* flags = nullptr;
    BCHK(B.alloc(&a64, NE)); BCHK(B.alloc(&r64, NE)); BCHK(B.alloc(&w64, NE));
    BCHK(B.alloc(&S64, B.s_elems));
    BCHK(B.alloc(&b32, NE)); BCHK(B.alloc(&r32, NE));
    BCHK(B.alloc(&c32, NE)); BCHK(B.alloc(&ynorm, nsys)); BCHK(B.alloc(&rn, nsys));
    BCHK(B.alloc(&part, (size_t)B.nch * kc)); BCHK(B.alloc(&sysv, nsys));
    BCHK(B.alloc(&sc, (size_t)nsys * B_N)); BCHK(B.alloc(&skip, nsys)); BCHK(B.alloc(&flags, 4));
    BCHK(B.alloc(&ypk, B.n_total));
    if (cudaMemsetAsync(a64, 0, sizeof(double) * NE, s) != cudaSuccess ||
        cudaMemsetAsync(flags, 0, 16, s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched init"));
    for (int b = 0; b < B.P; ++b)
        if (B.hp[b].n > 0 &&
            cudaMemcpyAsync(ypk + B.hp[b].n_off, probs[b].y, 8 * (size_t)B.hp[b].n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "batched y"));

    // ||y|| per system: broadcast y over the columns (W = 0)
    std::vector<double> hyn(nsys, 0.0);
    b_fill_kernel<double><<<gs(NE), 256, 0, s>>>(w64, NE, 0.0);
    b_residual_kernel<<<B.nch, kBT, 0, s>>>(B.chunks, B.probs, ypk, w64, r64, k, kc);
    count_launches(2);
    sys_dot<double>(B, r64, r64, part, ynorm, s);
    if (cudaMemcpyAsync(hyn.data(), ynorm, 8 * (size_t)nsys, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ret(cuda_fail(cudaGetLastError(), "batched norms"));
    for (auto& v : hyn) v = std::sqrt(v);

    // ---- one inner CG iteration (FP32 operator, FP64 scalars), captured as a CUDA graph
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const unsigned sg = (unsigned)((nsys + 255) / 256);
    const unsigned sgw = (unsigned)(((int64_t)nsys * 32 + 255) / 256);   // a warp per system
    auto record_iter = [&](cudaStream_t cs) -> gvt_status {
        GVT_CHECK(apply_f32(B, X, B.M32, B.N32, p32, S32, w32, lam, grid1, handle_err_word(h), cs, R.side,
                            R.ev_fork, R.ev_join));
        sys_dot<float>(B, p32, w32, part, sysv, cs);
        b_alpha_kernel<<<sg, 256, 0, cs>>>(sysv, sc, nsys, flags);
        b_update_kernel<float><<<B.nch, kBT, 0, cs>>>(B.chunks, B.probs, c32, r32, p32, w32, sc, kc, part);
        b_sys_sum_kernel<<<sgw, 256, 0, cs>>>(part, B.cfirst, B.P, kc, sysv);
        b_beta_kernel<<<sg, 256, 0, cs>>>(sysv, sc, nsys, flags + 1);
        b_pupdate_kernel<float><<<B.nch, kBT, 0, cs>>>(B.chunks, B.probs, p32, r32, sc, kc);
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
    const int graph_kernels = 7 + ((B.n1s > 0 || B.n2s > 0) ? 2 : 0) + (X.n > 0 ? 5 : 0);

    // ---- iterative refinement: FP64 residual, FP32 inner CG on the correction
    std::vector<double> hrn(nsys), hskip(nsys, 0.0);
    int64_t total_it = 0;
    const int check = std::max(1, opts.check_every > 1 ? opts.check_every : 5);
    gvt_status final_st = GVT_ERR_NOT_CONVERGED;
    for (int outer = 0; outer <= opts.max_refine; ++outer) {
        // r64 = y - (K a + lambda a)
        BCHK(apply<double>(B, B.M64, B.N64, a64, S64, w64, lam, grid1, s));
        b_residual_kernel<<<B.nch, kBT, 0, s>>>(B.chunks, B.probs, ypk, w64, r64, k, kc);
        count_launches(1);
        sys_dot<double>(B, r64, r64, part, rn, s);
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
        b_scale_kernel<<<B.nch, kBT, 0, s>>>(B.chunks, B.probs, r64, rn, b32, r32, p32, c32, kc);
        count_launches(1);
        sys_dot<float>(B, r32, r32, part, sysv, s);
        const double itol = std::max(opts.inner_tol, 1e-6);
        b_init_scal_kernel<<<sg, 256, 0, s>>>(sysv, sc, nsys, k, kc, itol, skip);
        count_launches(1);
        int64_t it = 0;
        while (total_it + it < opts.max_iter) {
            if (cudaMemsetAsync(flags + 1, 0, 4, s) != cudaSuccess || cudaGraphLaunch(gexec, s) != cudaSuccess)
                return ret(cuda_fail(cudaGetLastError(), "graph launch"));
            count_launches(graph_kernels);
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
        b_correct_kernel<<<B.nch, kBT, 0, s>>>(B.chunks, B.probs, a64, c32, rn, kc);
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
    if (X.n > 0) {
        int word = 0;
        if (cudaMemcpyAsync(&word, handle_err_word(h), sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ret(cuda_fail(cudaGetLastError(), "device error word"));
        if (word) {
            cudaMemsetAsync(handle_err_word(h), 0, sizeof(int), s);
            set_error("a bounded wait in a tensor-core stage of the batched solve expired");
            return ret(GVT_ERR_TIMEOUT);
        }
    }
    if (hf[0] && final_st != GVT_OK) {
        set_error("batched CG breakdown in at least one system");
        return ret(GVT_ERR_BREAKDOWN);
    }
    if (final_st != GVT_OK) set_error("batched solve: iteration limit reached before every system converged");
#undef BCHK
    return ret(final_st);
}

extern "C" gvt_status gvt_matvec_batched(gvt_handle* h, const gvt_problem* probs, int64_t n_probs,
                                         const double* shifts_host, int64_t n_cols, const float* const* v,
                                         float* const* w, void* stream)
{
    if (!h || !probs || n_probs <= 0 || n_probs > 65535 || !shifts_host || n_cols < 1 || n_cols > KC_MAX || !v ||
        !w) {
        set_error("gvt_matvec_batched: bad argument (1..65535 problems, 1..16 columns)");
        return GVT_ERR_INVALID_ARG;
    }
    for (int64_t c = 0; c < n_cols; ++c)
        if (!std::isfinite(shifts_host[c])) {
            set_error("gvt_matvec_batched: shifts must be finite");
            return GVT_ERR_INVALID_ARG;
        }
    for (int64_t b = 0; b < n_probs; ++b)
        if (probs[b].n > 0 && (!v[b] || !w[b])) {
            set_error("gvt_matvec_batched: problem " + std::to_string(b) + " has no input or output vector");
            return GVT_ERR_INVALID_ARG;
        }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchRun R;
    GVT_CHECK(batch_prepare(h, probs, n_probs, shifts_host, n_cols, false, "gvt_matvec_batched", s, R));
    const Batch& B = R.B;
    const float** dins = nullptr;
    float** douts = nullptr;
    GVT_CHECK(R.B.alloc(&dins, B.P));
    GVT_CHECK(R.B.alloc(&douts, B.P));
    GVT_CUDA(cudaMemcpyAsync(dins, v, sizeof(float*) * B.P, cudaMemcpyHostToDevice, s));
    GVT_CUDA(cudaMemcpyAsync(douts, w, sizeof(float*) * B.P, cudaMemcpyHostToDevice, s));
    b_pack_cols_kernel<<<B.P, kBT, 0, s>>>(B.probs, dins, R.v32, B.k, B.kc);
    GVT_LAUNCH_CHECK("batched pack");
    GVT_CHECK(R.apply32(h, s));
    b_unpack_cols_kernel<<<B.P, kBT, 0, s>>>(B.probs, R.w32, douts, B.k, B.kc);
    GVT_LAUNCH_CHECK("batched unpack");
    int word = 0;
    GVT_CUDA(cudaMemcpyAsync(&word, handle_err_word(h), sizeof(int), cudaMemcpyDeviceToHost, s));
    GVT_CUDA(cudaStreamSynchronize(s));
    if (word && R.X.n > 0) {
        cudaMemsetAsync(handle_err_word(h), 0, sizeof(int), s);
        set_error("a bounded wait in a tensor-core stage of the batched product expired");
        return GVT_ERR_TIMEOUT;
    }
    return GVT_OK;
}
