// Learned diagonal-plus-low-rank preconditioner for the kernel ridge system.
//
// Training learns V (the o_0 output, hence D, is held at its initial value
// c softplus(b3_0) = c), so the trained P = c (I + V V^T)^{-1}: a constant
// diagonal minus a learned rank-32 term, the structure of a Nystrom
// preconditioner with the subspace predicted per pair by the network.
//
// Per training pair i a small MLP maps the six features
//   x_i = ([M[d_i,d_i], N[t_i,t_i], log(1+deg d_i), log(1+deg t_i), slog g1_i, slog g2_i] - mu) / sigma
// (g1 = K 1 and g2 = K (g1 / mean g1), the kernel-graph degrees, through the signed log
// slog x = sign(x) log(1 + |x|)) through 6 -> 128 -> 128 -> 33 (ReLU) to D_i = softplus(o_0)
// and V_i = o_{1..32};
//   P r = s (z - V (I + V^T V)^{-1} V^T z),   s = sqrt(D),  z = s r,
// a diagonal matrix minus a rank-32 term in the Woodbury form, symmetric
// positive definite for any network output.  It approximates (K + lambda I)^{-1}
// and is trained on residual -> correction pairs (r_k, e_k = a* - a_k) from
// the exact solver with the loss mean_k ||P r_k - e_k||^2 / ||e_k||^2, by the
// forward / backward kernels below and Adam.
//
// Two arithmetics for the network:
//  * BF16 on the tensor cores (the default): every layer and every backward
//    product is one call of the library's tcgen05 GEMM (BF16 operands, FP32
//    accumulation in tensor memory).  Forward: Z1 = [x | 1] W1'^T (the bias b1 rides
//    on a constant-one feature), H1 = relu(Z1); Z2 = H1 W2^T, H2 = relu(Z2 + b2);
//    O = H2 W3^T + b3.  Backward: dH2 = dO W3, dZ2 = dH2 [H2 > 0], dH1 = dZ2 W2,
//    dZ1 = dH1 [H1 > 0], and the weight gradients dW = dZ^T H as GEMMs over the pairs
//    (K = n, split across SMs), from pair-contiguous transposed copies of the
//    activations that the elementwise passes write beside the row-major ones.
//    The bias gradients db2, db3 are column sums in FP64.  The split-K reduction
//    adds with atomics, so BF16 training is reproducible to rounding, not bitwise.
//  * FP32 SIMT (gvt_precond_set_dtype GVT_F32): tiles of 32 pairs held in
//    shared memory (lane = pair, warp = a block of 16 hidden units).  The backward
//    kernel recomputes the forward pass of its tile and keeps the weight gradients
//    of all its tiles in registers; blocks write partial gradients that one kernel
//    sums in a fixed order, so FP32 training is bitwise reproducible.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int PH = 128;       // hidden width
constexpr int PR = 32;        // rank
constexpr int PO = 33;        // outputs: 1 + rank
constexpr int PF = 6;         // features
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + PH * PF, OFF_W2 = OFF_B1 + PH, OFF_B2 = OFF_W2 + PH * PH,
              OFF_W3 = OFF_B2 + PH, OFF_B3 = OFF_W3 + PO * PH, NPARAM = OFF_B3 + PO;
constexpr int TP = 32;        // pairs per tile
constexpr int PT = 256;       // threads

__device__ __forceinline__ float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// an element of the training pairs or of a vector, as double (FP32, FP64 or BF16 storage)
__device__ __forceinline__ double ldv(float x) { return (double)x; }
__device__ __forceinline__ double ldv(double x) { return x; }
__device__ __forceinline__ double ldv(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// ------------------------------------------------------------------ features
__device__ __forceinline__ float slogf(double x) { return (float)(x < 0 ? -log1p(-x) : log1p(x)); }

// raw features: kernel diagonals, log(1 + degree) of drug and target, signed logs of the
// kernel-graph degrees g1 = K 1 and g2 = K (g1 / mean g1)
__global__ void feat_kernel(const int32_t* __restrict__ d, const int32_t* __restrict__ t, int64_t n,
                            const int32_t* __restrict__ seg_d, const int32_t* __restrict__ seg_t,
                            const double* __restrict__ M, int64_t ldm, const double* __restrict__ N, int64_t ldn,
                            const double* __restrict__ g1, const double* __restrict__ g2, float* __restrict__ X)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = d[i], b = t[i];
        X[i * PF + 0] = (float)M[(int64_t)a * ldm + a];
        X[i * PF + 1] = (float)N[(int64_t)b * ldn + b];
        X[i * PF + 2] = log1pf((float)(seg_d[a + 1] - seg_d[a]));
        X[i * PF + 3] = log1pf((float)(seg_t[b + 1] - seg_t[b]));
        X[i * PF + 4] = slogf(g1[i]);
        X[i * PF + 5] = slogf(g2[i]);
    }
}

// per-block sums of x and x^2 per feature (FP64), summed on the host in block order
__global__ void feat_moments_kernel(const float* __restrict__ X, int64_t n, double* __restrict__ part)
{
    __shared__ double sh[PT][2 * PF];
    double acc[2 * PF];
    for (int f = 0; f < 2 * PF; ++f) acc[f] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int f = 0; f < PF; ++f) {
            const double x = X[i * PF + f];
            acc[f] += x;
            acc[PF + f] += x * x;
        }
    for (int f = 0; f < 2 * PF; ++f) sh[threadIdx.x][f] = acc[f];
    __syncthreads();
    if (threadIdx.x < 2 * PF) {
        double s = 0;
        for (int l = 0; l < PT; ++l) s += sh[l][threadIdx.x];
        part[blockIdx.x * 2 * PF + threadIdx.x] = s;
    }
}

struct FeatNorm {
    float mu[PF], inv[PF];
};

__global__ void feat_norm_kernel(float* __restrict__ X, int64_t n, FeatNorm fn)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int f = 0; f < PF; ++f) X[i * PF + f] = (X[i * PF + f] - fn.mu[f]) * fn.inv[f];
}

__global__ void fill_ones_kernel(double* __restrict__ x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = 1.0;
}

__global__ void scale_vec_kernel(const double* __restrict__ x, double a, int64_t n, double* __restrict__ y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) y[i] = a * x[i];
}

// per-block sums of x (FP64)
__global__ void sum_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ part)
{
    __shared__ double sh[256];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a += x[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int l = 0; l < 256; ++l) s += sh[l];
        part[blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------ MLP
struct MlpSmem {
    float W1[PH * PF], b1[PH], W2[PH * PH], b2[PH], W3[PO * PH], b3[PO + 3];
    float X[TP][PF];
    float h1T[PH][TP];      // [unit][pair]
    float h1N[TP][PH];      // [pair][unit]
    float h2T[PH][TP];
    float h2N[TP][PH];
    float goT[PO][TP];
    float gz2T[PH][TP];
    float gz2N[TP][PH];
};

__device__ void load_weights(MlpSmem& S, const float* __restrict__ th)
{
    for (int i = threadIdx.x; i < PH * PF; i += PT) S.W1[i] = th[OFF_W1 + i];
    for (int i = threadIdx.x; i < PH; i += PT) {
        S.b1[i] = th[OFF_B1 + i];
        S.b2[i] = th[OFF_B2 + i];
    }
    for (int i = threadIdx.x; i < PH * PH; i += PT) S.W2[i] = th[OFF_W2 + i];
    for (int i = threadIdx.x; i < PO * PH; i += PT) S.W3[i] = th[OFF_W3 + i];
    for (int i = threadIdx.x; i < PO; i += PT) S.b3[i] = th[OFF_B3 + i];
}

// Forward of one tile (pairs p0 .. p0+TP-1, rows >= n are zero features).
// Leaves h1 / h2 (post-ReLU) in both layouts.
__device__ void tile_forward(MlpSmem& S, const float* __restrict__ X, int64_t p0, int64_t n)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < TP * PF; e += PT) {
        const int64_t i = p0 + e / PF;
        S.X[e / PF][e % PF] = i < n ? X[i * PF + e % PF] : 0.f;
    }
    __syncthreads();
    const int p = lane, u0 = w * 16;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int u = u0 + j;
        float z = S.b1[u];
#pragma unroll
        for (int f = 0; f < PF; ++f) z = fmaf(S.W1[u * PF + f], S.X[p][f], z);
        const float h = fmaxf(z, 0.f);
        S.h1T[u][p] = h;
        S.h1N[p][u] = h;
    }
    __syncthreads();
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = S.b2[u0 + j];
    for (int k = 0; k < PH; ++k) {
        const float hk = S.h1T[k][p];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = fmaf(S.W2[(u0 + j) * PH + k], hk, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float h = fmaxf(acc[j], 0.f);
        S.h2T[u0 + j][p] = h;
        S.h2N[p][u0 + j] = h;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PT, 1)
mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ X, int64_t n, float* __restrict__ O,
                   float* __restrict__ s_out, float scale)
{
    extern __shared__ __align__(16) unsigned char mlp_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(mlp_raw);
    load_weights(S, theta);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t tiles = (n + TP - 1) / TP;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t p0 = tile * TP;
        tile_forward(S, X, p0, n);
        const int64_t i = p0 + lane;
        for (int u = w; u < PO; u += 8) {
            float o = S.b3[u];
            for (int k = 0; k < PH; ++k) o = fmaf(S.W3[u * PH + k], S.h2T[k][lane], o);
            if (i < n) {
                O[i * PO + u] = o;
                if (u == 0) s_out[i] = sqrtf(scale * softplusf(o));
            }
        }
        __syncthreads();
    }
}

// Backward: G_O (n x 33) = dL/do; partial parameter gradients per block.
__global__ void __launch_bounds__(PT, 1)
mlp_backward_kernel(const float* __restrict__ theta, const float* __restrict__ X, int64_t n,
                    const float* __restrict__ GO, float* __restrict__ gpart)
{
    extern __shared__ __align__(16) unsigned char mlp_raw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(mlp_raw);
    load_weights(S, theta);
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    // register-held gradient accumulators
    const int u2 = t >> 1, kh = (t & 1) * 64;      // dW2[u2][kh .. kh+63]
    float gW2[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) gW2[j] = 0.f;
    const int k3 = t >> 1, uh = (t & 1) ? 17 : 0, un = (t & 1) ? 16 : 17;   // dW3[uh..uh+un-1][k3]
    float gW3[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) gW3[j] = 0.f;
    float gW1[PF] = {0.f, 0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;   // unit t < PH / output t < PO

    const int64_t tiles = (n + TP - 1) / TP;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t p0 = tile * TP;
        for (int e = t; e < TP * PO; e += PT) {
            const int64_t i = p0 + e / PO;
            S.goT[e % PO][e / PO] = i < n ? GO[i * PO + e % PO] : 0.f;
        }
        tile_forward(S, X, p0, n);   // syncs; goT visible too
        // dW3, db3
        for (int p = 0; p < TP; ++p) {
            const float hk = S.h2N[p][k3];
#pragma unroll
            for (int j = 0; j < 17; ++j)
                if (j < un) gW3[j] = fmaf(S.goT[uh + j][p], hk, gW3[j]);
        }
        if (t < PO)
            for (int p = 0; p < TP; ++p) gb3 += S.goT[t][p];
        // gz2 = (go W3) * [h2 > 0]
        {
            const int p = lane, k0 = w * 16;
            float acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
            for (int u = 0; u < PO; ++u) {
                const float g = S.goT[u][p];
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = fmaf(g, S.W3[u * PH + k0 + j], acc[j]);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float g = S.h2T[k0 + j][p] > 0.f ? acc[j] : 0.f;
                S.gz2T[k0 + j][p] = g;
                S.gz2N[p][k0 + j] = g;
            }
        }
        __syncthreads();
        // dW2, db2
        for (int p = 0; p < TP; ++p) {
            const float g = S.gz2N[p][u2];
#pragma unroll
            for (int j = 0; j < 64; ++j) gW2[j] = fmaf(g, S.h1N[p][kh + j], gW2[j]);
        }
        if (t < PH)
            for (int p = 0; p < TP; ++p) gb2 += S.gz2T[t][p];
        // gz1 = (gz2 W2) * [h1 > 0], written over h2T (no longer needed)
        {
            const int p = lane, k0 = w * 16;
            float acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
            for (int u = 0; u < PH; ++u) {
                const float g = S.gz2T[u][p];
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = fmaf(g, S.W2[u * PH + k0 + j], acc[j]);
            }
            __syncthreads();   // every thread finished reading h2T (masks) before it is overwritten
#pragma unroll
            for (int j = 0; j < 16; ++j) S.h2T[k0 + j][p] = S.h1T[k0 + j][p] > 0.f ? acc[j] : 0.f;
        }
        __syncthreads();
        // dW1, db1
        if (t < PH)
            for (int p = 0; p < TP; ++p) {
                const float g = S.h2T[t][p];
                gb1 += g;
#pragma unroll
                for (int f = 0; f < PF; ++f) gW1[f] = fmaf(g, S.X[p][f], gW1[f]);
            }
        __syncthreads();
    }
    float* out = gpart + (int64_t)blockIdx.x * NPARAM;
#pragma unroll
    for (int j = 0; j < 64; ++j) out[OFF_W2 + u2 * PH + kh + j] = gW2[j];
#pragma unroll
    for (int j = 0; j < 17; ++j)
        if (j < un) out[OFF_W3 + (uh + j) * PH + k3] = gW3[j];
    if (t < PH) {
#pragma unroll
        for (int f = 0; f < PF; ++f) out[OFF_W1 + t * PF + f] = gW1[f];
        out[OFF_B1 + t] = gb1;
        out[OFF_B2 + t] = gb2;
    }
    if (t < PO) out[OFF_B3 + t] = gb3;
}

__global__ void grad_reduce_kernel(const float* __restrict__ gpart, int nb, float* __restrict__ grad)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NPARAM; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += gpart[(int64_t)b * NPARAM + j];
        grad[j] = (float)s;
    }
}

// per-block sums of r.e and e.e
template <class TR>
__global__ void rescale_kernel(const TR* __restrict__ R, const TR* __restrict__ E, int64_t n, double* __restrict__ part)
{
    __shared__ double sh[2][256];
    double re = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = ldv(E[i]);
        re += ldv(R[i]) * e;
        rr += e * e;
    }
    sh[0][threadIdx.x] = re;
    sh[1][threadIdx.x] = rr;
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int l = 0; l < 256; ++l) s += sh[threadIdx.x][l];
        part[2 * blockIdx.x + threadIdx.x] = s;
    }
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1c, float b2c)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NPARAM; j += gridDim.x * blockDim.x) {
        m[j] = b1 * m[j] + (1.f - b1) * g[j];
        v[j] = b2 * v[j] + (1.f - b2) * g[j] * g[j];
        th[j] -= lr * (m[j] / b1c) / (sqrtf(v[j] / b2c) + eps);
    }
}

// ------------------------------------------------------------------ BF16 tensor-core MLP
// Padded widths of the GEMM operands: the 6 features and the constant one in 64 columns, the
// 33 outputs in 64 columns (forward) and 128 rows (the transposed output gradient).
constexpr int XW = 64;       // [x | 1 | 0...] width
constexpr int OW = 64;       // output width of the layer-3 GEMM
constexpr int OTR = 128;     // rows of the transposed output gradient

__device__ __forceinline__ __nv_bfloat16 bf(float x) { return __float2bfloat16_rn(x); }

// BF16 weight operands from the FP32 parameters (every one K-major for the GEMM):
// W1b[u][f] = W1[u][f] (f < 6), b1[u] (f = 6), 0; W2b = W2; W2T[k][u] = W2[u][k];
// W3b[o][k] = W3[o][k] (o < 33), 0; W3T[k][o] = W3[o][k] (o < 33), 0.
__global__ void pack_weights_kernel(const float* __restrict__ th, __nv_bfloat16* __restrict__ W1b,
                                    __nv_bfloat16* __restrict__ W2b, __nv_bfloat16* __restrict__ W2T,
                                    __nv_bfloat16* __restrict__ W3b, __nv_bfloat16* __restrict__ W3T)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int e = tid; e < PH * XW; e += nt) {
        const int u = e / XW, f = e % XW;
        W1b[e] = bf(f < PF ? th[OFF_W1 + u * PF + f] : f == PF ? th[OFF_B1 + u] : 0.f);
    }
    for (int e = tid; e < PH * PH; e += nt) {
        const int u = e / PH, k = e % PH;
        W2b[e] = bf(th[OFF_W2 + e]);
        W2T[k * PH + u] = bf(th[OFF_W2 + e]);
    }
    for (int e = tid; e < OW * PH; e += nt) {
        const int o = e / PH, k = e % PH;
        const float w = o < PO ? th[OFF_W3 + o * PH + k] : 0.f;
        W3b[e] = bf(w);
        W3T[k * OW + o] = bf(w);
    }
}

// Xb[i] = [x_i | 1 | 0...] (n x 64), XbT its transpose (64 x np, zero past n)
__global__ void pack_x_kernel(const float* __restrict__ X, int64_t n, int64_t np, __nv_bfloat16* __restrict__ Xb,
                              __nv_bfloat16* __restrict__ XbT)
{
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * XW; e += nt) {
        const int64_t i = e / XW;
        const int f = (int)(e % XW);
        Xb[e] = bf(f < PF ? X[i * PF + f] : f == PF ? 1.f : 0.f);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)XW * np; e += nt) {
        const int f = (int)(e / np);
        const int64_t i = e % np;
        XbT[e] = bf(i < n && f < PF ? X[i * PF + f] : (i < n && f == PF) ? 1.f : 0.f);
    }
}

// One block per 32 pairs: h = relu(z + b) (b may be NULL) to H (n x 128) and, if HT, to its
// transpose HT (128 x np; zero for the padding pairs n <= i < np).
constexpr int ACT_ROWS = 32;
__global__ void __launch_bounds__(256)
act_kernel(const float* __restrict__ Z, const float* __restrict__ th_bias, int64_t n, int64_t np,
           __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ HT)
{
    __shared__ float tile[ACT_ROWS][PH + 1];
    const int64_t i0 = (int64_t)blockIdx.x * ACT_ROWS;
    for (int e = threadIdx.x; e < ACT_ROWS * PH; e += blockDim.x) {
        const int r = e / PH, u = e % PH;
        const int64_t i = i0 + r;
        float h = 0.f;
        if (i < n) {
            h = fmaxf(Z[i * PH + u] + (th_bias ? th_bias[u] : 0.f), 0.f);
            H[i * PH + u] = bf(h);
        }
        tile[r][u] = h;
    }
    if (!HT) return;
    __syncthreads();
    for (int e = threadIdx.x; e < ACT_ROWS * PH; e += blockDim.x) {
        const int u = e / ACT_ROWS, r = e % ACT_ROWS;
        const int64_t i = i0 + r;
        if (i < np) HT[(int64_t)u * np + i] = bf(tile[r][u]);
    }
}

// O[i][o] = Ob[i][o] + b3[o] (o < 33), s_i = sqrt(scale softplus(o_0))
__global__ void out3_kernel(const float* __restrict__ Ob, const float* __restrict__ th, int64_t n,
                            float* __restrict__ O, float* __restrict__ s_out, float scale)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * PO;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / PO;
        const int o = (int)(e % PO);
        const float v = Ob[i * OW + o] + th[OFF_B3 + o];
        O[e] = v;
        if (o == 0) s_out[i] = sqrtf(scale * softplusf(v));
    }
}

// output gradient to the GEMM operands: dOb (n x 64, zero past 33) and dOT (128 x np, zero past
// 33 rows and n columns)
__global__ void pack_go_kernel(const float* __restrict__ GO, int64_t n, int64_t np, __nv_bfloat16* __restrict__ dOb,
                               __nv_bfloat16* __restrict__ dOT)
{
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * OW; e += nt) {
        const int64_t i = e / OW;
        const int o = (int)(e % OW);
        dOb[e] = bf(o < PO ? GO[i * PO + o] : 0.f);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)OTR * np; e += nt) {
        const int o = (int)(e / np);
        const int64_t i = e % np;
        dOT[e] = bf(o < PO && i < n ? GO[i * PO + o] : 0.f);
    }
}

// One block per 32 pairs: g = D [H > 0] to G (n x 128, if G) and GT (128 x np); per-block
// column sums of g (FP64) into part[block][128] (if part).
__global__ void __launch_bounds__(256)
relu_grad_kernel(const float* __restrict__ D, const __nv_bfloat16* __restrict__ Hm, int64_t n, int64_t np,
                 __nv_bfloat16* __restrict__ G, __nv_bfloat16* __restrict__ GT, double* __restrict__ part)
{
    __shared__ float tile[ACT_ROWS][PH + 1];
    const int64_t i0 = (int64_t)blockIdx.x * ACT_ROWS;
    for (int e = threadIdx.x; e < ACT_ROWS * PH; e += blockDim.x) {
        const int r = e / PH, u = e % PH;
        const int64_t i = i0 + r;
        float g = 0.f;
        if (i < n) {
            g = __bfloat162float(Hm[i * PH + u]) > 0.f ? D[i * PH + u] : 0.f;
            if (G) G[i * PH + u] = bf(g);
        }
        tile[r][u] = g;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ACT_ROWS * PH; e += blockDim.x) {
        const int u = e / ACT_ROWS, r = e % ACT_ROWS;
        const int64_t i = i0 + r;
        if (i < np) GT[(int64_t)u * np + i] = bf(tile[r][u]);
    }
    if (part && threadIdx.x < PH) {
        double acc = 0.0;
        for (int r = 0; r < ACT_ROWS; ++r) acc += (double)tile[r][threadIdx.x];
        part[(int64_t)blockIdx.x * PH + threadIdx.x] = acc;
    }
}

// column sums of GO (n x 33) per block of 256 pairs (FP64)
__global__ void go_colsum_kernel(const float* __restrict__ GO, int64_t n, double* __restrict__ part)
{
    __shared__ double sh[8][PO];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double a0 = 0.0, a1 = 0.0;   // columns lane and 32 + lane (lane 0 only)
    for (int64_t i = (int64_t)blockIdx.x * 256 + w; i < n && i < (int64_t)(blockIdx.x + 1) * 256; i += 8) {
        a0 += GO[i * PO + lane];
        if (lane == 0) a1 += GO[i * PO + 32];
    }
    sh[w][lane] = a0;
    if (lane == 0) sh[w][32] = a1;
    __syncthreads();
    if (threadIdx.x < PO) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[k][threadIdx.x];
        part[(int64_t)blockIdx.x * PO + threadIdx.x] = t;
    }
}

// gradient vector from the GEMM outputs and the bias partial sums (summed in block order)
__global__ void grad_assemble_kernel(const float* __restrict__ dW1g, const float* __restrict__ dW2g,
                                     const float* __restrict__ dW3g, const double* __restrict__ db2part, int nb2,
                                     const double* __restrict__ db3part, int nb3, float* __restrict__ grad)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NPARAM; j += gridDim.x * blockDim.x) {
        float g;
        if (j < OFF_B1) {
            const int u = (j - OFF_W1) / PF, f = (j - OFF_W1) % PF;
            g = dW1g[u * XW + f];
        } else if (j < OFF_W2) {
            g = dW1g[(j - OFF_B1) * XW + PF];
        } else if (j < OFF_B2) {
            g = dW2g[j - OFF_W2];
        } else if (j < OFF_W3) {
            double t = 0.0;
            for (int b = 0; b < nb2; ++b) t += db2part[(int64_t)b * PH + (j - OFF_B2)];
            g = (float)t;
        } else if (j < OFF_B3) {
            g = dW3g[j - OFF_W3];   // rows o < 33 of the 128 x 128 product, row-major like W3
        } else {
            double t = 0.0;
            for (int b = 0; b < nb3; ++b) t += db3part[(int64_t)b * PO + (j - OFF_B3)];
            g = (float)t;
        }
        grad[j] = g;
    }
}

// ------------------------------------------------------------------ low-rank algebra
constexpr int RB = 256;   // blocks of the reduction kernels

// partial Gram V^T V (32 x 32) per block
__global__ void __launch_bounds__(256) gram_kernel(const float* __restrict__ O, int64_t n, double* __restrict__ part)
{
    const int a = threadIdx.x >> 3, b0 = (threadIdx.x & 7) * 4;   // thread -> row a, 4 columns
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const float* v = O + i * PO + 1;
        const double va = v[a];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += va * (double)v[b0 + c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) part[(int64_t)blockIdx.x * PR * PR + a * PR + b0 + c] = acc[c];
}

// G = I + sum of parts; Cholesky factor L (lower, FP64) in place; one block of 32 threads
__global__ void chol_kernel(const double* __restrict__ part, int nb, double* __restrict__ L)
{
    __shared__ double G[PR][PR + 1];
    const int r = threadIdx.x;
    for (int c = 0; c < PR; ++c) {
        double s = (r == c) ? 1.0 : 0.0;
        for (int b = 0; b < nb; ++b) s += part[(int64_t)b * PR * PR + r * PR + c];
        G[r][c] = s;
    }
    __syncwarp();
    for (int k = 0; k < PR; ++k) {
        if (r == k) G[k][k] = sqrt(G[k][k]);
        __syncwarp();
        if (r > k) G[r][k] /= G[k][k];
        __syncwarp();
        if (r > k)
            for (int c = k + 1; c <= r; ++c) G[r][c] -= G[r][k] * G[c][k];
        __syncwarp();
    }
    for (int c = 0; c < PR; ++c) L[r * PR + c] = c <= r ? G[r][c] : 0.0;
}

// solve (L L^T) x = b for `cols` right-hand sides stored as H[j * cols + k]; one thread per column
__device__ void chol_solve_cols(const double* L, double* H, int cols, int k)
{
    double x[PR];
    for (int i = 0; i < PR; ++i) {
        double s = H[i * cols + k];
        for (int j = 0; j < i; ++j) s -= L[i * PR + j] * x[j];
        x[i] = s / L[i * PR + i];
    }
    for (int i = PR - 1; i >= 0; --i) {
        double s = x[i];
        for (int j = i + 1; j < PR; ++j) s -= L[j * PR + i] * x[j];
        x[i] = s / L[i * PR + i];
    }
    for (int i = 0; i < PR; ++i) H[i * cols + k] = x[i];
}

// partial h_k = V^T (s * r_k) (32 x K) and ||e_k||^2 (optional) per block; R, E column-major n x K
template <class T>
__global__ void __launch_bounds__(256)
vtz_kernel(const float* __restrict__ O, const float* __restrict__ s, const T* __restrict__ R, int64_t n, int K,
           const T* __restrict__ E, double* __restrict__ part, double* __restrict__ epart)
{
    // thread: column k = tid / 32 (8 columns per pass), rank index j = lane
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k0 = 0; k0 < K; k0 += 8) {
        const int k = k0 + w;
        double acc = 0.0, ee = 0.0;
        if (k < K)
            for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
                const double z = (double)s[i] * ldv(R[(int64_t)k * n + i]);
                acc += (double)O[i * PO + 1 + lane] * z;
                if (E && lane == 0) {
                    const double e = ldv(E[(int64_t)k * n + i]);
                    ee += e * e;
                }
            }
        if (k < K) {
            part[((int64_t)blockIdx.x * PR + lane) * K + k] = acc;
            if (E && lane == 0) epart[(int64_t)blockIdx.x * K + k] = ee;
        }
    }
}

// H (32 x K) = sum of parts, then H <- G^{-1} H; also ||e||^2 sums (if epart)
__global__ void sum_solve_kernel(const double* __restrict__ part, const double* __restrict__ epart, int nb, int K,
                                 const double* __restrict__ L, double* __restrict__ H, double* __restrict__ ee)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    for (int j = 0; j < PR; ++j) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[((int64_t)b * PR + j) * K + k];
        H[j * K + k] = s;
    }
    if (epart && ee) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += epart[(int64_t)b * K + k];
        ee[k] = s;
    }
    chol_solve_cols(L, H, K, k);
}

// z = P r = s (s r - V c)
template <class T>
__global__ void papply_kernel(const float* __restrict__ O, const float* __restrict__ s, const double* __restrict__ C,
                              const T* __restrict__ r, T* __restrict__ z, int64_t n)
{
    __shared__ double c[PR];
    if (threadIdx.x < PR) c[threadIdx.x] = C[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float* v = O + i * PO + 1;
        double vc = 0.0;
#pragma unroll
        for (int j = 0; j < PR; ++j) vc += (double)v[j] * c[j];
        const double si = s[i];
        z[i] = (T)(si * (si * (double)r[i] - vc));
    }
}

// ------------------------------------------------------------------ loss passes
constexpr int KMAX = 16;   // pairs per minibatch

// pass 1: per k, loss numerator sum of rho^2, and g_c = -V^T g_y (partials)
template <class TR>
__global__ void __launch_bounds__(256)
loss_pass1_kernel(const float* __restrict__ O, const float* __restrict__ s, const TR* __restrict__ R,
                  const TR* __restrict__ E, int64_t n, int K, const double* __restrict__ C,
                  const double* __restrict__ ee, double* __restrict__ lpart, double* __restrict__ gpart)
{
    __shared__ double c[PR * KMAX];
    __shared__ double red[8][PR + 1];
    for (int e = threadIdx.x; e < PR * K; e += blockDim.x) c[e] = C[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < K; ++k) {
        double lsum = 0.0, gacc = 0.0;   // lane j accumulates g_c[j]
        for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
            const float* v = O + i * PO + 1;
            const double vj = v[lane];
            double vc = vj * c[lane * K + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vc += __shfl_xor_sync(0xffffffffu, vc, o);
            const double si = s[i], r = ldv(R[(int64_t)k * n + i]), e = ldv(E[(int64_t)k * n + i]);
            const double y = si * r - vc;
            const double rho = si * y - e;
            const double gout = 2.0 * rho / (ee[k] * K);
            const double gy = si * gout;
            if (lane == 0) lsum += rho * rho / (ee[k] * K);
            gacc -= vj * gy;
        }
        red[w][lane] = gacc;
        if (lane == 0) red[w][PR] = lsum;
        __syncthreads();
        if (threadIdx.x < PR + 1) {
            double t = 0.0;
            for (int ww = 0; ww < 8; ++ww) t += red[ww][threadIdx.x];
            if (threadIdx.x < PR) gpart[((int64_t)blockIdx.x * PR + threadIdx.x) * K + k] = t;
            else lpart[(int64_t)blockIdx.x * K + k] = t;
        }
        __syncthreads();
    }
}

// pass 2: per-pair output gradient dL/do (n x 33); Gh = G^{-1} g_c, sym = g_G + g_G^T
template <class TR>
__global__ void __launch_bounds__(256)
loss_pass2_kernel(const float* __restrict__ O, const float* __restrict__ s, const TR* __restrict__ R,
                  const TR* __restrict__ E, int64_t n, int K, const double* __restrict__ C,
                  const double* __restrict__ Gh, const double* __restrict__ sym, const double* __restrict__ ee,
                  float* __restrict__ GO, double scale)
{
    __shared__ double c[PR * KMAX], gh[PR * KMAX], sy[PR * PR];
    for (int e = threadIdx.x; e < PR * K; e += blockDim.x) {
        c[e] = C[e];
        gh[e] = Gh[e];
    }
    for (int e = threadIdx.x; e < PR * PR; e += blockDim.x) sy[e] = sym[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
        const float* orow = O + i * PO;
        const double vj = orow[1 + lane];
        const double si = s[i];
        double gV = 0.0, gs = 0.0;
        for (int k = 0; k < K; ++k) {
            double vc = vj * c[lane * K + k], vg = vj * gh[lane * K + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vc += __shfl_xor_sync(0xffffffffu, vc, o);
                vg += __shfl_xor_sync(0xffffffffu, vg, o);
            }
            const double r = ldv(R[(int64_t)k * n + i]), e = ldv(E[(int64_t)k * n + i]);
            const double z = si * r;
            const double y = z - vc;
            const double rho = si * y - e;
            const double gout = 2.0 * rho / (ee[k] * K);
            const double gy = si * gout;
            const double gz = gy + vg;
            gs += y * gout + r * gz;
            gV += -gy * c[lane * K + k] + z * gh[lane * K + k];
        }
        // g_V += V (sym): row i of V times the 32 x 32 matrix
        double vs = 0.0;
        for (int a = 0; a < PR; ++a) vs += (double)orow[1 + a] * sy[a * PR + lane];
        gV += vs;
        float* go = GO + i * PO;
        go[1 + lane] = (float)gV;
        if (lane == 0) {
            // only V is trained: the diagonal output keeps its initial value
            go[0] = 0.f;
        }
    }
}

// sum partials, loss, Gh = G^{-1} g_c, sym = -(Gh C^T + C Gh^T)  (g_G = -sum_k gh_k c_k^T)
__global__ void loss_mid_kernel(const double* __restrict__ lpart, const double* __restrict__ gpart, int nb, int K,
                                const double* __restrict__ L, const double* __restrict__ C, double* __restrict__ Gh,
                                double* __restrict__ sym, double* __restrict__ loss)
{
    const int k = threadIdx.x;
    if (k < K) {
        for (int j = 0; j < PR; ++j) {
            double s = 0.0;
            for (int b = 0; b < nb; ++b) s += gpart[((int64_t)b * PR + j) * K + k];
            Gh[j * K + k] = s;
        }
        chol_solve_cols(L, Gh, K, k);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = 0.0;
        for (int kk = 0; kk < K; ++kk)
            for (int b = 0; b < nb; ++b) l += lpart[(int64_t)b * K + kk];
        *loss = l;
    }
    for (int e = threadIdx.x; e < PR * PR; e += blockDim.x) {
        const int a = e / PR, b = e % PR;
        double g = 0.0;
        for (int kk = 0; kk < K; ++kk) g += Gh[a * K + kk] * C[b * K + kk] + C[a * K + kk] * Gh[b * K + kk];
        sym[e] = -g;
    }
}

}  // namespace
}  // namespace gvt

// ------------------------------------------------------------------ object and host logic
struct gvt_precond {
    gvt_handle* h = nullptr;
    int64_t n = 0;
    float* theta = nullptr;
    float* X = nullptr;
    float* O = nullptr;
    float* s = nullptr;
    double* L = nullptr;     // 32 x 32 Cholesky factor of I + V^T V
    double* red = nullptr;   // reduction scratch
    double* H = nullptr;     // 32 x KMAX
    double* Gh = nullptr;
    double* sym = nullptr;
    double* ee = nullptr;
    double* loss = nullptr;
    double* lpart = nullptr;
    float* GO = nullptr;
    float* gpart = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    int64_t step = 0;
    float mu[gvt::PF], sd[gvt::PF];
    double scale = 1.0;      // D = scale * softplus(o_0)
    bool ready = false;      // O, s, L hold the current parameters' outputs
    int dtype = GVT_BF16;    // arithmetic of the network: GVT_BF16 (tensor cores) or GVT_F32 (SIMT)
    // BF16 path (allocated on first use): operands of the GEMMs, np = n rounded up to 64
    int64_t np = 0;
    bool bf_ready = false;   // buffers allocated and the features packed
    bool acts_t = false;     // the transposed activations of the current parameters are stored
    __nv_bfloat16 *Xb = nullptr, *XbT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr;
    __nv_bfloat16 *dOb = nullptr, *dOT = nullptr, *dZ2 = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2T = nullptr, *W3b = nullptr, *W3T = nullptr;
    float *Z = nullptr, *Ob = nullptr, *dW1g = nullptr, *dW2g = nullptr, *dW3g = nullptr;
    double *db2part = nullptr, *db3part = nullptr;
    std::vector<void*> allocs;
};

using namespace gvt;

namespace {

const int kMlpBlocks = 152;

template <class P_>
gvt_status palloc(gvt_precond* p, P_** out, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(P_)) != cudaSuccess) {
        cudaGetLastError();
        set_error("preconditioner: device allocation failed");
        return GVT_ERR_ALLOC;
    }
    p->allocs.push_back(q);
    *out = static_cast<P_*>(q);
    return GVT_OK;
}

// set on every forward pass: the attribute belongs to the current device's context (cheap)
gvt_status mlp_smem_attr()
{
    GVT_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem)));
    GVT_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem)));
    return GVT_OK;
}

unsigned ew_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// BF16 path: buffers and the packed features, once
gvt_status bf16_setup(gvt_precond* p, cudaStream_t st)
{
    if (p->bf_ready) return GVT_OK;
    const int64_t n = std::max<int64_t>(p->n, 1);
    p->np = (n + 63) / 64 * 64;
    const int64_t np = p->np;
    GVT_CHECK(palloc(p, &p->Xb, n * XW)); GVT_CHECK(palloc(p, &p->XbT, XW * np));
    GVT_CHECK(palloc(p, &p->H1, n * PH)); GVT_CHECK(palloc(p, &p->H1T, PH * np));
    GVT_CHECK(palloc(p, &p->H2, n * PH)); GVT_CHECK(palloc(p, &p->H2T, PH * np));
    GVT_CHECK(palloc(p, &p->dOb, n * OW)); GVT_CHECK(palloc(p, &p->dOT, OTR * np));
    GVT_CHECK(palloc(p, &p->dZ2, n * PH)); GVT_CHECK(palloc(p, &p->dZ2T, PH * np)); GVT_CHECK(palloc(p, &p->dZ1T, PH * np));
    GVT_CHECK(palloc(p, &p->W1b, PH * XW)); GVT_CHECK(palloc(p, &p->W2b, PH * PH)); GVT_CHECK(palloc(p, &p->W2T, PH * PH));
    GVT_CHECK(palloc(p, &p->W3b, OW * PH)); GVT_CHECK(palloc(p, &p->W3T, PH * OW));
    GVT_CHECK(palloc(p, &p->Z, n * PH)); GVT_CHECK(palloc(p, &p->Ob, n * OW));
    GVT_CHECK(palloc(p, &p->dW1g, PH * XW)); GVT_CHECK(palloc(p, &p->dW2g, PH * PH)); GVT_CHECK(palloc(p, &p->dW3g, OTR * PH));
    GVT_CHECK(palloc(p, &p->db2part, (np / ACT_ROWS) * PH));
    GVT_CHECK(palloc(p, &p->db3part, ((n + 255) / 256) * PO));
    if (p->n > 0) {
        pack_x_kernel<<<ew_grid(XW * np), 256, 0, st>>>(p->X, p->n, np, p->Xb, p->XbT);
        GVT_LAUNCH_CHECK("preconditioner pack features");
    }
    p->bf_ready = true;
    return GVT_OK;
}

// C (rows x cols, ld ldc) = A B^T on the tensor cores (BF16 operands, K-major)
gvt_status gemm_bf16(gvt_precond* p, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb,
                     float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, cudaStream_t st)
{
    return tc_gemm_bf16(A, lda, B, ldb, C, ldc, M, N, K, handle_err_word(p->h), st, GVT_TC_PAIRS_OFF);
}

// BF16 forward: O and s (and, with want_t, the transposed activations for the backward GEMMs)
gvt_status forward_bf16(gvt_precond* p, bool want_t, cudaStream_t st)
{
    GVT_CHECK(bf16_setup(p, st));
    const int64_t n = p->n, np = p->np;
    if (n == 0) return GVT_OK;
    pack_weights_kernel<<<64, 256, 0, st>>>(p->theta, p->W1b, p->W2b, p->W2T, p->W3b, p->W3T);
    GVT_LAUNCH_CHECK("preconditioner pack weights");
    const unsigned ab = (unsigned)(np / ACT_ROWS);
    GVT_CHECK(gemm_bf16(p, p->Xb, XW, p->W1b, XW, p->Z, PH, n, PH, XW, st));
    act_kernel<<<ab, 256, 0, st>>>(p->Z, nullptr, n, np, p->H1, want_t ? p->H1T : nullptr);
    GVT_LAUNCH_CHECK("preconditioner layer 1");
    GVT_CHECK(gemm_bf16(p, p->H1, PH, p->W2b, PH, p->Z, PH, n, PH, PH, st));
    act_kernel<<<ab, 256, 0, st>>>(p->Z, p->theta + OFF_B2, n, np, p->H2, want_t ? p->H2T : nullptr);
    GVT_LAUNCH_CHECK("preconditioner layer 2");
    GVT_CHECK(gemm_bf16(p, p->H2, PH, p->W3b, PH, p->Ob, OW, n, OW, PH, st));
    out3_kernel<<<ew_grid(n * PO), 256, 0, st>>>(p->Ob, p->theta, n, p->O, p->s, (float)p->scale);
    GVT_LAUNCH_CHECK("preconditioner layer 3");
    p->acts_t = want_t;
    return GVT_OK;
}

// BF16 backward from GO = dL/do (n x 33): p->grad (the forward with want_t must be current)
gvt_status backward_bf16(gvt_precond* p, cudaStream_t st)
{
    const int64_t n = p->n, np = p->np;
    if (n == 0) return GVT_OK;
    const unsigned ab = (unsigned)(np / ACT_ROWS);
    const int nb3 = (int)((n + 255) / 256);
    pack_go_kernel<<<ew_grid(OTR * np), 256, 0, st>>>(p->GO, n, np, p->dOb, p->dOT);
    go_colsum_kernel<<<nb3, 256, 0, st>>>(p->GO, n, p->db3part);
    GVT_LAUNCHED(2, "preconditioner output gradient");
    GVT_CHECK(gemm_bf16(p, p->dOb, OW, p->W3T, OW, p->Z, PH, n, PH, OW, st));            // dH2
    relu_grad_kernel<<<ab, 256, 0, st>>>(p->Z, p->H2, n, np, p->dZ2, p->dZ2T, p->db2part);
    GVT_LAUNCH_CHECK("preconditioner layer-2 gradient");
    GVT_CHECK(gemm_bf16(p, p->dZ2, PH, p->W2T, PH, p->Z, PH, n, PH, PH, st));            // dH1
    relu_grad_kernel<<<ab, 256, 0, st>>>(p->Z, p->H1, n, np, nullptr, p->dZ1T, nullptr);
    GVT_LAUNCH_CHECK("preconditioner layer-1 gradient");
    GVT_CHECK(gemm_bf16(p, p->dZ1T, np, p->XbT, np, p->dW1g, XW, PH, XW, np, st));       // dW1 | db1
    GVT_CHECK(gemm_bf16(p, p->dZ2T, np, p->H1T, np, p->dW2g, PH, PH, PH, np, st));       // dW2
    GVT_CHECK(gemm_bf16(p, p->dOT, np, p->H2T, np, p->dW3g, PH, OTR, PH, np, st));       // dW3
    grad_assemble_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(p->dW1g, p->dW2g, p->dW3g, p->db2part, (int)ab,
                                                                p->db3part, nb3, p->grad);
    GVT_LAUNCH_CHECK("preconditioner gradient");
    return GVT_OK;
}

// O, s, L for the current parameters (with want_t, in BF16, also the activations the backward
// GEMMs read)
gvt_status forward(gvt_precond* p, cudaStream_t st, bool want_t = false)
{
    if (p->dtype == GVT_BF16) {
        GVT_CHECK(forward_bf16(p, want_t, st));
    } else {
        GVT_CHECK(mlp_smem_attr());
        mlp_forward_kernel<<<kMlpBlocks * 1, PT, sizeof(MlpSmem), st>>>(p->theta, p->X, p->n, p->O, p->s,
                                                                        (float)p->scale);
        GVT_LAUNCH_CHECK("preconditioner forward");
    }
    gram_kernel<<<RB, 256, 0, st>>>(p->O, p->n, p->red);
    chol_kernel<<<1, PR, 0, st>>>(p->red, RB, p->L);
    GVT_LAUNCHED(2, "preconditioner forward");
    p->ready = true;
    return GVT_OK;
}

}  // namespace

namespace gvt {
// z = P r for FP32 or FP64 vectors of length n (the parameters' outputs must be current)
template <class T>
gvt_status precond_apply(gvt_precond* p, const T* r, T* z, cudaStream_t st)
{
    if (!p->ready) GVT_CHECK(forward(p, st));
    vtz_kernel<T><<<RB, 256, 0, st>>>(p->O, p->s, r, p->n, 1, nullptr, p->red, nullptr);
    sum_solve_kernel<<<1, 32, 0, st>>>(p->red, nullptr, RB, 1, p->L, p->H, nullptr);
    papply_kernel<T><<<152 * 8, 256, 0, st>>>(p->O, p->s, p->H, r, z, p->n);
    GVT_LAUNCHED(3, "preconditioner apply");
    return GVT_OK;
}
template gvt_status precond_apply<float>(gvt_precond*, const float*, float*, cudaStream_t);
template gvt_status precond_apply<double>(gvt_precond*, const double*, double*, cudaStream_t);
int64_t precond_size(const gvt_precond* p) { return p->n; }
}  // namespace gvt

namespace {
// loss and dL/dtheta (into p->grad) for K <= KMAX pairs (R, E stored as TR)
template <class TR>
gvt_status loss_grad(gvt_precond* p, const TR* R, const TR* E, int K, cudaStream_t st)
{
    GVT_CHECK(forward(p, st, true));
    const int64_t n = p->n;
    double* part = p->red;                       // RB * 32 * K
    double* epart = p->red + (size_t)RB * PR * KMAX;
    vtz_kernel<TR><<<RB, 256, 0, st>>>(p->O, p->s, R, n, K, E, part, epart);
    sum_solve_kernel<<<1, 32, 0, st>>>(part, epart, RB, K, p->L, p->H, p->ee);
    loss_pass1_kernel<TR><<<RB, 256, 0, st>>>(p->O, p->s, R, E, n, K, p->H, p->ee, p->lpart, part);
    loss_mid_kernel<<<1, 256, 0, st>>>(p->lpart, part, RB, K, p->L, p->H, p->Gh, p->sym, p->loss);
    loss_pass2_kernel<TR><<<RB * 2, 256, 0, st>>>(p->O, p->s, R, E, n, K, p->H, p->Gh, p->sym, p->ee, p->GO,
                                                  p->scale);
    GVT_LAUNCHED(5, "preconditioner loss");
    if (p->dtype == GVT_BF16) return backward_bf16(p, st);
    mlp_backward_kernel<<<kMlpBlocks, PT, sizeof(MlpSmem), st>>>(p->theta, p->X, n, p->GO, p->gpart);
    grad_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(p->gpart, kMlpBlocks, p->grad);
    GVT_LAUNCHED(2, "preconditioner backward");
    return GVT_OK;
}
}  // namespace

extern "C" {

gvt_status gvt_precond_create(gvt_handle* h, gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                              const gvt_matrix* N, const float* theta_host, void* stream, gvt_precond** out)
{
    if (!h || !plan || !desc || !M || !out || !M->data || (!desc->homogeneous && (!N || !N->data))) {
        set_error("gvt_precond_create: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const gvt_matrix* Nn = desc->homogeneous ? M : N;
    if (!plan->out_is_in || M->rows < plan->m_cols || M->cols < plan->m_cols || Nn->rows < plan->q_cols ||
        Nn->cols < plan->q_cols || M->dtype != GVT_F64 || Nn->dtype != GVT_F64) {
        set_error("gvt_precond_create: needs a training plan and square FP64 kernel matrices covering its ids");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gvt_precond* p = new (std::nothrow) gvt_precond();
    if (!p) return GVT_ERR_ALLOC;
    p->h = h;
    p->n = plan->n_in;
    const int64_t n = std::max<int64_t>(p->n, 1);
    auto fail = [&](gvt_status s) { gvt_precond_destroy(p); return s; };
    gvt_status s;
#define PCHK(x) do { if ((s = (x)) != GVT_OK) return fail(s); } while (0)
    PCHK(palloc(p, &p->theta, NPARAM)); PCHK(palloc(p, &p->X, n * PF)); PCHK(palloc(p, &p->O, n * PO));
    PCHK(palloc(p, &p->s, n)); PCHK(palloc(p, &p->L, PR * PR));
    PCHK(palloc(p, &p->red, (size_t)RB * PR * KMAX * 2 + (size_t)RB * PR * PR));
    PCHK(palloc(p, &p->H, PR * KMAX)); PCHK(palloc(p, &p->Gh, PR * KMAX)); PCHK(palloc(p, &p->sym, PR * PR));
    PCHK(palloc(p, &p->ee, KMAX)); PCHK(palloc(p, &p->loss, 1)); PCHK(palloc(p, &p->lpart, (size_t)RB * KMAX));
    PCHK(palloc(p, &p->GO, n * PO)); PCHK(palloc(p, &p->gpart, (size_t)kMlpBlocks * NPARAM));
    PCHK(palloc(p, &p->grad, NPARAM)); PCHK(palloc(p, &p->m, NPARAM)); PCHK(palloc(p, &p->v, NPARAM));
    if (cudaMemcpyAsync(p->theta, theta_host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(p->m, 0, sizeof(float) * NPARAM, st) != cudaSuccess ||
        cudaMemsetAsync(p->v, 0, sizeof(float) * NPARAM, st) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "preconditioner init"));
    if (p->n > 0) {
        // kernel-graph degrees with the exact FP64 operator: g1 = K 1, g2 = K (g1 / mean g1)
        double *ones = nullptr, *g1 = nullptr, *g2 = nullptr;
        PCHK(palloc(p, &ones, n)); PCHK(palloc(p, &g1, n)); PCHK(palloc(p, &g2, n));
        fill_ones_kernel<<<152 * 8, 256, 0, st>>>(ones, p->n);
        count_launches(1);
        PCHK(pairwise_apply<double>(plan, desc, M, Nn, ones, g1, st));
        sum_kernel<<<RB, 256, 0, st>>>(g1, p->n, p->red);
        count_launches(1);
        std::vector<double> part(RB);
        if (cudaMemcpyAsync(part.data(), p->red, sizeof(double) * RB, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "preconditioner features"));
        double tot = 0.0;
        for (double x : part) tot += x;
        const double mean = tot / p->n;
        scale_vec_kernel<<<152 * 8, 256, 0, st>>>(g1, mean != 0.0 ? 1.0 / mean : 1.0, p->n, ones);
        count_launches(1);
        PCHK(pairwise_apply<double>(plan, desc, M, Nn, ones, g2, st));
        feat_kernel<<<152 * 8, 256, 0, st>>>(plan->d_in, plan->t_in, p->n, plan->in_by[0].seg, plan->in_by[1].seg,
                                             static_cast<const double*>(M->data), M->ld,
                                             static_cast<const double*>(Nn->data), Nn->ld, g1, g2, p->X);
        feat_moments_kernel<<<RB, PT, 0, st>>>(p->X, p->n, p->red);
        count_launches(2);
        std::vector<double> mom((size_t)RB * 2 * PF);
        if (cudaMemcpyAsync(mom.data(), p->red, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "preconditioner features"));
        double sum[2 * PF];
        for (int f = 0; f < 2 * PF; ++f) sum[f] = 0.0;
        for (int b = 0; b < RB; ++b)
            for (int f = 0; f < 2 * PF; ++f) sum[f] += mom[(size_t)b * 2 * PF + f];
        FeatNorm fn;
        for (int f = 0; f < PF; ++f) {
            const double mu = sum[f] / p->n;
            const double var = std::max(0.0, sum[PF + f] / p->n - mu * mu);
            p->mu[f] = (float)mu;
            p->sd[f] = var > 1e-20 ? (float)std::sqrt(var) : 1.0f;
            fn.mu[f] = p->mu[f];
            fn.inv[f] = 1.0f / p->sd[f];
        }
        feat_norm_kernel<<<152 * 8, 256, 0, st>>>(p->X, p->n, fn);
        count_launches(1);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "preconditioner create"));
#undef PCHK
    *out = p;
    return GVT_OK;
}

gvt_status gvt_precond_destroy(gvt_precond* p)
{
    if (!p) return GVT_OK;
    cudaDeviceSynchronize();
    for (void* a : p->allocs) cudaFree(a);
    delete p;
    return GVT_OK;
}

int64_t gvt_precond_num_params(void) { return NPARAM; }

gvt_status gvt_precond_set_dtype(gvt_precond* p, int32_t dtype)
{
    if (!p || (dtype != GVT_BF16 && dtype != GVT_F32)) {
        set_error("gvt_precond_set_dtype: bad preconditioner or dtype (GVT_BF16 or GVT_F32)");
        return GVT_ERR_INVALID_ARG;
    }
    if (dtype != p->dtype) {
        p->dtype = dtype;
        p->ready = false;
    }
    return GVT_OK;
}

gvt_status gvt_precond_params(gvt_precond* p, float* host, int32_t set, void* stream)
{
    if (!p || !host) {
        set_error("gvt_precond_params: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GVT_CUDA(cudaMemcpyAsync(set ? (void*)p->theta : (void*)host, set ? (const void*)host : (const void*)p->theta,
                             sizeof(float) * NPARAM, set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st));
    GVT_CUDA(cudaStreamSynchronize(st));
    if (set) p->ready = false;
    return GVT_OK;
}

gvt_status gvt_precond_features(gvt_precond* p, float* mu_sd_host, float* X_dev_out, void* stream)
{
    if (!p) {
        set_error("gvt_precond_features: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    if (mu_sd_host)
        for (int f = 0; f < PF; ++f) {
            mu_sd_host[f] = p->mu[f];
            mu_sd_host[PF + f] = p->sd[f];
        }
    if (X_dev_out && p->n > 0)
        GVT_CUDA(cudaMemcpyAsync(X_dev_out, p->X, sizeof(float) * p->n * PF, cudaMemcpyDeviceToDevice,
                                 static_cast<cudaStream_t>(stream)));
    return GVT_OK;
}

gvt_status gvt_precond_outputs(gvt_precond* p, float* O_dev_out, void* stream)
{
    if (!p || !O_dev_out) {
        set_error("gvt_precond_outputs: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GVT_CHECK(forward(p, st));
    GVT_CUDA(cudaMemcpyAsync(O_dev_out, p->O, sizeof(float) * p->n * PO, cudaMemcpyDeviceToDevice, st));
    return GVT_OK;
}

gvt_status gvt_precond_apply(gvt_precond* p, const void* r, void* z, int32_t dtype, void* stream)
{
    if (!p || (p->n > 0 && (!r || !z)) || (dtype != GVT_F32 && dtype != GVT_F64)) {
        set_error("gvt_precond_apply: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == GVT_F32) return precond_apply<float>(p, static_cast<const float*>(r), static_cast<float*>(z), st);
    return precond_apply<double>(p, static_cast<const double*>(r), static_cast<double*>(z), st);
}

gvt_status gvt_precond_loss_grad(gvt_precond* p, const float* R, const float* E, int64_t K, double* loss_host,
                                 float* grad_host, void* stream)
{
    if (!p || !R || !E || K < 1 || K > KMAX) {
        set_error("gvt_precond_loss_grad: bad argument (1 <= K <= 16)");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GVT_CHECK(loss_grad<float>(p, R, E, (int)K, st));
    if (loss_host) GVT_CUDA(cudaMemcpyAsync(loss_host, p->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_host) GVT_CUDA(cudaMemcpyAsync(grad_host, p->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, st));
    GVT_CUDA(cudaStreamSynchronize(st));
    return GVT_OK;
}

gvt_status gvt_precond_scale(gvt_precond* p, double* get, const double* set)
{
    if (!p) {
        set_error("gvt_precond_scale: NULL");
        return GVT_ERR_INVALID_ARG;
    }
    if (set) {
        if (!(*set > 0.0)) {
            set_error("gvt_precond_scale: the scale must be > 0");
            return GVT_ERR_INVALID_ARG;
        }
        p->scale = *set;
        p->ready = false;
    }
    if (get) *get = p->scale;
    return GVT_OK;
}

}  // extern "C"

namespace {
template <class TR>
gvt_status train(gvt_precond* p, const TR* R, const TR* E, int64_t K_total, int32_t steps, int32_t batch, double lr,
                 double* loss_history, cudaStream_t st)
{
    const int64_t n = p->n;
    if (p->step == 0 && n > 0) {
        // output scale c = sum e.e / sum r.e: e ~ c r fitted towards the corrections (about 1 / lambda)
        rescale_kernel<TR><<<RB, 256, 0, st>>>(R, E, n * K_total, p->red);
        GVT_LAUNCH_CHECK("rescale");
        std::vector<double> part(2 * RB);
        GVT_CUDA(cudaMemcpyAsync(part.data(), p->red, sizeof(double) * 2 * RB, cudaMemcpyDeviceToHost, st));
        GVT_CUDA(cudaStreamSynchronize(st));
        double re = 0.0, ee = 0.0;
        for (int b = 0; b < RB; ++b) {
            re += part[2 * b];
            ee += part[2 * b + 1];
        }
        if (ee > 0.0 && re > 0.0) p->scale = ee / re;
        p->ready = false;
    }
    for (int it = 0; it < steps; ++it) {
        // minibatch: `batch` consecutive pair columns, cycling through the data set
        const int64_t k0 = ((int64_t)it * batch) % K_total;
        const int K = (int)std::min<int64_t>(batch, K_total - k0);
        GVT_CHECK(loss_grad<TR>(p, R + k0 * n, E + k0 * n, K, st));
        ++p->step;
        const float b1c = 1.f - std::pow(0.9f, (float)p->step), b2c = 1.f - std::pow(0.999f, (float)p->step);
        adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(p->theta, p->grad, p->m, p->v, (float)lr, b1c, b2c);
        GVT_LAUNCH_CHECK("adam");
        p->ready = false;
        if (loss_history) GVT_CUDA(cudaMemcpyAsync(loss_history + it, p->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    GVT_CUDA(cudaStreamSynchronize(st));
    return GVT_OK;
}
}  // namespace

extern "C" gvt_status gvt_precond_train(gvt_precond* p, const void* R, const void* E, int32_t data_dtype,
                                        int64_t K_total, int32_t steps, int32_t batch, double lr,
                                        double* loss_history, void* stream)
{
    if (!p || !R || !E || K_total < 1 || steps < 0 || batch < 1 || batch > KMAX || !(lr > 0.0) ||
        (data_dtype != GVT_F32 && data_dtype != GVT_BF16)) {
        set_error("gvt_precond_train: bad argument (1 <= batch <= 16, data GVT_F32 or GVT_BF16)");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (data_dtype == GVT_BF16)
        return train<__nv_bfloat16>(p, static_cast<const __nv_bfloat16*>(R), static_cast<const __nv_bfloat16*>(E),
                                    K_total, steps, batch, lr, loss_history, st);
    return train<float>(p, static_cast<const float*>(R), static_cast<const float*>(E), K_total, steps, batch, lr,
                        loss_history, st);
}
