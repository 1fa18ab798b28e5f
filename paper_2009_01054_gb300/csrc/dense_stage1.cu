// Stage 1 as a dense tensor-core product: S = B W with W densified.
//
// For a two-sided group with dense factor B (Y x K) and input recipe W (the
// sparse K x X matrix of Theorem 1 holding coef * v_j at (bcol_j, x_j)),
// S[Y x X] = B W is computed as the BF16 GEMM  S = A' B'^T  with
//   A' = [hi(B) | hi(B) | lo(B)]     (Y x 3K', K' = K rounded up to 64)
//   B' = [hi(W^T) | lo(W^T) | hi(W^T)] (X x 3K')
// so that A' B'^T = hi*hi + hi*lo + lo*hi: the product of the hi/lo BF16
// splits without the lo*lo term.  Each product is accurate to about
// 3 * 2^-18 relative (the splits are exact to 2^-18 and the dropped term is
// below 2^-18); sums accumulate in FP32 in TMEM.
#include <cuda_bf16.h>

#include "gvt_internal.h"

namespace gvt {
namespace {

__global__ void split3_kernel(const float* __restrict__ src, int64_t ld_src, int64_t rows, int64_t cols, int square,
                              int pattern_b, __nv_bfloat16* __restrict__ dst, int64_t kp)
{
    const int64_t total = rows * kp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kp, k = i % kp;
        float x = (k < cols) ? src[r * ld_src + k] : 0.f;
        if (square) x *= x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        __nv_bfloat16* d = dst + r * 3 * kp + k;
        d[0] = hi;
        d[kp] = pattern_b ? lo : hi;
        d[2 * kp] = pattern_b ? hi : lo;
    }
}

// W^T[x, t] += coef * v[perm_j] for every entry (x = key_j, t = bcol_j)
__global__ void densify_kernel(S1Sources srcs, const int32_t* __restrict__ key0, const int32_t* __restrict__ key1,
                               const int32_t* __restrict__ key2, const int32_t* __restrict__ key3, int64_t n,
                               const float* __restrict__ v, float* __restrict__ Wt, int64_t kp)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int si = 0; si < kMaxSources; ++si) {
            if (si >= srcs.count) break;
            const int32_t* key = si == 0 ? key0 : si == 1 ? key1 : si == 2 ? key2 : key3;
            const S1Source& sr = srcs.src[si];
            atomicAdd(&Wt[(int64_t)key[j] * kp + sr.bcol[j]], (float)sr.coef * v[sr.perm[j]]);
        }
    }
}

__global__ void zero_f32_kernel(float* __restrict__ x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.f;
}

unsigned g1(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace

size_t dense_stage1_workspace(int64_t Y, int64_t K, int64_t X)
{
    const int64_t kp = (K + 63) / 64 * 64;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(2 * (size_t)Y * 3 * kp) + al(4 * (size_t)X * kp) + al(2 * (size_t)X * 3 * kp);
}

gvt_status dense_stage1(const float* B, int64_t ldb, int64_t Y, int64_t K, int square, const S1Sources& srcs,
                        const int32_t* const keys[kMaxSources], int64_t n, const float* v, int64_t X, float* S,
                        int64_t lds, void* ws, int* err, cudaStream_t s)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    const int64_t kp = (K + 63) / 64 * 64;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* p = static_cast<char*>(ws);
    __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(p);
    p += al(2 * (size_t)Y * 3 * kp);
    float* Wt = reinterpret_cast<float*>(p);
    p += al(4 * (size_t)X * kp);
    __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(p);

    split3_kernel<<<g1(Y * kp), 256, 0, s>>>(B, ldb, Y, K, square, 0, Ap, kp);
    zero_f32_kernel<<<g1(X * kp), 256, 0, s>>>(Wt, X * kp);
    GVT_LAUNCHED(2, "dense stage 1 prepare");
    if (n > 0) {
        densify_kernel<<<g1(n), 256, 0, s>>>(srcs, keys[0], keys[1], keys[2], keys[3], n, v, Wt, kp);
        GVT_LAUNCH_CHECK("densify");
    }
    split3_kernel<<<g1(X * kp), 256, 0, s>>>(Wt, kp, X, kp, 0, 1, Bp, kp);
    GVT_LAUNCH_CHECK("split W");
    return tc_gemm_bf16(Ap, 3 * kp, Bp, 3 * kp, S, lds, Y, X, 3 * kp, err, s);
}

}  // namespace gvt
