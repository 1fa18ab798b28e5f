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
// below 2^-18); sums accumulate in FP32 in TMEM.  A' depends only on the
// factor, so a caller that runs several groups with the same factor passes
// reuse_a to keep the split already in the workspace.
#include <cuda_bf16.h>

#include "gvt_internal.h"

namespace gvt {
namespace {

// hi and lo BF16 halves of 8 consecutive values (lo = x - hi, rounded)
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
        h[e] = *reinterpret_cast<const uint32_t*>(&hb);
        l[e] = *reinterpret_cast<const uint32_t*>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// dst row r = [hi | hi | lo] (pattern 0) or [hi | lo | hi] (pattern 1) of src row r,
// each part kp wide (zero beyond cols); 8 columns per thread, 16-byte stores.
__global__ void split3_kernel(const float* __restrict__ src, int64_t ld_src, int64_t rows, int64_t cols, int square,
                              int pattern_b, __nv_bfloat16* __restrict__ dst, int64_t kp)
{
    const int64_t per_row = kp / 8;
    const int64_t total = rows * per_row;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / per_row, k0 = (i - r * per_row) * 8;
        const float* sp = src + r * ld_src + k0;
        float x[8];
        if (k0 + 8 <= cols && (reinterpret_cast<uintptr_t>(sp) & 15) == 0) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(sp));
            const float4 b = __ldg(reinterpret_cast<const float4*>(sp) + 1);
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = (k0 + e < cols) ? sp[e] : 0.f;
        }
        if (square) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] *= x[e];
        }
        uint4 hi, lo;
        split8(x, hi, lo);
        uint4* d = reinterpret_cast<uint4*>(dst + r * 3 * kp + k0);
        d[0] = hi;
        d[per_row] = pattern_b ? lo : hi;
        d[2 * per_row] = pattern_b ? hi : lo;
    }
}

// One CTA per row x of W^T: accumulate the row's entries (its segments of every
// source) in shared memory, then write [hi | lo | hi] of the row.  Replaces a
// zero-fill, global atomics and a separate split pass.
__global__ void __launch_bounds__(256)
densify_split_kernel(S1Sources srcs, const float* __restrict__ v, __nv_bfloat16* __restrict__ Bp, int64_t kp)
{
    extern __shared__ float wrow[];
    const int64_t x = blockIdx.x;
    for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) wrow[k] = 0.f;
    __syncthreads();
#pragma unroll
    for (int si = 0; si < kMaxSources; ++si) {
        if (si >= srcs.count) break;
        const S1Source sr = srcs.src[si];
        const int32_t j0 = sr.seg[x], j1 = sr.seg[x + 1];
        const float c = (float)sr.coef;
        for (int32_t j = j0 + (int32_t)threadIdx.x; j < j1; j += (int32_t)blockDim.x)
            atomicAdd(&wrow[sr.bcol[j]], c * v[sr.perm[j]]);
    }
    __syncthreads();
    const int64_t per_row = kp / 8;
    uint4* d = reinterpret_cast<uint4*>(Bp + x * 3 * kp);
    for (int64_t q = threadIdx.x; q < per_row; q += blockDim.x) {
        float xs[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xs[e] = wrow[q * 8 + e];
        uint4 hi, lo;
        split8(xs, hi, lo);
        d[q] = hi;
        d[per_row + q] = lo;
        d[2 * per_row + q] = hi;
    }
}

// fallback for rows too wide for shared memory: W^T[x, t] += coef * v[perm_j]
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

constexpr int64_t kRowSmemMax = 160 * 1024;   // widest W^T row (bytes) densified in shared memory

}  // namespace

size_t dense_stage1_workspace(int64_t Y, int64_t K, int64_t X)
{
    const int64_t kp = (K + 63) / 64 * 64;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t wt = 4 * (size_t)kp <= (size_t)kRowSmemMax ? 0 : al(4 * (size_t)X * kp);
    return al(2 * (size_t)Y * 3 * kp) + wt + al(2 * (size_t)X * 3 * kp);
}

gvt_status dense_stage1(const float* B, int64_t ldb, int64_t Y, int64_t K, int square, const S1Sources& srcs,
                        const int32_t* const keys[kMaxSources], int64_t n, const float* v, int64_t X, float* S,
                        int64_t lds, void* ws, int reuse_a, int* err, cudaStream_t s)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    const int64_t kp = (K + 63) / 64 * 64;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const bool rows_in_smem = 4 * (size_t)kp <= (size_t)kRowSmemMax;
    char* p = static_cast<char*>(ws);
    __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(p);
    p += al(2 * (size_t)Y * 3 * kp);
    float* Wt = reinterpret_cast<float*>(p);
    if (!rows_in_smem) p += al(4 * (size_t)X * kp);
    __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(p);

    if (!reuse_a) {
        split3_kernel<<<g1(Y * kp / 8), 256, 0, s>>>(B, ldb, Y, K, square, 0, Ap, kp);
        GVT_LAUNCH_CHECK("split B");
    }
    if (rows_in_smem) {
        const size_t smem = 4 * (size_t)kp;
        if (smem > 48 * 1024) {
            static bool attr = false;
            if (!attr) {
                GVT_CUDA(cudaFuncSetAttribute(densify_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kRowSmemMax));
                attr = true;
            }
        }
        densify_split_kernel<<<(unsigned)X, 256, smem, s>>>(srcs, v, Bp, kp);
        GVT_LAUNCH_CHECK("densify and split W");
    } else {
        zero_f32_kernel<<<g1(X * kp), 256, 0, s>>>(Wt, X * kp);
        GVT_LAUNCH_CHECK("zero W");
        if (n > 0) {
            densify_kernel<<<g1(n), 256, 0, s>>>(srcs, keys[0], keys[1], keys[2], keys[3], n, v, Wt, kp);
            GVT_LAUNCH_CHECK("densify");
        }
        split3_kernel<<<g1(X * kp / 8), 256, 0, s>>>(Wt, kp, X, kp, 0, 1, Bp, kp);
        GVT_LAUNCH_CHECK("split W");
    }
    return tc_gemm_bf16(Ap, 3 * kp, Bp, 3 * kp, S, lds, Y, X, 3 * kp, err, s);
}

}  // namespace gvt
