// Operands of the dense (tensor-core) stages.
//
// A dense x dense Kronecker term can run both GVT stages as GEMMs
// (Theorem 1's two products with W densified):
//   stage 1   S[Y x X]  = B[Y x K] W[K x X],        W^T row x holds coef * v_j at column bcol_j
//   stage 2   C[mb x Y] = A[mb x X] S[Y x X]^T,     u_i += C[arow_i, srow_i]
// Each FP32 operand is split into a 3K'-wide 16-bit operand (K' = K rounded
// up to 64) so that one GEMM of the splits gives hi*hi + hi*lo + lo*hi:
//   left  operand  [hi | hi | lo]      right operand  [hi | lo | hi]
// or, in the single-pass form, kept as its K'-wide hi part alone (one GEMM of
// the hi parts: FP16 products accurate to about 2^-11 relative, for inner
// operators whose error an FP64 outer refinement removes).
// Two split formats:
//   BF16 : hi = bf16(x), lo = bf16(x - hi); no scaling.  Products are
//          accurate to about 3 * 2^-17 relative.
//   FP16 : each row is first scaled by a power of two s_r that puts its
//          largest magnitude in [2^13, 2^14); hi = fp16(s x), lo = fp16(s x - hi).
//          hi and lo carry 22 significant bits, the dropped lo*lo term is
//          below 2^-22 relative, so products are accurate to about 2^-21 --
//          FP32-class.  The GEMM epilogue multiplies by 1/s_row and 1/s_col
//          (exact powers of two).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gvt_internal.h"
#include "split16.cuh"

namespace gvt {
namespace {

using split16::row_scale;
using split16::split8_bf16;
using split16::split8_f16;
using split16::store3;

constexpr int kSplitThreads = 256;
constexpr int64_t kRowSmemMax = 160 * 1024;   // widest W^T row (bytes) densified in shared memory
// Row passes that gather through a column permutation stage the row in shared memory first: a
// gather straight from global memory reads a 32-byte sector per 4-byte value.  1024 threads a
// block and rows of up to 100 KB keep two blocks (64 warps) on an SM.
constexpr int kPermThreads = 1024;
constexpr int64_t kPermRowMax = 100 * 1024;

// largest of v over the block (red: one slot per warp)
__device__ __forceinline__ float block_max(float v, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    float m = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
    return m;
}

__device__ __forceinline__ void load8(const float* sp, int64_t k0, int64_t cols, int square, float (&x)[8])
{
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
}

// One CTA per row: dst row r = the `parts`-part split of src row rowperm[r] (r without rowperm),
// its entry k taken from column colperm[k] (k without colperm); zero beyond cols.
template <bool F16>
__global__ void __launch_bounds__(kSplitThreads)
split_rows_kernel(const float* __restrict__ src, int64_t ld, int64_t cols, int square, int pattern_b,
                  uint4* __restrict__ dst, float* __restrict__ inv_scale, int64_t kp, int parts,
                  const int32_t* __restrict__ rowperm, const int32_t* __restrict__ colperm)
{
    __shared__ float red[kSplitThreads / 32];
    const int64_t r = blockIdx.x;
    const float* row = src + (rowperm ? (int64_t)rowperm[r] : r) * ld;
    const int64_t per_row = kp / 8;
    float s = 1.f;
    if (F16) {
        float m = 0.f;
        for (int64_t q = threadIdx.x; q * 8 < cols; q += blockDim.x) {
            float x[8];
            load8(row + q * 8, q * 8, cols, square, x);
#pragma unroll
            for (int e = 0; e < 8; ++e) m = fmaxf(m, fabsf(x[e]));
        }
        float inv;
        row_scale(block_max(m, red), s, inv);
        if (threadIdx.x == 0) inv_scale[r] = inv;
    }
    // (a column permutation leaves the row's largest magnitude, hence its scale, unchanged)
    uint4* d = dst + r * parts * per_row;
    for (int64_t q = threadIdx.x; q < per_row; q += blockDim.x) {
        float x[8];
        if (colperm) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t k = q * 8 + e;
                const float a = k < cols ? __ldg(row + colperm[k]) : 0.f;
                x[e] = square ? a * a : a;
            }
        } else {
            load8(row + q * 8, q * 8, cols, square, x);
        }
        uint4 hi, lo;
        if (F16) split8_f16(x, s, hi, lo);
        else split8_bf16(x, hi, lo);
        store3(d, q, per_row, pattern_b, parts, hi, lo);
    }
}

// Dense tiles of W^T in relabelled coordinates, one CTA per relabelled row x': the entries of
// original column x = xperm[x'] (its segment of the source ordered by x) whose relabelled row
// k' = krank[bcol] falls in a dense tile (dense[(x' / bn) * nk + k' / 64]) are accumulated in
// shared memory at k', then the row is split like densify_split_kernel's.
template <bool F16>
__global__ void __launch_bounds__(kSplitThreads)
densify_tiles_kernel(S1Source src, const int32_t* __restrict__ xperm, const int32_t* __restrict__ krank,
                     const uint8_t* __restrict__ dense, int bn, int64_t nk, const float* __restrict__ v,
                     uint4* __restrict__ dst, float* __restrict__ inv_scale, int64_t kp, int parts)
{
    extern __shared__ float wrow[];
    __shared__ float red[kSplitThreads / 32];
    const int64_t xr = blockIdx.x;
    for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) wrow[k] = 0.f;
    __syncthreads();
    const int32_t x = xperm[xr];
    const uint8_t* drow = dense + (xr / bn) * nk;
    const float c = (float)src.coef;
    for (int32_t j = src.seg[x] + (int32_t)threadIdx.x; j < src.seg[x + 1]; j += (int32_t)blockDim.x) {
        const int32_t k = krank[src.bcol[j]];
        if (drow[k >> 6]) atomicAdd(&wrow[k], c * v[src.perm[j]]);
    }
    __syncthreads();
    const int64_t per_row = kp / 8;
    float s = 1.f;
    if (F16) {
        float m = 0.f;
        for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) m = fmaxf(m, fabsf(wrow[k]));
        float inv;
        row_scale(block_max(m, red), s, inv);
        if (threadIdx.x == 0) inv_scale[xr] = inv;
    }
    uint4* d = dst + xr * parts * per_row;
    for (int64_t q = threadIdx.x; q < per_row; q += blockDim.x) {
        float xs[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xs[e] = wrow[q * 8 + e];
        uint4 hi, lo;
        if (F16) split8_f16(xs, s, hi, lo);
        else split8_bf16(xs, hi, lo);
        store3(d, q, per_row, 1, parts, hi, lo);
    }
}

// S[y, x] += Sd[y, xrank[x]] (the dense tiles' part, computed in relabelled columns)
__global__ void merge_cols_kernel(float* __restrict__ S, int64_t lds, const float* __restrict__ Sd, int64_t ldsd,
                                  const int32_t* __restrict__ xrank, int64_t Y, int64_t X)
{
    for (int64_t y = blockIdx.x; y < Y; y += gridDim.x) {
        float* srow = S + y * lds;
        const float* drow = Sd + y * ldsd;
        for (int64_t x = threadIdx.x; x < X; x += blockDim.x) srow[x] += __ldg(drow + xrank[x]);
    }
}

// The same with the row of Sd staged in shared memory (4 X bytes), one row per pass of a block.
__global__ void __launch_bounds__(kPermThreads)
merge_cols_smem_kernel(float* __restrict__ S, int64_t lds, const float* __restrict__ Sd, int64_t ldsd,
                       const int32_t* __restrict__ xrank, int64_t Y, int64_t X)
{
    extern __shared__ float drow_s[];
    const bool vec = (lds % 4 == 0) && (ldsd % 4 == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(Sd) & 15) == 0) && ((reinterpret_cast<uintptr_t>(xrank) & 15) == 0);
    const int64_t xv = vec ? X / 4 * 4 : 0;
    for (int64_t y = blockIdx.x; y < Y; y += gridDim.x) {
        const float* drow = Sd + y * ldsd;
        float* srow = S + y * lds;
        __syncthreads();   // the previous row's gathers are done
        for (int64_t x = (int64_t)threadIdx.x * 4; x < xv; x += 4 * blockDim.x)
            *reinterpret_cast<float4*>(drow_s + x) = __ldg(reinterpret_cast<const float4*>(drow + x));
        for (int64_t x = xv + threadIdx.x; x < X; x += blockDim.x) drow_s[x] = __ldg(drow + x);
        __syncthreads();
        for (int64_t x = (int64_t)threadIdx.x * 4; x < xv; x += 4 * blockDim.x) {
            const int4 r = __ldg(reinterpret_cast<const int4*>(xrank + x));
            float4 v = *reinterpret_cast<const float4*>(srow + x);
            v.x += drow_s[r.x];
            v.y += drow_s[r.y];
            v.z += drow_s[r.z];
            v.w += drow_s[r.w];
            *reinterpret_cast<float4*>(srow + x) = v;
        }
        for (int64_t x = xv + threadIdx.x; x < X; x += blockDim.x) srow[x] += drow_s[xrank[x]];
    }
}

// The merge fused with the split of S that follows it: block r takes row y = rowperm[r] (r without
// rowperm), stages Sd's row y in shared memory, forms S[y, x] + Sd[y, xrank[x]], writes it back
// to S (for the consumers of S in FP32) and splits it as dst row r.  A thread keeps its values of
// the merged row in registers between the two passes: groups of 8, at most kMergeGroups a thread
// (kp <= 8 * kMergeGroups * kPermThreads).
constexpr int kMergeGroups = 4;
template <bool F16>
__global__ void __launch_bounds__(kPermThreads)
merge_split_rows_kernel(float* __restrict__ S, int64_t lds, const float* __restrict__ Sd, int64_t ldsd,
                        const int32_t* __restrict__ xrank, int64_t X, int pattern_b, uint4* __restrict__ dst,
                        float* __restrict__ inv_scale, int64_t kp, int parts, const int32_t* __restrict__ rowperm)
{
    extern __shared__ float drow_s[];
    __shared__ float red[kPermThreads / 32];
    const int64_t r = blockIdx.x;
    const int64_t y = rowperm ? (int64_t)rowperm[r] : r;
    float* srow = S + y * lds;
    const float* drow = Sd + y * ldsd;
    const bool vec = (lds % 4 == 0) && (ldsd % 4 == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(Sd) & 15) == 0);
    const int64_t xv = vec ? X / 4 * 4 : 0;
    for (int64_t x = (int64_t)threadIdx.x * 4; x < xv; x += 4 * blockDim.x)
        *reinterpret_cast<float4*>(drow_s + x) = __ldg(reinterpret_cast<const float4*>(drow + x));
    for (int64_t x = xv + threadIdx.x; x < X; x += blockDim.x) drow_s[x] = __ldg(drow + x);
    __syncthreads();
    const int64_t per_row = kp / 8;
    float val[kMergeGroups][8];
    float m = 0.f;
#pragma unroll
    for (int g = 0; g < kMergeGroups; ++g) {
        const int64_t q = threadIdx.x + (int64_t)g * blockDim.x;
        const int64_t x0 = q * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) val[g][e] = 0.f;
        if (q >= per_row || x0 >= X) continue;
        if (vec && x0 + 8 <= X) {
            float4 a = *reinterpret_cast<const float4*>(srow + x0);
            float4 b = *reinterpret_cast<const float4*>(srow + x0 + 4);
            a.x += drow_s[xrank[x0]];
            a.y += drow_s[xrank[x0 + 1]];
            a.z += drow_s[xrank[x0 + 2]];
            a.w += drow_s[xrank[x0 + 3]];
            b.x += drow_s[xrank[x0 + 4]];
            b.y += drow_s[xrank[x0 + 5]];
            b.z += drow_s[xrank[x0 + 6]];
            b.w += drow_s[xrank[x0 + 7]];
            *reinterpret_cast<float4*>(srow + x0) = a;
            *reinterpret_cast<float4*>(srow + x0 + 4) = b;
            val[g][0] = a.x; val[g][1] = a.y; val[g][2] = a.z; val[g][3] = a.w;
            val[g][4] = b.x; val[g][5] = b.y; val[g][6] = b.z; val[g][7] = b.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (x0 + e < X) {
                    const float v = srow[x0 + e] + drow_s[xrank[x0 + e]];
                    srow[x0 + e] = v;
                    val[g][e] = v;
                }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) m = fmaxf(m, fabsf(val[g][e]));
    }
    float sc = 1.f;
    if (F16) {
        float inv;
        row_scale(block_max(m, red), sc, inv);
        if (threadIdx.x == 0) inv_scale[r] = inv;
    }
    uint4* d = dst + r * parts * per_row;
#pragma unroll
    for (int g = 0; g < kMergeGroups; ++g) {
        const int64_t q = threadIdx.x + (int64_t)g * blockDim.x;
        if (q >= per_row) continue;
        uint4 hi, lo;
        if (F16) split8_f16(val[g], sc, hi, lo);
        else split8_bf16(val[g], hi, lo);
        store3(d, q, per_row, pattern_b, parts, hi, lo);
    }
}

// split_rows_kernel for a column permutation: the source row (cols values) is staged in shared
// memory, its largest magnitude taken on the way, then split through colperm from there.
template <bool F16>
__global__ void __launch_bounds__(kPermThreads)
split_rows_perm_kernel(const float* __restrict__ src, int64_t ld, int64_t cols, int square, int pattern_b,
                       uint4* __restrict__ dst, float* __restrict__ inv_scale, int64_t kp, int parts,
                       const int32_t* __restrict__ rowperm, const int32_t* __restrict__ colperm)
{
    extern __shared__ float row_s[];
    __shared__ float red[kPermThreads / 32];
    const int64_t r = blockIdx.x;
    const float* row = src + (rowperm ? (int64_t)rowperm[r] : r) * ld;
    float m = 0.f;
    const bool vec = ((reinterpret_cast<uintptr_t>(row) & 15) == 0);
    const int64_t cv = vec ? cols / 4 * 4 : 0;
    for (int64_t k = (int64_t)threadIdx.x * 4; k < cv; k += 4 * blockDim.x) {
        float4 a = __ldg(reinterpret_cast<const float4*>(row + k));
        if (square) {
            a.x *= a.x;
            a.y *= a.y;
            a.z *= a.z;
            a.w *= a.w;
        }
        *reinterpret_cast<float4*>(row_s + k) = a;
        m = fmaxf(m, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
    }
    for (int64_t k = cv + threadIdx.x; k < cols; k += blockDim.x) {
        float a = __ldg(row + k);
        if (square) a *= a;
        row_s[k] = a;
        m = fmaxf(m, fabsf(a));
    }
    float s = 1.f;
    if (F16) {
        float inv;
        row_scale(block_max(m, red), s, inv);   // (its barriers also publish row_s)
        if (threadIdx.x == 0) inv_scale[r] = inv;
    } else {
        __syncthreads();
    }
    const int64_t per_row = kp / 8;
    uint4* d = dst + r * parts * per_row;
    for (int64_t q = threadIdx.x; q < per_row; q += blockDim.x) {
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t k = q * 8 + e;
            x[e] = k < cols ? row_s[colperm[k]] : 0.f;
        }
        uint4 hi, lo;
        if (F16) split8_f16(x, s, hi, lo);
        else split8_bf16(x, hi, lo);
        store3(d, q, per_row, pattern_b, parts, hi, lo);
    }
}

// One CTA per row x of W^T: accumulate the row's entries (its segment of every
// source) in shared memory, then write the [hi | lo | hi] split of the row (its hi part
// alone when parts == 1).
template <bool F16>
__global__ void __launch_bounds__(kSplitThreads)
densify_split_kernel(S1Sources srcs, const float* __restrict__ v, uint4* __restrict__ dst,
                     float* __restrict__ inv_scale, int64_t kp, int parts)
{
    extern __shared__ float wrow[];
    __shared__ float red[kSplitThreads / 32];
    const int64_t x = blockIdx.x;
    for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) wrow[k] = 0.f;
    __syncthreads();
    // sources one after another, so that a cell written by several sources sums in a fixed
    // order; within a source the cells of distinct pairs are distinct, except for a source whose
    // column is the key itself, whose whole segment sums into cell (x, x) by a fixed-order
    // block reduction (results are reproducible bit for bit unless pairs repeat)
#pragma unroll
    for (int si = 0; si < kMaxSources; ++si) {
        if (si >= srcs.count) break;
        const S1Source sr = srcs.src[si];
        const int32_t j0 = sr.seg[x], j1 = sr.seg[x + 1];
        const float c = (float)sr.coef;
        if (sr.same) {
            float acc = 0.f;
            for (int32_t j = j0 + (int32_t)threadIdx.x; j < j1; j += (int32_t)blockDim.x) acc += c * v[sr.perm[j]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int w = 0; w < kSplitThreads / 32; ++w) t += red[w];
                wrow[x] += t;
            }
        } else {
            for (int32_t j = j0 + (int32_t)threadIdx.x; j < j1; j += (int32_t)blockDim.x)
                atomicAdd(&wrow[sr.bcol[j]], c * v[sr.perm[j]]);
        }
        __syncthreads();
    }
    const int64_t per_row = kp / 8;
    float s = 1.f;
    if (F16) {
        float m = 0.f;
        for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) m = fmaxf(m, fabsf(wrow[k]));
        float inv;
        row_scale(block_max(m, red), s, inv);
        if (threadIdx.x == 0) inv_scale[x] = inv;
    }
    uint4* d = dst + x * parts * per_row;
    for (int64_t q = threadIdx.x; q < per_row; q += blockDim.x) {
        float xs[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xs[e] = wrow[q * 8 + e];
        uint4 hi, lo;
        if (F16) split8_f16(xs, s, hi, lo);
        else split8_bf16(xs, hi, lo);
        store3(d, q, per_row, 1, parts, hi, lo);
    }
}

// rows too wide for shared memory: W^T[x, t] += coef * v[perm_j] in global memory
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

// u[perm_i] += C[arow_i, srow_i]
__global__ void gather_c_kernel(const float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ arow,
                                const int32_t* __restrict__ srow, const int32_t* __restrict__ perm, int64_t n,
                                float* __restrict__ u)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[perm[i]] += C[(int64_t)arow[i] * ldc + srow[i]];
}

unsigned g1(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

int64_t dense_kp(int64_t K) { return (K + 63) / 64 * 64; }

size_t dense_operand_bytes(int64_t rows, int64_t K, int parts)
{
    return al256(2 * (size_t)rows * parts * (size_t)dense_kp(K)) + al256(4 * (size_t)std::max<int64_t>(rows, 1));
}

DenseOperand dense_operand_at(void* base, int64_t rows, int64_t K, int parts)
{
    DenseOperand o;
    o.data = base;
    o.inv_scale = reinterpret_cast<float*>(static_cast<char*>(base) +
                                           al256(2 * (size_t)rows * parts * (size_t)dense_kp(K)));
    o.rows = rows;
    o.kp = dense_kp(K);
    o.parts = parts;
    return o;
}

size_t dense_w_scratch_bytes(int64_t X, int64_t K)
{
    return 4 * (size_t)dense_kp(K) <= (size_t)kRowSmemMax ? 0 : al256(4 * (size_t)X * (size_t)dense_kp(K));
}

gvt_status dense_split_rows(const float* src, int64_t ld, int64_t rows, int64_t cols, int square, bool f16,
                            int pattern_b, const DenseOperand& dst, cudaStream_t s, const int32_t* rowperm,
                            const int32_t* colperm)
{
    if (rows <= 0) return GVT_OK;
    if (rows > INT32_MAX) {
        set_error("dense split: too many rows");
        return GVT_ERR_UNSUPPORTED;
    }
    uint4* d = static_cast<uint4*>(dst.data);
    const int64_t perm_smem = 4 * ((cols + 3) / 4 * 4);
    if (colperm && perm_smem <= kPermRowMax) {
        const void* fn = f16 ? reinterpret_cast<const void*>(split_rows_perm_kernel<true>)
                             : reinterpret_cast<const void*>(split_rows_perm_kernel<false>);
        if (perm_smem > 48 * 1024) GVT_CHECK(ensure_smem_attr(fn, (int)perm_smem));
        if (f16)
            split_rows_perm_kernel<true><<<(unsigned)rows, kPermThreads, (size_t)perm_smem, s>>>(
                src, ld, cols, square, pattern_b, d, dst.inv_scale, dst.kp, dst.parts, rowperm, colperm);
        else
            split_rows_perm_kernel<false><<<(unsigned)rows, kPermThreads, (size_t)perm_smem, s>>>(
                src, ld, cols, square, pattern_b, d, dst.inv_scale, dst.kp, dst.parts, rowperm, colperm);
    } else if (f16)
        split_rows_kernel<true><<<(unsigned)rows, kSplitThreads, 0, s>>>(src, ld, cols, square, pattern_b, d,
                                                                         dst.inv_scale, dst.kp, dst.parts, rowperm,
                                                                         colperm);
    else
        split_rows_kernel<false><<<(unsigned)rows, kSplitThreads, 0, s>>>(src, ld, cols, square, pattern_b, d,
                                                                          dst.inv_scale, dst.kp, dst.parts, rowperm,
                                                                          colperm);
    GVT_LAUNCH_CHECK("dense split rows");
    return GVT_OK;
}

gvt_status dense_split_w(const S1Sources& srcs, const int32_t* const keys[kMaxSources], int64_t n, const float* v,
                         int64_t X, bool f16, const DenseOperand& dst, float* wide_scratch, cudaStream_t s)
{
    if (X <= 0) return GVT_OK;
    const int64_t kp = dst.kp;
    uint4* d = static_cast<uint4*>(dst.data);
    if (4 * kp <= kRowSmemMax) {
        const size_t smem = 4 * (size_t)kp;
        if (smem > 48 * 1024) {
            if (f16) GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(densify_split_kernel<true>), (int)smem));
            else GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(densify_split_kernel<false>), (int)smem));
        }
        if (f16)
            densify_split_kernel<true><<<(unsigned)X, kSplitThreads, smem, s>>>(srcs, v, d, dst.inv_scale, kp,
                                                                               dst.parts);
        else
            densify_split_kernel<false><<<(unsigned)X, kSplitThreads, smem, s>>>(srcs, v, d, dst.inv_scale, kp,
                                                                                dst.parts);
        GVT_LAUNCH_CHECK("densify and split W");
        return GVT_OK;
    }
    zero_f32_kernel<<<g1(X * kp), 256, 0, s>>>(wide_scratch, X * kp);
    GVT_LAUNCH_CHECK("zero W");
    if (n > 0) {
        densify_kernel<<<g1(n), 256, 0, s>>>(srcs, keys[0], keys[1], keys[2], keys[3], n, v, wide_scratch, kp);
        GVT_LAUNCH_CHECK("densify");
    }
    return dense_split_rows(wide_scratch, kp, X, kp, 0, f16, 1, dst, s);
}

gvt_status dense_gemm(const DenseOperand& a, const DenseOperand& b, bool f16, float* C, int64_t ldc, int* err,
                      cudaStream_t s, int pair_mode, long long stall_cycles, const TcSparse* sparse)
{
    if (a.kp != b.kp || a.parts != b.parts) {
        set_error("dense stage: operand widths differ");
        return GVT_ERR_INVALID_ARG;
    }
    const int64_t kw = (int64_t)a.parts * a.kp;
    return tc_gemm(a.data, kw, b.data, kw, C, ldc, a.rows, b.rows, kw, f16,
                   f16 ? a.inv_scale : nullptr, f16 ? b.inv_scale : nullptr, err, s, pair_mode, stall_cycles, sparse);
}

gvt_status dense_densify_tiles(const S1Source& src, const int32_t* xperm, const int32_t* krank, const uint8_t* dense,
                               int bn, int64_t nk, const float* v, int64_t X, bool f16, const DenseOperand& dst,
                               cudaStream_t s)
{
    if (X <= 0) return GVT_OK;
    const int64_t kp = dst.kp;
    if (4 * kp > kRowSmemMax) {
        set_error("dense tiles: W rows too wide for shared memory");
        return GVT_ERR_UNSUPPORTED;
    }
    const size_t smem = 4 * (size_t)kp;
    if (smem > 48 * 1024) {
        if (f16) GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(densify_tiles_kernel<true>), (int)smem));
        else GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(densify_tiles_kernel<false>), (int)smem));
    }
    uint4* d = static_cast<uint4*>(dst.data);
    if (f16)
        densify_tiles_kernel<true><<<(unsigned)X, kSplitThreads, smem, s>>>(src, xperm, krank, dense, bn, nk, v, d,
                                                                            dst.inv_scale, kp, dst.parts);
    else
        densify_tiles_kernel<false><<<(unsigned)X, kSplitThreads, smem, s>>>(src, xperm, krank, dense, bn, nk, v, d,
                                                                             dst.inv_scale, kp, dst.parts);
    GVT_LAUNCH_CHECK("densify dense tiles of W");
    return GVT_OK;
}

gvt_status dense_merge_cols(float* S, int64_t lds, const float* Sd, int64_t ldsd, const int32_t* xrank, int64_t Y,
                            int64_t X, cudaStream_t s)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    const int64_t smem = 4 * ((X + 3) / 4 * 4);
    if (smem <= kPermRowMax) {
        if (smem > 48 * 1024)
            GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(merge_cols_smem_kernel), (int)smem));
        merge_cols_smem_kernel<<<(unsigned)std::min<int64_t>(Y, 152 * 2), kPermThreads, (size_t)smem, s>>>(
            S, lds, Sd, ldsd, xrank, Y, X);
    } else {
        merge_cols_kernel<<<(unsigned)std::min<int64_t>(Y, 152 * 8), 256, 0, s>>>(S, lds, Sd, ldsd, xrank, Y, X);
    }
    GVT_LAUNCH_CHECK("merge dense part of S");
    return GVT_OK;
}

bool dense_merge_split_fits(int64_t X)
{
    return 4 * ((X + 3) / 4 * 4) <= kPermRowMax && dense_kp(X) <= 8 * kMergeGroups * kPermThreads;
}

gvt_status dense_merge_split(float* S, int64_t lds, const float* Sd, int64_t ldsd, const int32_t* xrank, int64_t Y,
                             int64_t X, bool f16, int pattern_b, const DenseOperand& dst, cudaStream_t s,
                             const int32_t* rowperm)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    if (!dense_merge_split_fits(X) || dst.kp != dense_kp(X) || Y > INT32_MAX) {
        set_error("merge and split of S: row too long");
        return GVT_ERR_UNSUPPORTED;
    }
    const int64_t smem = 4 * ((X + 3) / 4 * 4);
    const void* fn = f16 ? reinterpret_cast<const void*>(merge_split_rows_kernel<true>)
                         : reinterpret_cast<const void*>(merge_split_rows_kernel<false>);
    if (smem > 48 * 1024) GVT_CHECK(ensure_smem_attr(fn, (int)smem));
    uint4* d = static_cast<uint4*>(dst.data);
    if (f16)
        merge_split_rows_kernel<true><<<(unsigned)Y, kPermThreads, (size_t)smem, s>>>(
            S, lds, Sd, ldsd, xrank, X, pattern_b, d, dst.inv_scale, dst.kp, dst.parts, rowperm);
    else
        merge_split_rows_kernel<false><<<(unsigned)Y, kPermThreads, (size_t)smem, s>>>(
            S, lds, Sd, ldsd, xrank, X, pattern_b, d, dst.inv_scale, dst.kp, dst.parts, rowperm);
    GVT_LAUNCH_CHECK("merge and split of S");
    return GVT_OK;
}

gvt_status dense_gather(const float* C, int64_t ldc, const S2Outputs& outs, float* u, cudaStream_t s)
{
    if (outs.n <= 0) return GVT_OK;
    gather_c_kernel<<<g1(outs.n), 256, 0, s>>>(C, ldc, outs.arow, outs.srow, outs.perm, outs.n, u);
    GVT_LAUNCH_CHECK("dense stage 2 gather");
    return GVT_OK;
}

}  // namespace gvt
