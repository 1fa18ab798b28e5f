// The two stages of the generalized vec trick (Theorem 1) and the small
// kernels around them.
//
// Stage 1 (sparse, SIMT): S = B W, W holding v_j at (bcol_j, x_j), computed
// column tile by column tile over input pairs sorted by x (segments).  A block
// stages the entries of its columns in shared memory as (row offset, weight)
// records; every thread owns a few output rows of each of those columns in
// registers and streams its part of the needed row of B^T with 16-byte loads.
//
// Stage 2 (sampled gather-dot): u_i = <A[arow_i, :], S[srow_i, :]>, one warp
// per output pair, outputs sorted by arow so that consecutive warps share the
// A row in L1; 16-byte vector loads of both rows.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "gvt_internal.h"

namespace gvt {
namespace {

template <class T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int N = 4;
    __device__ static void split(const float4& q, float* o) { o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w; }
    __device__ static float4 make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static void split(const double2& q, double* o) { o[0] = q.x; o[1] = q.y; }
    __device__ static double2 make(const double* o) { return make_double2(o[0], o[1]); }
};

// 16-byte loads of a stored type TB widened to the arithmetic type T (FP16 storage: the
// single-pass operands of the dense stages, rows scaled by powers of two, read in FP32)
template <class TB, class T> struct Ld;
template <> struct Ld<float, float> : Vec<float> {};
template <> struct Ld<double, double> : Vec<double> {};
template <> struct Ld<__half, float> {
    using type = uint4;
    static constexpr int N = 8;
    __device__ static void split(const uint4& q, float* o)
    {
        const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(h[e]);
            o[2 * e] = f.x;
            o[2 * e + 1] = f.y;
        }
    }
};
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld1(const double* p) { return __ldg(p); }

__host__ __device__ inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

unsigned grid1d(int64_t n, int threads, int64_t cap = 152 * 32)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ------------------------------------------------------------------ stage 1
// Tile: blockDim = NT threads, each owning RPT rows y (RPT/VEC 16-byte loads per
// entry), and kS1Cols consecutive columns x of S.  A warp's rows are 32 * RPT
// consecutive ones; its q-th load covers VEC rows per lane, lanes side by side,
// so that one load instruction of the warp reads 512 contiguous bytes (with each
// thread's RPT rows consecutive, a warp instruction spread over 1 KB in half
// sectors and the L1 data pipe bound the kernel).  The
// entries of the tile's columns are contiguous in every sorted source; they
// are staged in shared memory as (row offset of B^T, weight) records, which
// every warp reads with one broadcast load per entry.
// Grid order: column tiles fastest (blockIdx.x), row blocks slowest, so that
// all the CTAs of one pass read the same NT * RPT rows of B^T: that slice
// (K x 1024 FP32 values, 80 MB at K = 20000) stays in L2 while every entry
// of the pass reads its part, instead of each entry streaming its whole
// B^T row from HBM.
constexpr int kS1Cols = 4;
constexpr int kS1Chunk = 512;     // staged entries per round

template <class T>
struct S1Entry {
    int64_t off;   // bcol * ldb
    T w;           // coef * v[perm]
};

template <class T, int MODE, int NT, int RPT>
__global__ void __launch_bounds__(NT)
stage1_sparse_kernel(const T* __restrict__ Bt, int64_t ldb, S1Sources srcs,
                    const T* __restrict__ v, T* __restrict__ S, int64_t lds, int64_t Y, int64_t X)
{
    constexpr int VEC = Vec<T>::N;
    constexpr int NV = RPT / VEC;
    constexpr int U = 4;   // entries in flight per thread
    using VT = typename Vec<T>::type;
    __shared__ S1Entry<T> ent[kS1Chunk];
    __shared__ int32_t sseg[kMaxSources][kS1Cols + 1];

    // rows of this thread: acc index k <-> row y0 + (k / VEC) * 32 * VEC + k % VEC
    constexpr int QS = 32 * VEC;   // distance between a thread's successive loads, in rows
    const int64_t y0 = (int64_t)blockIdx.y * (NT * RPT) + (int64_t)(threadIdx.x >> 5) * (32 * RPT) +
                       (int64_t)(threadIdx.x & 31) * VEC;
    const int64_t x0 = (int64_t)blockIdx.x * kS1Cols;
    const bool vec_rows = (y0 + (NV - 1) * QS + VEC <= Y) && (ldb % VEC == 0) && aligned16(Bt);
    const T* __restrict__ by = Bt + y0;

    if (threadIdx.x < kMaxSources * (kS1Cols + 1)) {
        const int si = threadIdx.x / (kS1Cols + 1), c = threadIdx.x % (kS1Cols + 1);
        if (si < srcs.count) {
            const int64_t x = min(x0 + c, X);
#pragma unroll
            for (int k = 0; k < kMaxSources; ++k)
                if (k == si) sseg[si][c] = srcs.src[k].seg[x];
        }
    }

    T acc[RPT][kS1Cols];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int c = 0; c < kS1Cols; ++c) acc[k][c] = T(0);

#pragma unroll
    for (int si = 0; si < kMaxSources; ++si) {
        if (si >= srcs.count) break;
        const S1Source& sr = srcs.src[si];
        const T coef = (T)sr.coef;
        __syncthreads();
        const int32_t jb = sseg[si][0], je = sseg[si][kS1Cols];
        for (int32_t j0 = jb; j0 < je; j0 += kS1Chunk) {
            __syncthreads();   // the previous round's records are consumed
            for (int k = threadIdx.x; k < kS1Chunk && j0 + k < je; k += NT) {
                const int32_t j = j0 + k;
                ent[k].off = (int64_t)sr.bcol[j] * ldb;
                ent[k].w = coef * v[sr.perm[j]];
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < kS1Cols; ++c) {
                const int lo = max(sseg[si][c], j0) - j0;
                const int hi = min(sseg[si][c + 1], j0 + kS1Chunk) - j0;
                int k = lo;
                for (; k + U <= hi; k += U) {
                    T b[U][RPT];
                    T w[U];
#pragma unroll
                    for (int e = 0; e < U; ++e) {
                        const S1Entry<T> r = ent[k + e];
                        w[e] = r.w;
                        const T* row = by + r.off;
                        if (vec_rows) {
#pragma unroll
                            for (int q = 0; q < NV; ++q)
                                Vec<T>::split(__ldg(reinterpret_cast<const VT*>(row + q * QS)), &b[e][q * VEC]);
                        } else {
#pragma unroll
                            for (int q = 0; q < RPT; ++q) {
                                const int64_t dy = (q / VEC) * QS + q % VEC;
                                b[e][q] = (y0 + dy < Y) ? __ldg(row + dy) : T(0);
                            }
                        }
                    }
#pragma unroll
                    for (int e = 0; e < U; ++e)
#pragma unroll
                        for (int q = 0; q < RPT; ++q) {
                            const T bq = MODE == FM_SQUARE ? b[e][q] * b[e][q] : b[e][q];
                            acc[q][c] = fma(w[e], bq, acc[q][c]);
                        }
                }
                for (; k < hi; ++k) {
                    const S1Entry<T> r = ent[k];
                    const T* row = by + r.off;
                    T b[RPT];
                    if (vec_rows) {
#pragma unroll
                        for (int q = 0; q < NV; ++q)
                            Vec<T>::split(__ldg(reinterpret_cast<const VT*>(row + q * QS)), &b[q * VEC]);
                    } else {
#pragma unroll
                        for (int q = 0; q < RPT; ++q) {
                            const int64_t dy = (q / VEC) * QS + q % VEC;
                            b[q] = (y0 + dy < Y) ? __ldg(row + dy) : T(0);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        const T bq = MODE == FM_SQUARE ? b[q] * b[q] : b[q];
                        acc[q][c] = fma(r.w, bq, acc[q][c]);
                    }
                }
            }
        }
    }

    const bool vec_cols = (x0 + kS1Cols <= X) && (lds % VEC == 0) && aligned16(S) && (x0 % VEC == 0);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t y = y0 + (q / VEC) * QS + q % VEC;   // increasing in q
        if (y >= Y) break;
        T* srow = S + y * lds + x0;
        if (vec_cols) {
#pragma unroll
            for (int c = 0; c < kS1Cols; c += VEC)
                *reinterpret_cast<VT*>(srow + c) = Vec<T>::make(&acc[q][c]);
        } else {
#pragma unroll
            for (int c = 0; c < kS1Cols; ++c)
                if (x0 + c < X) srow[c] = acc[q][c];
        }
    }
}

template <class T>
__global__ void stage1_identity_kernel(S1Sources srcs, const T* __restrict__ v, T* __restrict__ S,
                                       int64_t lds, int64_t Y, int64_t X)
{
    // one warp per column x: its lanes take the segment's entries, sources one after the
    // other (a cell hit by several sources, or by a repeated pair, sums through atomics)
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < X; x += nw) {
#pragma unroll
        for (int si = 0; si < kMaxSources; ++si) {
            if (si >= srcs.count) break;
            const S1Source sr = srcs.src[si];
            const T coef = (T)sr.coef;
            for (int32_t j = sr.seg[x] + lane; j < sr.seg[x + 1]; j += 32) {
                const int32_t y = sr.bcol[j];
                if (y < Y) atomicAdd(&S[(int64_t)y * lds + x], coef * v[sr.perm[j]]);
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ stage 2
constexpr int kS2Threads = 256;
constexpr int kS2Group = 4;      // outputs per warp, processed together

// A warp takes kS2Group consecutive outputs (sorted by A row).  When they
// share their A row -- the common case, every A row serves ~n/m outputs --
// each chunk of the A row is loaded once for the whole group, so a group
// costs 1 + kS2Group row loads per chunk instead of 2 * kS2Group.
// The kernel waits on its row loads, so what counts is the loads in flight per SM: the chunk loop
// is unrolled by two (two chunks' loads issued together) at two blocks per SM (128 registers),
// which measured 5.72 ms for the kernel-filling remainder against 6.56 ms for one chunk at a time
// at three blocks per SM (80 registers, a few spilled), 6.22 ms unrolled at three blocks, and
// 7.67 ms for one chunk at two blocks.
// FP16 storage (TB = __half): A and S rows scaled by powers of two, whose inverses (ascale,
// sscale, one per row) multiply each finished dot.
template <class T, class TB, int MODE>
__global__ void __launch_bounds__(kS2Threads, 2)
stage2_gather_kernel(const TB* __restrict__ A, int64_t lda, const float* __restrict__ ascale,
                    const TB* __restrict__ S, int64_t lds, const float* __restrict__ sscale,
                    int64_t X, S2Outputs outs, T coef, T* __restrict__ u)
{
    constexpr int VEC = Ld<TB, T>::N;
    constexpr int G = kS2Group;
    using VT = typename Ld<TB, T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (kS2Threads / 32);
    const bool vec_ok = (lda % VEC == 0) && (lds % VEC == 0) && aligned16(A) && aligned16(S);
    const int64_t xv = vec_ok ? (X / VEC) * VEC : 0;
    for (int64_t grp = (int64_t)blockIdx.x * (kS2Threads / 32) + (threadIdx.x >> 5);
         grp * G < outs.n; grp += nwarps) {
        const int64_t i0 = grp * G;
        const int ng = (outs.n - i0 < G) ? (int)(outs.n - i0) : G;
        int32_t ar = 0, sr = 0, pm = 0;
        if (lane < ng) {
            ar = outs.arow[i0 + lane];
            sr = outs.srow[i0 + lane];
            pm = outs.perm[i0 + lane];
        }
        const int32_t ar0 = __shfl_sync(0xffffffffu, ar, 0);
        const bool same = __all_sync(0xffffffffu, lane >= ng || ar == ar0);
        const TB* arow[G];
        const TB* srow[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            // groups shorter than G repeat their last output; only real ones are written
            const int gg = g < ng ? g : ng - 1;
            arow[g] = A + (int64_t)__shfl_sync(0xffffffffu, ar, gg) * lda;
            srow[g] = S + (int64_t)__shfl_sync(0xffffffffu, sr, gg) * lds;
        }
        T acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = T(0);
        if (same) {
#pragma unroll 2
            for (int64_t x = (int64_t)lane * VEC; x < xv; x += 32 * VEC) {
                T a[VEC], sv[G][VEC];
                Ld<TB, T>::split(__ldg(reinterpret_cast<const VT*>(arow[0] + x)), a);
#pragma unroll
                for (int g = 0; g < G; ++g) Ld<TB, T>::split(__ldg(reinterpret_cast<const VT*>(srow[g] + x)), sv[g]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const T ak = MODE == FM_SQUARE ? a[k] * a[k] : a[k];
#pragma unroll
                    for (int g = 0; g < G; ++g) acc[g] = fma(ak, sv[g][k], acc[g]);
                }
            }
        } else {
#pragma unroll 2
            for (int64_t x = (int64_t)lane * VEC; x < xv; x += 32 * VEC) {
                T a[G][VEC], sv[G][VEC];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    Ld<TB, T>::split(__ldg(reinterpret_cast<const VT*>(arow[g] + x)), a[g]);
                    Ld<TB, T>::split(__ldg(reinterpret_cast<const VT*>(srow[g] + x)), sv[g]);
                }
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const T ak = MODE == FM_SQUARE ? a[g][k] * a[g][k] : a[g][k];
                        acc[g] = fma(ak, sv[g][k], acc[g]);
                    }
            }
        }
        for (int64_t x = xv + lane; x < X; x += 32) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const T av = (T)ld1(arow[g] + x);
                const T ak = MODE == FM_SQUARE ? av * av : av;
                acc[g] = fma(ak, (T)ld1(srow[g] + x), acc[g]);
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], off);
        if (lane < ng) {
            T mine = acc[0];
#pragma unroll
            for (int g = 1; g < G; ++g)
                if (lane == g) mine = acc[g];
            if (ascale) mine *= (T)ascale[ar] * (T)sscale[sr];
            u[pm] += coef * mine;
        }
    }
}

template <class T>
__global__ void stage2_identity_kernel(const T* __restrict__ S, int64_t lds, int64_t X,
                                       S2Outputs outs, T coef, T* __restrict__ u)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < outs.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = outs.arow[i];
        if (a < X) u[outs.perm[i]] += coef * S[(int64_t)outs.srow[i] * lds + a];
    }
}

// ------------------------------------------------------------------ one-sided terms
// one warp per segment
template <class T>
__global__ void segment_sums_kernel(const int32_t* __restrict__ seg, const int32_t* __restrict__ perm,
                                    int64_t K, const T* __restrict__ v, T coef, T* __restrict__ s)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < K; x += nw) {
        T acc = T(0);
        for (int32_t j = seg[x] + lane; j < seg[x + 1]; j += 32) acc += v[perm[j]];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) s[x] += coef * acc;
    }
}

// z_g[r] = sum_x F[r, x] s_g[x] for G vectors s_g = s + g lds in one pass over F
template <class T, int MODE, int G>
__global__ void gemv_rows_multi_kernel(const T* __restrict__ F, int64_t ldf, int64_t R, int64_t X,
                                       const T* __restrict__ s, int64_t lds, T* __restrict__ z, int64_t ldz)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += nw) {
        const T* row = F + r * ldf;
        T acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = T(0);
        for (int64_t x = lane; x < X; x += 32) {
            const T f = MODE == FM_SQUARE ? row[x] * row[x] : row[x];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = fma(f, s[g * lds + x], acc[g]);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], off);
            if (lane == 0) z[g * ldz + r] = acc[g];
        }
    }
}

// 16-byte vectors of T
template <class T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int width = 4;
    __device__ static void unpack(const float4& q, float (&o)[4])
    {
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int width = 2;
    __device__ static void unpack(const double2& q, double (&o)[2])
    {
        o[0] = q.x; o[1] = q.y;
    }
};

// The same product with 16-byte loads: one block of kGemvBlock threads per row, so that a row's
// loads are all in flight at once (about four per thread for rows of 2000 FP32), then a fixed-order
// block reduction.  F and the s_g 16-byte aligned, ldf and lds multiples of the vector width (the
// host checks).  Columns past the last whole vector are read one element per thread.
constexpr int kGemvBlock = 128;

template <class T, int MODE, int G>
__global__ void __launch_bounds__(kGemvBlock)
gemv_rows_multi_vec_kernel(const T* __restrict__ F, int64_t ldf, int64_t R, int64_t X,
                           const T* __restrict__ s, int64_t lds, T* __restrict__ z, int64_t ldz)
{
    using V = typename Vec16<T>::type;
    constexpr int W = Vec16<T>::width;
    constexpr int NWARP = kGemvBlock / 32;
    __shared__ T red[G][NWARP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t Xv = X / W * W;
    for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
        const T* row = F + r * ldf;
        T acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = T(0);
#pragma unroll 4
        for (int64_t x = (int64_t)threadIdx.x * W; x < Xv; x += kGemvBlock * W) {
            T f[W];
            Vec16<T>::unpack(__ldg(reinterpret_cast<const V*>(row + x)), f);
#pragma unroll
            for (int e = 0; e < W; ++e)
                if (MODE == FM_SQUARE) f[e] *= f[e];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                T sv[W];
                Vec16<T>::unpack(__ldg(reinterpret_cast<const V*>(s + g * lds + x)), sv);
#pragma unroll
                for (int e = 0; e < W; ++e) acc[g] = fma(f[e], sv[e], acc[g]);
            }
        }
        for (int64_t x = Xv + threadIdx.x; x < X; x += kGemvBlock) {
            const T f = MODE == FM_SQUARE ? row[x] * row[x] : row[x];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = fma(f, s[g * lds + x], acc[g]);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], off);
            if (lane == 0) red[g][warp] = acc[g];
        }
        __syncthreads();
        if (threadIdx.x < G) {
            T t = T(0);
#pragma unroll
            for (int w = 0; w < NWARP; ++w) t += red[threadIdx.x][w];
            z[threadIdx.x * ldz + r] = t;
        }
        __syncthreads();
    }
}

template <class T>
struct GatherSet {
    const T* z[kMaxOneSidedShare];
    const int32_t* idx[kMaxOneSidedShare];
    int count;
};

// u[i] += sum_g z_g[idx_g[i]]
template <class T>
__global__ void gather_add_multi_kernel(GatherSet<T> gs, int64_t n, T* __restrict__ u)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T acc = T(0);
#pragma unroll
        for (int g = 0; g < kMaxOneSidedShare; ++g)
            if (g < gs.count) acc += gs.z[g][gs.idx[g][i]];
        u[i] += acc;
    }
}

template <class T>
__global__ void transpose_kernel(const T* __restrict__ B, int64_t ldb, int64_t rows, int64_t cols,
                                 T* __restrict__ Bt, int64_t ldt)
{
    __shared__ T tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = B[r * ldb + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) Bt[c * ldt + r] = tile[threadIdx.x][k];
    }
}

template <class T>
__global__ void zero_kernel(T* __restrict__ x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = T(0);
}

template <class S, class D>
__device__ inline D cvt(S x) { return (D)x; }
template <> __device__ inline __nv_bfloat16 cvt<double, __nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <> __device__ inline __nv_bfloat16 cvt<float, __nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ inline double cvt<__nv_bfloat16, double>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <> __device__ inline float cvt<__nv_bfloat16, float>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ inline __nv_bfloat16 cvt<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 x) { return x; }

template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = cvt<S, D>(src[i]);
}

// Gaussian base kernel, FP64: a 32x32 output tile per block, features staged
// through shared memory in chunks of 32 dimensions.
template <class D>
__global__ void gaussian_kernel_kernel(const double* __restrict__ X, int64_t rx,
                                       const double* __restrict__ Y, int64_t ry, int64_t dim,
                                       double gamma, D* __restrict__ K, int64_t ldk)
{
    __shared__ double xs[32][33];
    __shared__ double ys[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t a0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t k0 = 0; k0 < dim; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int64_t a = a0 + r, b = b0 + r, k = k0 + tx;
            xs[r][tx] = (a < rx && k < dim) ? X[a * dim + k] : 0.0;
            ys[r][tx] = (b < ry && k < dim) ? Y[b * dim + k] : 0.0;
        }
        __syncthreads();
        const int kmax = (dim - k0 < 32) ? (int)(dim - k0) : 32;
        for (int kk = 0; kk < kmax; ++kk) {
            const double yv = ys[tx][kk];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const double d = xs[ty + 8 * i][kk] - yv;
                acc[i] = fma(d, d, acc[i]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + ty + 8 * i, b = b0 + tx;
        if (a < rx && b < ry) K[a * ldk + b] = cvt<double, D>(exp(-gamma * acc[i]));
    }
}

// Linear kernel K[a, b] = <X_a, Y_b> (Sec. 5: rows of a similarity matrix as feature vectors),
// FP64 sums over 32-wide feature tiles staged in shared memory; 32 x 32 output tile per block.
template <class D>
__global__ void linear_kernel_kernel(const double* __restrict__ X, int64_t rx, const double* __restrict__ Y,
                                     int64_t ry, int64_t dim, D* __restrict__ K, int64_t ldk)
{
    __shared__ double xs[32][33];
    __shared__ double ys[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t a0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t k0 = 0; k0 < dim; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int64_t a = a0 + r, b = b0 + r, k = k0 + tx;
            xs[r][tx] = (a < rx && k < dim) ? X[a * dim + k] : 0.0;
            ys[r][tx] = (b < ry && k < dim) ? Y[b * dim + k] : 0.0;
        }
        __syncthreads();
        const int kmax = (dim - k0 < 32) ? (int)(dim - k0) : 32;
        for (int kk = 0; kk < kmax; ++kk) {
            const double yv = ys[tx][kk];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fma(xs[ty + 8 * i][kk], yv, acc[i]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + ty + 8 * i, b = b0 + tx;
        if (a < rx && b < ry) K[a * ldk + b] = cvt<double, D>(acc[i]);
    }
}

// Tanimoto (MinMax) kernel of binary fingerprints, Sec. 5:
//   K[a, b] = |x_a AND y_b| / |x_a OR y_b|   (popcounts over `words` 32-bit words)
// with K = 1 when both fingerprints are empty.  32 x 32 output tile per block.
template <class D>
__global__ void tanimoto_kernel_kernel(const uint32_t* __restrict__ X, int64_t rx, const uint32_t* __restrict__ Y,
                                       int64_t ry, int64_t words, D* __restrict__ K, int64_t ldk)
{
    __shared__ uint32_t xs[32][33];
    __shared__ uint32_t ys[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int64_t a0 = (int64_t)blockIdx.y * 32, b0 = (int64_t)blockIdx.x * 32;
    uint32_t inter[4] = {0, 0, 0, 0}, uni[4] = {0, 0, 0, 0};
    for (int64_t k0 = 0; k0 < words; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int64_t a = a0 + r, b = b0 + r, k = k0 + tx;
            xs[r][tx] = (a < rx && k < words) ? X[a * words + k] : 0u;
            ys[r][tx] = (b < ry && k < words) ? Y[b * words + k] : 0u;
        }
        __syncthreads();
        const int kmax = (words - k0 < 32) ? (int)(words - k0) : 32;
        for (int kk = 0; kk < kmax; ++kk) {
            const uint32_t yv = ys[tx][kk];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t xv = xs[ty + 8 * i][kk];
                inter[i] += __popc(xv & yv);
                uni[i] += __popc(xv | yv);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + ty + 8 * i, b = b0 + tx;
        if (a < rx && b < ry)
            K[a * ldk + b] = cvt<double, D>(uni[i] ? (double)inter[i] / (double)uni[i] : 1.0);
    }
}

}  // namespace

size_t dtype_size(int dt)
{
    switch (dt) {
    case GVT_F64: return 8;
    case GVT_F32: return 4;
    case GVT_BF16: return 2;
    default: return 0;
    }
}

template <class T, int NT, int RPT>
static void launch_stage1(const T* Bt, int64_t ldb, int mode, const S1Sources& srcs, const T* v, T* S,
                          int64_t lds, int64_t Y, int64_t X, int64_t gx, cudaStream_t s)
{
    dim3 grid((unsigned)gx, (unsigned)((Y + NT * RPT - 1) / (NT * RPT)));
    if (mode == FM_SQUARE)
        stage1_sparse_kernel<T, FM_SQUARE, NT, RPT><<<grid, NT, 0, s>>>(Bt, ldb, srcs, v, S, lds, Y, X);
    else
        stage1_sparse_kernel<T, FM_DENSE, NT, RPT><<<grid, NT, 0, s>>>(Bt, ldb, srcs, v, S, lds, Y, X);
}

template <class T>
gvt_status stage1_sparse(const T* Bt, int64_t ldb, int mode, const S1Sources& srcs, const T* v,
                        T* S, int64_t lds, int64_t Y, int64_t X, cudaStream_t s)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    // rows per block: 1024 (128 x 8) for tall S, 256 (64 x 4) for short S (FP64: 512 / 128)
    constexpr bool f32 = sizeof(T) == 4;
    const int64_t gx = (X + kS1Cols - 1) / kS1Cols;
    const int64_t rows = Y >= 768 ? (f32 ? 1024 : 512) : (f32 ? 256 : 128);
    if (gx > INT32_MAX || (Y + rows - 1) / rows > 65535) {
        set_error("stage 1: too many rows or columns");
        return GVT_ERR_UNSUPPORTED;
    }
    if (Y >= 768) {
        if (f32) launch_stage1<T, 128, 8>(Bt, ldb, mode, srcs, v, S, lds, Y, X, gx, s);
        else launch_stage1<T, 128, 4>(Bt, ldb, mode, srcs, v, S, lds, Y, X, gx, s);
    } else {
        if (f32) launch_stage1<T, 64, 4>(Bt, ldb, mode, srcs, v, S, lds, Y, X, gx, s);
        else launch_stage1<T, 64, 2>(Bt, ldb, mode, srcs, v, S, lds, Y, X, gx, s);
    }
    GVT_LAUNCH_CHECK("stage1_sparse");
    return GVT_OK;
}

template <class T>
gvt_status stage1_identity(const S1Sources& srcs, const T* v, T* S, int64_t lds, int64_t Y,
                           int64_t X, cudaStream_t s)
{
    if (Y <= 0 || X <= 0) return GVT_OK;
    stage1_identity_kernel<T><<<grid1d(X * 32, 256), 256, 0, s>>>(srcs, v, S, lds, Y, X);
    GVT_LAUNCH_CHECK("stage1_identity");
    return GVT_OK;
}

template <class T>
gvt_status stage2_gather(const T* A, int64_t lda, int mode, const T* S, int64_t lds, int64_t X,
                        const S2Outputs& outs, double coef, T* u, cudaStream_t s)
{
    if (outs.n <= 0) return GVT_OK;
    const int64_t groups = (outs.n + kS2Group - 1) / kS2Group;
    const int64_t g = std::min<int64_t>((groups + (kS2Threads / 32) - 1) / (kS2Threads / 32), 152 * 64);
    if (mode == FM_SQUARE)
        stage2_gather_kernel<T, T, FM_SQUARE><<<(unsigned)g, kS2Threads, 0, s>>>(A, lda, nullptr, S, lds, nullptr, X,
                                                                                 outs, (T)coef, u);
    else
        stage2_gather_kernel<T, T, FM_DENSE><<<(unsigned)g, kS2Threads, 0, s>>>(A, lda, nullptr, S, lds, nullptr, X,
                                                                                outs, (T)coef, u);
    GVT_LAUNCH_CHECK("stage2_gather");
    return GVT_OK;
}

gvt_status stage2_gather_f16(const void* A, int64_t lda, const float* ascale, const void* S, int64_t lds,
                             const float* sscale, int64_t X, const S2Outputs& outs, double coef, float* u,
                             cudaStream_t s)
{
    if (outs.n <= 0) return GVT_OK;
    const int64_t groups = (outs.n + kS2Group - 1) / kS2Group;
    const int64_t g = std::min<int64_t>((groups + (kS2Threads / 32) - 1) / (kS2Threads / 32), 152 * 64);
    stage2_gather_kernel<float, __half, FM_DENSE><<<(unsigned)g, kS2Threads, 0, s>>>(
        static_cast<const __half*>(A), lda, ascale, static_cast<const __half*>(S), lds, sscale, X, outs, (float)coef, u);
    GVT_LAUNCH_CHECK("stage2_gather_f16");
    return GVT_OK;
}

template <class T>
gvt_status stage2_identity(const T* S, int64_t lds, int64_t X, const S2Outputs& outs, double coef,
                           T* u, cudaStream_t s)
{
    if (outs.n <= 0) return GVT_OK;
    stage2_identity_kernel<T><<<grid1d(outs.n, 256), 256, 0, s>>>(S, lds, X, outs, (T)coef, u);
    GVT_LAUNCH_CHECK("stage2_identity");
    return GVT_OK;
}

template <class T>
gvt_status segment_sums(const int32_t* seg, const int32_t* perm, int64_t K, const T* v, double coef,
                        T* s_out, cudaStream_t s)
{
    if (K <= 0) return GVT_OK;
    segment_sums_kernel<T><<<grid1d(K * 32, 256), 256, 0, s>>>(seg, perm, K, v, (T)coef, s_out);
    GVT_LAUNCH_CHECK("segment_sums");
    return GVT_OK;
}

template <class T>
gvt_status gemv_rows_multi(const T* F, int64_t ldf, int mode, int64_t R, int64_t X, const T* svecs, int64_t lds,
                           int count, T* z, int64_t ldz, cudaStream_t s)
{
    if (R <= 0 || count <= 0) return GVT_OK;
    const unsigned g = grid1d(R * 32, 256, 152 * 16);
    const unsigned gv = (unsigned)std::min<int64_t>(R, 152 * 64);   // a block per row
    constexpr int W = Vec16<T>::width;
    const bool vec = ((uintptr_t)F & 15) == 0 && ((uintptr_t)svecs & 15) == 0 && ldf % W == 0 && lds % W == 0;
#define GVT_GEMV_MULTI(G)                                                                                    \
    if (vec && mode == FM_SQUARE)                                                                            \
        gemv_rows_multi_vec_kernel<T, FM_SQUARE, G><<<gv, kGemvBlock, 0, s>>>(F, ldf, R, X, svecs, lds, z, ldz); \
    else if (vec)                                                                                            \
        gemv_rows_multi_vec_kernel<T, FM_DENSE, G><<<gv, kGemvBlock, 0, s>>>(F, ldf, R, X, svecs, lds, z, ldz);  \
    else if (mode == FM_SQUARE)                                                                              \
        gemv_rows_multi_kernel<T, FM_SQUARE, G><<<g, 256, 0, s>>>(F, ldf, R, X, svecs, lds, z, ldz);         \
    else                                                                                                     \
        gemv_rows_multi_kernel<T, FM_DENSE, G><<<g, 256, 0, s>>>(F, ldf, R, X, svecs, lds, z, ldz);
    switch (count) {
    case 1: GVT_GEMV_MULTI(1) break;
    case 2: GVT_GEMV_MULTI(2) break;
    case 3: GVT_GEMV_MULTI(3) break;
    default: GVT_GEMV_MULTI(4) break;
    }
#undef GVT_GEMV_MULTI
    GVT_LAUNCH_CHECK("gemv_rows_multi");
    return GVT_OK;
}

template <class T>
gvt_status gather_add_multi(const T* const* z, const int32_t* const* idx, int count, int64_t n, T* u,
                            cudaStream_t s)
{
    if (n <= 0 || count <= 0) return GVT_OK;
    GatherSet<T> gs{};
    gs.count = count < kMaxOneSidedShare ? count : kMaxOneSidedShare;
    for (int g = 0; g < gs.count; ++g) {
        gs.z[g] = z[g];
        gs.idx[g] = idx[g];
    }
    gather_add_multi_kernel<T><<<grid1d(n, 256), 256, 0, s>>>(gs, n, u);
    GVT_LAUNCH_CHECK("gather_add_multi");
    return GVT_OK;
}

template <class T>
gvt_status transpose(const T* B, int64_t ldb, int64_t rows, int64_t cols, T* Bt, int64_t ldt,
                     cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return GVT_OK;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(B, ldb, rows, cols, Bt, ldt);
    GVT_LAUNCH_CHECK("transpose");
    return GVT_OK;
}

template <class T>
gvt_status vec_zero(T* x, int64_t n, cudaStream_t s)
{
    if (n <= 0) return GVT_OK;
    zero_kernel<T><<<grid1d(n, 256), 256, 0, s>>>(x, n);
    GVT_LAUNCH_CHECK("zero");
    return GVT_OK;
}

gvt_status convert(const void* src, int sdt, void* dst, int ddt, int64_t n, cudaStream_t s)
{
    if (n <= 0) return GVT_OK;
    const unsigned g = grid1d(n, 256);
#define GVT_CVT(ST, SD, DT, DD)                                                               \
    if (sdt == SD && ddt == DD) {                                                             \
        convert_kernel<ST, DT><<<g, 256, 0, s>>>(static_cast<const ST*>(src), static_cast<DT*>(dst), n); \
        GVT_LAUNCH_CHECK("convert");                                                          \
        return GVT_OK;                                                                        \
    }
    GVT_CVT(double, GVT_F64, double, GVT_F64)
    GVT_CVT(double, GVT_F64, float, GVT_F32)
    GVT_CVT(double, GVT_F64, __nv_bfloat16, GVT_BF16)
    GVT_CVT(float, GVT_F32, double, GVT_F64)
    GVT_CVT(float, GVT_F32, float, GVT_F32)
    GVT_CVT(float, GVT_F32, __nv_bfloat16, GVT_BF16)
    GVT_CVT(__nv_bfloat16, GVT_BF16, double, GVT_F64)
    GVT_CVT(__nv_bfloat16, GVT_BF16, float, GVT_F32)
    GVT_CVT(__nv_bfloat16, GVT_BF16, __nv_bfloat16, GVT_BF16)
#undef GVT_CVT
    set_error("convert: unsupported dtype pair");
    return GVT_ERR_INVALID_ARG;
}

gvt_status gaussian_kernel(const double* X, int64_t rx, const double* Y, int64_t ry, int64_t dim,
                           double gamma, void* K, int64_t ldk, int dtype, cudaStream_t s)
{
    if (rx <= 0 || ry <= 0) return GVT_OK;
    dim3 grid((unsigned)((ry + 31) / 32), (unsigned)((rx + 31) / 32));
    dim3 block(32, 8);
    switch (dtype) {
    case GVT_F64:
        gaussian_kernel_kernel<double><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, gamma, (double*)K, ldk);
        break;
    case GVT_F32:
        gaussian_kernel_kernel<float><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, gamma, (float*)K, ldk);
        break;
    case GVT_BF16:
        gaussian_kernel_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, gamma,
                                                                    (__nv_bfloat16*)K, ldk);
        break;
    default:
        set_error("gaussian_kernel: bad dtype");
        return GVT_ERR_INVALID_ARG;
    }
    GVT_LAUNCH_CHECK("gaussian_kernel");
    return GVT_OK;
}

gvt_status linear_kernel(const double* X, int64_t rx, const double* Y, int64_t ry, int64_t dim, void* K,
                         int64_t ldk, int dtype, cudaStream_t s)
{
    if (rx <= 0 || ry <= 0) return GVT_OK;
    dim3 grid((unsigned)((ry + 31) / 32), (unsigned)((rx + 31) / 32));
    dim3 block(32, 8);
    switch (dtype) {
    case GVT_F64:
        linear_kernel_kernel<double><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, (double*)K, ldk);
        break;
    case GVT_F32:
        linear_kernel_kernel<float><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, (float*)K, ldk);
        break;
    case GVT_BF16:
        linear_kernel_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(X, rx, Y, ry, dim, (__nv_bfloat16*)K, ldk);
        break;
    default:
        set_error("linear_kernel: bad dtype");
        return GVT_ERR_INVALID_ARG;
    }
    GVT_LAUNCH_CHECK("linear_kernel");
    return GVT_OK;
}

gvt_status tanimoto_kernel(const uint32_t* X, int64_t rx, const uint32_t* Y, int64_t ry, int64_t words, void* K,
                           int64_t ldk, int dtype, cudaStream_t s)
{
    if (rx <= 0 || ry <= 0) return GVT_OK;
    dim3 grid((unsigned)((ry + 31) / 32), (unsigned)((rx + 31) / 32));
    dim3 block(32, 8);
    switch (dtype) {
    case GVT_F64:
        tanimoto_kernel_kernel<double><<<grid, block, 0, s>>>(X, rx, Y, ry, words, (double*)K, ldk);
        break;
    case GVT_F32:
        tanimoto_kernel_kernel<float><<<grid, block, 0, s>>>(X, rx, Y, ry, words, (float*)K, ldk);
        break;
    case GVT_BF16:
        tanimoto_kernel_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(X, rx, Y, ry, words, (__nv_bfloat16*)K, ldk);
        break;
    default:
        set_error("tanimoto_kernel: bad dtype");
        return GVT_ERR_INVALID_ARG;
    }
    GVT_LAUNCH_CHECK("tanimoto_kernel");
    return GVT_OK;
}

#define GVT_INST(T)                                                                                 \
    template gvt_status stage1_sparse<T>(const T*, int64_t, int, const S1Sources&, const T*, T*,      \
                                        int64_t, int64_t, int64_t, cudaStream_t);                     \
    template gvt_status stage1_identity<T>(const S1Sources&, const T*, T*, int64_t, int64_t,        \
                                           int64_t, cudaStream_t);                                  \
    template gvt_status stage2_gather<T>(const T*, int64_t, int, const T*, int64_t, int64_t,          \
                                        const S2Outputs&, double, T*, cudaStream_t);                \
    template gvt_status stage2_identity<T>(const T*, int64_t, int64_t, const S2Outputs&, double, T*, \
                                           cudaStream_t);                                           \
    template gvt_status segment_sums<T>(const int32_t*, const int32_t*, int64_t, const T*, double,  \
                                        T*, cudaStream_t);                                          \
    template gvt_status gemv_rows_multi<T>(const T*, int64_t, int, int64_t, int64_t, const T*, int64_t, int, \
                                           T*, int64_t, cudaStream_t);                                   \
    template gvt_status gather_add_multi<T>(const T* const*, const int32_t* const*, int, int64_t, T*,     \
                                            cudaStream_t);                                               \
    template gvt_status transpose<T>(const T*, int64_t, int64_t, int64_t, T*, int64_t,              \
                                     cudaStream_t);                                                 \
    template gvt_status vec_zero<T>(T*, int64_t, cudaStream_t);

GVT_INST(float)
GVT_INST(double)

}  // namespace gvt
