// Plan construction kernels: a stable LSD radix sort of pair components,
// segment offsets (the CSC column pointers of the sparse W of Theorem 1),
// gathers and index validation.
#include <climits>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int kSortThreads = 256;                 // 8 warps
constexpr int kSortWarpItems = 256;               // consecutive elements per warp
constexpr int kSortTile = kSortWarpItems * 8;     // 2048 elements per block
constexpr int kDigits = 256;                      // 8-bit digits

// Pass 1 of a radix pass: per block, the count of every digit and the stable
// rank of every element among the block's elements with the same digit.
__global__ void __launch_bounds__(kSortThreads)
radix_rank_kernel(const int32_t* __restrict__ keys, int64_t n, int shift,
                  int32_t* __restrict__ tile_rank, int32_t* __restrict__ counts, int num_tiles)
{
    __shared__ int cnt[8][kDigits + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 8 * (kDigits + 1); i += kSortThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kSortWarpItems;
    const unsigned lt = (1u << lane) - 1u;
    int dig[8], lrank[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t e = base + r * 32 + lane;
        const int dg = (e < n) ? ((keys[e] >> shift) & (kDigits - 1)) : kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const int leader = __ffs(peers) - 1;
        const int before = cnt[warp][dg];
        __syncwarp();
        if (lane == leader) cnt[warp][dg] = before + __popc(peers);
        __syncwarp();
        dig[r] = dg;
        lrank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // exclusive prefix over the warps, per digit (thread d owns digit d)
        const int d = threadIdx.x;
        int run = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
        counts[(int64_t)d * num_tiles + blockIdx.x] = run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t e = base + r * 32 + lane;
        if (e < n) tile_rank[e] = cnt[warp][dig[r]] + lrank[r];
    }
}

// Pass 2: move every element to its stable position.
__global__ void radix_scatter_kernel(const int32_t* __restrict__ keys_in,
                                     const int32_t* __restrict__ vals_in, int64_t n, int shift,
                                     const int32_t* __restrict__ tile_rank,
                                     const int32_t* __restrict__ offsets, int num_tiles,
                                     int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = keys_in[e];
        const int dg = (k >> shift) & (kDigits - 1);
        const int64_t tile = e / kSortTile;
        const int32_t pos = offsets[(int64_t)dg * num_tiles + tile] + tile_rank[e];
        keys_out[pos] = k;
        vals_out[pos] = vals_in ? vals_in[e] : (int32_t)e;
    }
}

// ------------------------------------------------------------- exclusive scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;   // 1024

__device__ int block_exclusive_scan(int x, int* smem_warp, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < kScanThreads / 32) ? smem_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) smem_warp[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    const int r = smem_warp[warp] + incl - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads)
scan_block_sums_kernel(const int32_t* __restrict__ in, int64_t L, int32_t* __restrict__ sums)
{
    __shared__ int sw[32];
    __shared__ int tot;
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (b0 + i < L) s += in[b0 + i];
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums, in place.
__global__ void __launch_bounds__(kScanThreads)
scan_sums_kernel(int32_t* __restrict__ sums, int64_t nb)
{
    __shared__ int sw[32];
    __shared__ int tot;
    int carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanBlock) {
        const int64_t b0 = c0 + threadIdx.x * kScanItems;
        int v[kScanItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (b0 + i < nb) ? sums[b0 + i] : 0;
            s += v[i];
        }
        int ex = block_exclusive_scan(s, sw, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (b0 + i < nb) sums[b0 + i] = ex;
            ex += v[i];
        }
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(const int32_t* __restrict__ in, int64_t L, const int32_t* __restrict__ sums,
                  int32_t* __restrict__ out)
{
    __shared__ int sw[32];
    __shared__ int tot;
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (b0 + i < L) ? in[b0 + i] : 0;
        s += v[i];
    }
    int ex = block_exclusive_scan(s, sw, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (b0 + i < L) out[b0 + i] = ex;
        ex += v[i];
    }
}

gvt_status exclusive_scan(const int32_t* in, int64_t L, int32_t* out, int32_t* sums,
                          cudaStream_t s)
{
    if (L <= 0) return GVT_OK;
    const int64_t nb = (L + kScanBlock - 1) / kScanBlock;
    scan_block_sums_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, L, sums);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, nb);
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, L, sums, out);
    GVT_LAUNCHED(3, "scan");
    return GVT_OK;
}

__global__ void iota_kernel(int32_t* __restrict__ out, const int32_t* __restrict__ keys,
                            int32_t* __restrict__ key_out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = (int32_t)i;
        key_out[i] = keys[i];
    }
}

__global__ void segment_offsets_kernel(const int32_t* __restrict__ key, int64_t n, int64_t K,
                                       int32_t* __restrict__ seg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = (i == 0) ? -1 : key[i - 1];
        const int64_t cur = (i == n) ? K : key[i];
        for (int64_t k = prev + 1; k <= cur; ++k) seg[k] = (int32_t)i;
    }
}

__global__ void gather_i32_kernel(const int32_t* __restrict__ in, const int32_t* __restrict__ perm,
                                  int64_t n, int32_t* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

__global__ void minmax_init_kernel(int32_t* mm)
{
    mm[0] = INT_MAX;
    mm[1] = INT_MIN;
}

__global__ void minmax_kernel(const int32_t* __restrict__ x, int64_t n, int32_t* __restrict__ mm)
{
    int lo = INT_MAX, hi = INT_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = x[i];
        lo = min(lo, v);
        hi = max(hi, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

}  // namespace

size_t sort_workspace_bytes(int64_t n)
{
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t L = tiles * kDigits;
    const int64_t nb = (L + kScanBlock - 1) / kScanBlock;
    auto al = [](int64_t b) { return (size_t)((b + 255) & ~int64_t(255)); };
    return al(4 * n) * 5 + al(4 * L) * 2 + al(4 * (nb + 1));
}

gvt_status radix_sort_by_key(const int32_t* keys, int64_t n, int64_t K, int32_t* out_key,
                             int32_t* out_perm, void* ws, cudaStream_t s)
{
    if (n <= 0) return GVT_OK;
    int bits = 0;
    while (bits < 31 && (int64_t(1) << bits) < K) ++bits;
    const int passes = (bits + 7) / 8;
    if (passes == 0) {
        iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(out_perm, keys, out_key, n);
        GVT_LAUNCH_CHECK("iota");
        return GVT_OK;
    }
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t L = tiles * kDigits;
    auto al = [](int64_t b) { return (size_t)((b + 255) & ~int64_t(255)); };
    char* p = static_cast<char*>(ws);
    int32_t* ka = reinterpret_cast<int32_t*>(p); p += al(4 * n);
    int32_t* kb = reinterpret_cast<int32_t*>(p); p += al(4 * n);
    int32_t* va = reinterpret_cast<int32_t*>(p); p += al(4 * n);
    int32_t* vb = reinterpret_cast<int32_t*>(p); p += al(4 * n);
    int32_t* rank = reinterpret_cast<int32_t*>(p); p += al(4 * n);
    int32_t* counts = reinterpret_cast<int32_t*>(p); p += al(4 * L);
    int32_t* offs = reinterpret_cast<int32_t*>(p); p += al(4 * L);
    int32_t* sums = reinterpret_cast<int32_t*>(p);

    const int32_t* kin = keys;
    const int32_t* vin = nullptr;   // first pass: values are the indices themselves
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const bool last = (pass == passes - 1);
        int32_t* kout = last ? out_key : ((pass & 1) ? kb : ka);
        int32_t* vout = last ? out_perm : ((pass & 1) ? vb : va);
        radix_rank_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(kin, n, shift, rank, counts,
                                                                  (int)tiles);
        GVT_LAUNCH_CHECK("radix_rank");
        GVT_CHECK(exclusive_scan(counts, L, offs, sums, s));
        radix_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(kin, vin, n, shift, rank, offs,
                                                              (int)tiles, kout, vout);
        GVT_LAUNCH_CHECK("radix_scatter");
        kin = kout;
        vin = vout;
    }
    return GVT_OK;
}

gvt_status segment_offsets(const int32_t* sorted_key, int64_t n, int64_t K, int32_t* seg,
                           cudaStream_t s)
{
    segment_offsets_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(sorted_key, n, K, seg);
    GVT_LAUNCH_CHECK("segment_offsets");
    return GVT_OK;
}

gvt_status gather_i32(const int32_t* in, const int32_t* perm, int64_t n, int32_t* out,
                      cudaStream_t s)
{
    if (n <= 0) return GVT_OK;
    gather_i32_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, perm, n, out);
    GVT_LAUNCH_CHECK("gather_i32");
    return GVT_OK;
}

gvt_status minmax_i32(const int32_t* x, int64_t n, int32_t* mm, cudaStream_t s)
{
    minmax_init_kernel<<<1, 1, 0, s>>>(mm);
    minmax_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, n, mm);
    GVT_LAUNCHED(2, "minmax");
    return GVT_OK;
}

}  // namespace gvt
