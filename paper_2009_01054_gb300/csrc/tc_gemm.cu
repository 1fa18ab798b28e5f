// Dense stages on the 5th-generation tensor cores.
//
// A BF16 or FP16 GEMM  C[M x N] (FP32) = rs[m] cs[n] (A[M x K] * B[N x K]^T)[m, n]
// with both operands K-major (row-major with K innermost) and optional FP32
// row and column scales applied in the epilogue.  One CTA computes a 128 x BN
// tile of C (optionally one K slice of it, reduced with atomic adds):
//   warp 0, one thread : TMA producer -- cp.async.bulk.tensor 2-D loads of
//                        128 x 64 (A) and BN x 64 (B) tiles, 128-byte swizzle,
//                        into a ring of tc_stages<BN>() slots (as many as fit
//                        in shared memory), completion on mbarriers;
//   warp 1, one thread : MMA issuer -- tcgen05.mma kind::f16 (BF16 or FP16 in,
//                        both operands the same type, FP32 accumulate in TMEM),
//                        K = 16 per instruction, then tcgen05.commit to free the
//                        ring slot;
//   warps 2-9          : folding -- the accumulation runs in chunks of
//                        TC_CHUNK k-blocks, alternating between two TMEM
//                        accumulators; after each chunk these warps read the
//                        chunk's accumulator (tcgen05.ld 32x32b; warp w reaches
//                        TMEM lanes 32 (w % 4)..+31, and warps w, w + 4 split the
//                        columns) and add it into FP32 registers, then free it.
//                        At the end they scale and store the sums to C.
// Why the folding: the tensor core's accumulation rounds toward zero, so one
// long accumulation chain drifts systematically (about -1e-5 relative after
// K = 4096 on positive data, measured on GB300), while chunks of 512 stay near
// FP32 rounding (-7e-7) and the folds round to nearest.
// SM-pair form (PAIR = true): a cluster of two CTAs on neighbouring SMs
// computes a 256 x BN tile with tcgen05.mma.cta_group::2 (M = 256).  Each CTA
// loads its own 128 rows of A and half of the BN rows of B, so per SM the
// tensor core reads 128 + BN/2 operand rows from shared memory per k-block
// instead of 128 + BN; each CTA's TMEM holds the accumulator of its own 128
// rows.  Only the even CTA issues MMAs.  The tile loads of both CTAs
// complete on the even CTA's ring barrier (cp.async.bulk.tensor .cta_group::2),
// the MMA commits arrive on both CTAs' barriers (multicast), and the odd CTA's
// folding warps release an accumulator on the even CTA's barrier.  (Having the
// odd CTA wait for its own loads and forward their completion instead adds a
// hop to every ring slot and measured half the speed.)
// Epilogue: the folding warps stage the 128 x BN tile in the (then idle) ring
// memory and store it row by row, 32 consecutive columns per warp instruction.
// Two sparse forms (no split K), for the per-tile dense/sparse stages: a
// block-sparse B (also in the SM-pair form), where the CTA of N tile j runs only over the
// k-blocks kb_list[kb_off[j] .. kb_off[j+1]) (in each of the `parts` K
// segments of a split operand, kb_stride k-blocks apart; an N tile with no
// k-block stores zeros); and a tile list, where CTA b computes only output
// tile tile_list[b] = (m tile, n tile) (one SM).
// Grouped tiles (one-SM, for many small independent GEMMs in one launch): CTA b
// reads its record group[b] -- first A row, first B row, k-block count, valid
// rows and columns, and the output's offset and row stride -- and computes one
// 128 x BN tile over k-blocks 0 .. nkb-1 of its rows.
// CTA order (one-SM grid form): groups of TC_GROUP_M m tiles, m tile fastest
// within a group, so that the CTAs resident at one time share operand strips
// in L2; the caller orders a tile list the same way.
// Every wait on an mbarrier is bounded by a clock budget, and the waits of the
// pipeline also end as soon as another thread of the CTA has timed out; on
// expiry the thread records GVT_ERR_TIMEOUT in a device error word, the kernel
// waits (bounded) for the copies it issued and for its MMAs, frees its TMEM
// and returns.  A test switch (stall_cycles > 0, one-SM form only) makes the
// MMA thread first wait on a barrier that nothing arrives on, for that many
// cycles, so that the timeout path runs on demand.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;            // BF16 elements in one 128-byte swizzle row
constexpr int TC_MAX_STAGES = 8;
constexpr size_t TC_SMEM_LIMIT = 227 * 1024;
constexpr int TC_THREADS = 320;           // producer warp, MMA warp, 8 folding warps
constexpr int TC_FOLD_WARPS = 8;
constexpr int TC_CHUNK = 8;               // k-blocks (8 x 64 = 512 of K) per accumulation chunk
// m tiles per group of the CTA order: a wave of 152 CTAs then covers 16 A strips of 128 rows and
// about 9 B strips of 256 rows (the two operands' bytes per wave about equal), instead of 152 A
// strips and one B strip
constexpr int TC_GROUP_M = 16;
constexpr long long TC_TIMEOUT_CYCLES = 4000000000ll;   // about 2 s at 2 GHz
constexpr long long TC_DRAIN_CYCLES = 20000000ll;       // about 10 ms

struct TcShared {
    uint64_t full[TC_MAX_STAGES];
    uint64_t empty[TC_MAX_STAGES];
    uint64_t acc_full[2];    // chunk accumulated into TMEM buffer b
    uint64_t acc_empty[2];   // folding warps have read buffer b
    uint64_t mma_done;       // every MMA this CTA issued has completed
    uint64_t never;          // nothing arrives on it: the target of the test stall
    uint32_t tmem_base;
    int timeout;
    int issued;      // TMA stage loads issued
    int consumed;    // stage loads the MMA thread has waited for (one-SM form)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that also acquires what other CTAs of the cluster released before arriving
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on timeout, or as soon as *abort (a
// shared-memory flag, may be NULL) is set by another thread that timed out.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int* abort = nullptr,
                                          long long budget = TC_TIMEOUT_CYCLES)
{
    const long long t0 = clock64();
    while (!(CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))) {
        if (clock64() - t0 > budget) return false;
        if (abort && *(const volatile int*)abort) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Arrive on the barrier at the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint64_t* bar, uint32_t rank)
{
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// Every thread of both CTAs of the cluster.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// SM-pair form: load into this CTA's shared memory, completing on the barrier at the same offset
// in CTA `rank` of the pair.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint64_t* bar, uint32_t rank,
                                                 int x, int y)
{
    uint32_t rbar;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(smem_u32(bar)), "r"(rank));
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(rbar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Every tcgen05 instruction of one kernel uses the same CTA group: ::1 in the one-SM form, ::2 in
// the SM-pair form, where the allocation is made collectively by warp 0 of both CTAs.
template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    if constexpr (PAIR)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                     "r"(ncols)
                     : "memory");
    else
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                     "r"(ncols)
                     : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_relinquish()
{
    if constexpr (PAIR)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    else
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    if constexpr (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, 16-bit x 16-bit -> FP32
template <bool PAIR>
__device__ __forceinline__ void umma_f16kind(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate)
{
    if constexpr (PAIR)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread completed: in the
// one-SM form on this CTA's barrier, in the SM-pair form on the barrier at the same offset in
// both CTAs of the pair.
template <bool PAIR>
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    if constexpr (PAIR)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
            ::"r"(smem_u32(bar)), "h"((uint16_t)3)
            : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(bar))
                     : "memory");
}

// SM-pair form: arrive on this CTA's barrier only.
__device__ __forceinline__ void umma_commit_local_pair(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout written by TMA: rows of 128 bytes, 8-row (1024-byte) swizzle atoms
// stacked along M/N.  Fields: start address >> 4 (bits 0-13), leading byte
// offset >> 4 (bits 16-29, unused for this layout), stride byte offset >> 4
// (bits 32-45) = 1024 B between 8-row groups, descriptor version 1 (bits
// 46-47), base offset 0 (tiles are 1024-byte aligned), layout type
// SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B both BF16 (format 1 at bits 7-9 and 10-12) or both FP16 (format 0),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
// (M = 128 for one SM, 256 for an SM pair).
template <int BN, bool F16, bool PAIR>
__host__ __device__ constexpr uint32_t idesc_f16kind_f32()
{
    return (1u << 4) | (F16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)((PAIR ? 2 * TC_BM : TC_BM) >> 4) << 24);
}

// B rows one CTA loads per k-block: all BN, or its half of them in the SM-pair form
template <int BN, bool PAIR>
__host__ __device__ constexpr int tc_b_rows()
{
    return PAIR ? BN / 2 : BN;
}

// ring depth: as many A + B stages as fit in shared memory beside the barriers; narrow tiles
// keep a 4-deep ring so that two CTAs share an SM (their grids are the split-K ones)
template <int BN, bool PAIR>
__host__ __device__ constexpr int tc_stages()
{
    constexpr size_t stage = (size_t)(TC_BM + tc_b_rows<BN, PAIR>()) * TC_BK * 2;
    constexpr size_t n = (TC_SMEM_LIMIT - sizeof(TcShared) - 1024) / stage;
    constexpr int cap = BN <= 64 ? 4 : TC_MAX_STAGES;
    return n > (size_t)cap ? cap : (int)n;
}

template <int BN, bool PAIR>
__host__ __device__ constexpr size_t tc_smem_bytes()
{
    return (size_t)tc_stages<BN, PAIR>() * (TC_BM + tc_b_rows<BN, PAIR>()) * TC_BK * 2 + sizeof(TcShared) + 1024;
}

// TMEM columns of the two accumulators, rounded up to a power of two
template <int BN>
__host__ __device__ constexpr uint32_t tc_tmem_cols()
{
    return 2 * BN <= 128 ? 128u : 2 * BN <= 256 ? 256u : 512u;
}

template <int BN, bool F16, bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               float* __restrict__ C, int64_t ldc, int M, int N, int kb_total, int kb_per_split,
               int atomic_out, const float* __restrict__ row_scale, const float* __restrict__ col_scale,
               int* __restrict__ err, long long stall_cycles, const int* __restrict__ kb_list,
               const int* __restrict__ kb_off, int kb_parts, int kb_stride, const int2* __restrict__ tile_list,
               const TcGroupTile* __restrict__ group)
{
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "UMMA N");
    static_assert(!PAIR || BN % 16 == 0, "UMMA N for M = 256");
    constexpr int TC_STAGES = tc_stages<BN, PAIR>();
    static_assert(TC_STAGES >= 2, "ring depth");
    constexpr int B_ROWS = tc_b_rows<BN, PAIR>();
    constexpr int A_BYTES = TC_BM * TC_BK * 2;
    constexpr int B_BYTES = B_ROWS * TC_BK * 2;
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms");
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int HALF = BN / 2;            // columns one folding warp owns
    constexpr uint32_t TMEM_COLS = tc_tmem_cols<BN>();  // two accumulators
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment of the shared-space offset (swizzle atoms, descriptor base offset 0);
    // the offset is the same in both CTAs of a pair, as the leader's descriptors require
    unsigned char* tiles = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    TcShared* sh = reinterpret_cast<TcShared*>(tiles + TC_STAGES * STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // SM pair: CTA rank 0 (the leader) holds rows 0-127 of the 256-row tile and B rows
    // 0..BN/2-1, rank 1 the rest
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const bool leader = rank == 0;
    int mt = PAIR ? (int)(blockIdx.x >> 1) * 2 + (int)rank : (int)blockIdx.x, nt = blockIdx.y;
    if (!PAIR && tile_list) {
        const int2 tl = tile_list[blockIdx.x];
        mt = tl.x;
        nt = tl.y;
    } else if (!PAIR && group) {
        mt = nt = 0;
    } else {
        // grouped order: consecutive CTAs (clusters, in the SM-pair form) take TC_GROUP_M m tiles
        // (fastest) by as many n tiles as a wave holds, so that the CTAs resident at one time share
        // their A and B strips in L2; both CTAs of a pair get the same 256-row tile
        const int64_t ux = PAIR ? gridDim.x / 2 : gridDim.x;   // units along m: tiles or pairs
        const int64_t gm = PAIR ? TC_GROUP_M / 2 : TC_GROUP_M;
        const int64_t pid = (int64_t)blockIdx.y * ux + (PAIR ? blockIdx.x >> 1 : blockIdx.x);
        const int64_t per_group = gm * gridDim.y;
        const int64_t g = pid / per_group;
        const int64_t first = g * gm;
        const int64_t gsz = min(ux - first, gm);
        const int64_t r = pid - g * per_group;
        const int unit = (int)(first + r % gsz);
        mt = PAIR ? unit * 2 + (int)rank : unit;
        nt = (int)(r / gsz);
    }
    // grouped tiles: A rows, B rows, k-blocks and output placement come from the tile's record
    const TcGroupTile gt = (!PAIR && group) ? group[blockIdx.x] : TcGroupTile{};
    const bool grouped = !PAIR && group != nullptr;
    const int m0 = grouped ? gt.a_row : mt * TC_BM;
    const int n0 = grouped ? gt.b_row : nt * BN;
    const int nb0 = n0 + (int)rank * B_ROWS;   // first B row this CTA loads
    // k-blocks of this CTA: a contiguous range (split K), or kb_parts copies of this N tile's list
    const int kl0 = kb_list ? kb_off[nt] : 0;
    const int kcount = kb_list ? kb_off[nt + 1] - kl0 : 0;
    const int kb0 = grouped ? 0 : blockIdx.z * kb_per_split;
    const int kb1 = grouped ? gt.nkb : min(kb_total, kb0 + kb_per_split);
    const int nkb = kb_list ? kcount * kb_parts : max(kb1 - kb0, 0);
    const int nchunks = (nkb + TC_CHUNK - 1) / TC_CHUNK;

    if (threadIdx.x == 0) {
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(&sh->full[st], 1);   // SM pair: only the leader's are used
            mbar_init(&sh->empty[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->acc_full[b], 1);
            mbar_init(&sh->acc_empty[b], PAIR ? 2 * TC_FOLD_WARPS : TC_FOLD_WARPS);
        }
        mbar_init(&sh->mma_done, 1);
        mbar_init(&sh->never, 1);
        sh->timeout = 0;
        sh->issued = 0;
        sh->consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc<PAIR>(&sh->tmem_base, TMEM_COLS);
        tmem_relinquish<PAIR>();
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync();   // barriers of both CTAs initialised before any remote arrival
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int i = 0;
            for (; i < nkb; ++i) {
                const int st = i % TC_STAGES;
                if (i >= TC_STAGES && !mbar_wait(&sh->empty[st], ((i / TC_STAGES) - 1) & 1, &sh->timeout)) {
                    atomicExch(&sh->timeout, 1);
                    break;
                }
                if (*(volatile int*)&sh->timeout) break;
                unsigned char* sa = tiles + st * STAGE_BYTES;
                const int kx = (kb_list ? (i / kcount) * kb_stride + kb_list[kl0 + i % kcount] : kb0 + i) * TC_BK;
                if constexpr (PAIR) {
                    // the leader's slot completes when the loads of both CTAs landed
                    if (leader) mbar_expect_tx(&sh->full[st], 2 * STAGE_BYTES);
                    tma_load_2d_pair(sa, &mapA, &sh->full[st], 0, kx, m0);
                    tma_load_2d_pair(sa + A_BYTES, &mapB, &sh->full[st], 0, kx, nb0);
                } else {
                    mbar_expect_tx(&sh->full[st], STAGE_BYTES);
                    tma_load_2d(sa, &mapA, &sh->full[st], kx, m0);
                    tma_load_2d(sa + A_BYTES, &mapB, &sh->full[st], kx, nb0);
                }
            }
            sh->issued = i;
        }
    } else if (warp == 1) {
        if (lane == 0 && (!PAIR || leader)) {
            // ---- MMA issuer: chunk c accumulates into TMEM buffer c & 1
            constexpr uint32_t idesc = idesc_f16kind_f32<BN, F16, PAIR>();
            int i = 0;
            bool ok = true;
            if (!PAIR && stall_cycles > 0 && !mbar_wait(&sh->never, 0, nullptr, stall_cycles)) {
                atomicExch(&sh->timeout, 1);   // the test stall: nothing arrives on `never`
                ok = false;
            }
            for (int c = 0; c < nchunks && ok; ++c) {
                const int b = c & 1;
                if (c >= 2 && !mbar_wait<PAIR>(&sh->acc_empty[b], ((c >> 1) - 1) & 1, &sh->timeout)) {
                    atomicExch(&sh->timeout, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t dst = tmem + (uint32_t)(b * BN);
                const int i_end = min(nkb, (c + 1) * TC_CHUNK);
                for (; i < i_end; ++i) {
                    const int st = i % TC_STAGES;
                    if (!mbar_wait<PAIR>(&sh->full[st], (i / TC_STAGES) & 1, &sh->timeout) ||
                        *(volatile int*)&sh->timeout) {
                        atomicExch(&sh->timeout, 1);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + st * STAGE_BYTES);
                    const uint64_t da = sdesc_sw128(sa), db = sdesc_sw128(sa + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk)   // +32 bytes along K per instruction
                        umma_f16kind<PAIR>(dst, da + 2 * kk, db + 2 * kk, idesc,
                                           (i > c * TC_CHUNK || kk > 0) ? 1u : 0u);
                    umma_commit<PAIR>(&sh->empty[st]);
                }
                if (ok) umma_commit<PAIR>(&sh->acc_full[b]);
            }
            sh->consumed = i;
            if (PAIR && i > 0) {
                // the peer's shared memory and TMEM stay in use until these MMAs complete
                umma_commit_local_pair(&sh->mma_done);
                if (!mbar_wait(&sh->mma_done, 0)) atomicExch(&sh->timeout, 1);
            } else if (!PAIR && i > 0) {
                // TMEM is freed at the end: every MMA issued must have completed by then, also
                // when a timeout left its accumulator unread
                umma_commit<false>(&sh->mma_done);
                if (!mbar_wait(&sh->mma_done, 0)) atomicExch(&sh->timeout, 1);
            }
        }
    } else {
        // ---- folding warps: FP32 register sums of the chunk accumulators
        const int fw = warp - 2;                 // 0..7
        const int quarter = warp & 3;            // TMEM lanes this warp may read
        const int col0 = (fw >> 2) * HALF;       // column half
        const int row = quarter * 32 + lane;     // tile row of this thread
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
        float acc[HALF];
#pragma unroll
        for (int e = 0; e < HALF; ++e) acc[e] = 0.f;
        // (an N tile without k-blocks in the block-sparse form stores its zero sums)
        bool good = nkb > 0 || kb_list != nullptr;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (!mbar_wait(&sh->acc_full[b], (c >> 1) & 1, &sh->timeout)) {
                atomicExch(&sh->timeout, 1);
                good = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int j = 0; j + 32 <= HALF; j += 32) {   // two loads in flight per wait
                uint32_t r0[16], r1[16];
                tmem_ld16(tl + (uint32_t)(b * BN + j), r0);
                tmem_ld16(tl + (uint32_t)(b * BN + j + 16), r1);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    acc[j + e] += __uint_as_float(r0[e]);
                    acc[j + 16 + e] += __uint_as_float(r1[e]);
                }
            }
            if constexpr (HALF % 32 != 0) {
                constexpr int j = HALF / 32 * 32;
                uint32_t r0[16];
                tmem_ld16(tl + (uint32_t)(b * BN + j), r0);
                tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[j + e] += __uint_as_float(r0[e]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR && !leader) mbar_arrive_remote(&sh->acc_empty[b], 0);
                else mbar_arrive(&sh->acc_empty[b]);
            }
        }
        // Stage the tile in the ring memory: once the last chunk's accumulator has arrived, every
        // MMA, and with it every read of the ring and every tile load, has completed.  The row
        // stride BN + 1 puts the 32 rows a warp writes at one column in 32 different banks.
        constexpr int SLD = BN + 1;
        static_assert((size_t)TC_BM * SLD * sizeof(float) <= (size_t)TC_STAGES * STAGE_BYTES, "staging");
        float* stage = reinterpret_cast<float*>(tiles);
        if (good) {
#pragma unroll
            for (int e = 0; e < HALF; ++e) stage[row * SLD + col0 + e] = acc[e];
        }
        asm volatile("bar.sync 1, %0;" ::"n"(TC_FOLD_WARPS * 32) : "memory");   // folding warps only
        if ((nkb > 0 || kb_list != nullptr) && *(volatile int*)&sh->timeout == 0) {
            const int ncols = grouped ? min(BN, gt.n_valid) : min(BN, N - n0);
            const int nrows = grouped ? min(TC_BM, gt.m_valid) : min(TC_BM, M - m0);
            float* cbase = grouped ? C + gt.c_off : C + (int64_t)m0 * ldc + n0;
            const int64_t ldo = grouped ? gt.ldc : ldc;
            for (int r = fw; r < nrows; r += TC_FOLD_WARPS) {
                const int gm = m0 + r;
                const float rs = row_scale ? row_scale[gm] : 1.f;
                float* crow = cbase + (int64_t)r * ldo;
                for (int cc = lane; cc < ncols; cc += 32) {
                    float f = stage[r * SLD + cc] * rs;
                    if (col_scale) f *= col_scale[n0 + cc];
                    if (atomic_out) atomicAdd(crow + cc, f);
                    else crow[cc] = f;
                }
            }
        }
    }

    __syncthreads();
    if (threadIdx.x == 0 && sh->timeout) {
        atomicExch(err, (int)GVT_ERR_TIMEOUT);
        if constexpr (PAIR) {
            // the loads of both CTAs complete on the leader's barriers, whose phases need not
            // finish after a timeout: give copies in flight a fixed time to land (they take
            // microseconds)
            const long long t0 = clock64();
            while (clock64() - t0 < TC_DRAIN_CYCLES) {
            }
        } else {
            // wait (bounded) for the tile copies that were issued but never consumed
            for (int i = sh->consumed; i < sh->issued; ++i)
                if (!mbar_wait(&sh->full[i % TC_STAGES], (i / TC_STAGES) & 1)) break;
        }
    }
    tc_fence_before();
    // SM pair: neither CTA frees TMEM or exits while the other may still arrive on its barriers
    if constexpr (PAIR) cluster_sync();
    else __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc<PAIR>(tmem, TMEM_COLS);
    }
}

__global__ void zero_rows_kernel(float* __restrict__ C, int64_t ldc, int64_t M, int64_t N)
{
    const int64_t total = M * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        C[(i / N) * ldc + (i % N)] = 0.f;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

gvt_status get_encode()
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (g_encode_err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return GVT_ERR_CUDA;
    }
    return GVT_OK;
}

gvt_status make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int64_t ld, int box_rows, bool f16)
{
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return GVT_ERR_CUDA;
    }
    return GVT_OK;
}

template <int BN, bool F16, bool PAIR>
gvt_status launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int64_t ldc, int64_t M, int64_t N,
                     int64_t K, const float* rs, const float* cs, int* err, long long stall, const TcSparse& sp,
                     cudaStream_t s)
{
    const int pairs = (int)((M + 2 * TC_BM - 1) / (2 * TC_BM));
    int gx = PAIR ? 2 * pairs : (int)((M + TC_BM - 1) / TC_BM), gy = (int)((N + BN - 1) / BN);
    const int kb_total = (int)(K / TC_BK);
    if (sp.tile_list || sp.group) {   // one CTA per listed output tile
        gx = (int)sp.n_tiles;
        gy = 1;
    }
    const int tiles = gx * gy;
    // split K only when the output tiles alone leave most SMs idle (never in the sparse forms)
    int splits = tiles >= 100 ? 1 : (148 + tiles - 1) / tiles;
    splits = std::max(1, std::min(splits, kb_total / 8));
    if (sp.kb_list || sp.tile_list || sp.group) splits = 1;
    const int kb_per = (kb_total + splits - 1) / splits;
    splits = (kb_total + kb_per - 1) / kb_per;
    const int atomic_out = splits > 1 ? 1 : 0;
    if (atomic_out) {
        zero_rows_kernel<<<152 * 4, 256, 0, s>>>(C, ldc, M, N);
        GVT_LAUNCH_CHECK("tc zero");
    }
    const size_t smem = tc_smem_bytes<BN, PAIR>();
    auto kern = tc_gemm_kernel<BN, F16, PAIR>;
    GVT_CHECK(ensure_smem_attr(reinterpret_cast<const void*>(kern), (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gx, gy, splits);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = PAIR ? 2 : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 1 : 0;
    GVT_CUDA(cudaLaunchKernelEx(&cfg, kern, ma, mb, C, ldc, (int)M, (int)N, kb_total, kb_per, atomic_out, rs, cs,
                                err, stall, sp.kb_list, sp.kb_off, sp.kb_parts, sp.kb_stride,
                                reinterpret_cast<const int2*>(sp.tile_list), sp.group));
    GVT_LAUNCH_CHECK("tc_gemm");
    return GVT_OK;
}

template <bool F16, bool PAIR>
gvt_status launch_tc_bn(int BN, const CUtensorMap& ma, const CUtensorMap& mb, float* C, int64_t ldc, int64_t M,
                        int64_t N, int64_t K, const float* rs, const float* cs, int* err, long long stall,
                        const TcSparse& sp, cudaStream_t s)
{
    if (BN == 64) return launch_tc<64, F16, PAIR>(ma, mb, C, ldc, M, N, K, rs, cs, err, stall, sp, s);
    if (BN == 128) return launch_tc<128, F16, PAIR>(ma, mb, C, ldc, M, N, K, rs, cs, err, stall, sp, s);
    if (BN == 224) return launch_tc<224, F16, PAIR>(ma, mb, C, ldc, M, N, K, rs, cs, err, stall, sp, s);
    return launch_tc<256, F16, PAIR>(ma, mb, C, ldc, M, N, K, rs, cs, err, stall, sp, s);
}

}  // namespace

gvt_status tc_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                   int64_t N, int64_t K, bool f16, const float* row_scale, const float* col_scale, int* err,
                   cudaStream_t s, int pair_mode, long long stall_cycles, const TcSparse* sparse)
{
    const TcSparse sp = sparse ? *sparse : TcSparse{};
    if (M <= 0 || N <= 0) return GVT_OK;
    const bool grouped = sp.group != nullptr;
    if (K <= 0 || K % TC_BK != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K ||
        (!grouped && ldc < N) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || M > INT32_MAX || N > INT32_MAX ||
        K / TC_BK > INT32_MAX) {
        set_error("tc_gemm: K must be a positive multiple of 64, lda/ldb multiples of 8, "
                  "A and B 16-byte aligned");
        return GVT_ERR_INVALID_ARG;
    }
    if (grouped && (sp.kb_list || sp.tile_list || sp.n_tiles > INT32_MAX)) {
        set_error("tc_gemm: grouped tiles take no k-block or tile list, and at most 2^31 - 1 tiles");
        return GVT_ERR_INVALID_ARG;
    }
    if (grouped && sp.n_tiles == 0) return GVT_OK;
    if ((M + TC_BM - 1) / TC_BM > 2147483647ll || (!grouped && (N + 63) / 64 > 65535)) {
        set_error("tc_gemm: matrix too large");
        return GVT_ERR_UNSUPPORTED;
    }
    GVT_CHECK(get_encode());
    // SM pairs only on request: on GB300 both forms reach the same rate on these shapes (the
    // pair form reads 30 % fewer operand bytes per SM, but the loads are not the bound)
    // SM pairs on request, also for a block-sparse B (both CTAs of a pair share the N tile and
    // its k-block list); tile lists and grouped tiles run on one SM
    const bool pair = pair_mode == GVT_TC_PAIRS_ON && !sp.tile_list && !grouped;
    if (sp.kb_list && sp.tile_list) {
        set_error("tc_gemm: a block-sparse B and a tile list cannot be combined");
        return GVT_ERR_INVALID_ARG;
    }
    if (sp.tile_list && sp.n_tiles == 0) return GVT_OK;
    if (stall_cycles > 0 && pair) {
        set_error("tc_gemm: the test stall exists in the one-SM tile form only");
        return GVT_ERR_UNSUPPORTED;
    }
    // widest N tile that still gives >= 64 output tiles (fewer split-K partial sums to reduce);
    // 224 instead of 256 where it fills more of the 152 SMs in the same single wave
    const int64_t gx = (M + TC_BM - 1) / TC_BM;
    int BN = 256;
    while (BN > 64 && gx * ((N + BN - 1) / BN) < 64) BN /= 2;
    if (N <= 64) BN = 64;
    else if (N <= 128 && BN > 128) BN = 128;
    if (BN == 256 && N > 256) {
        const int64_t t256 = gx * ((N + 255) / 256), t224 = gx * ((N + 223) / 224);
        if (t256 < t224 && t224 <= 152) BN = 224;
    }
    if (sp.kb_list || sp.tile_list || grouped) {   // the caller's tiling fixes the N tile
        if (sp.bn != 64 && sp.bn != 128 && sp.bn != 224 && sp.bn != 256) {
            set_error("tc_gemm: sparse forms need an N tile of 64, 128, 224 or 256");
            return GVT_ERR_INVALID_ARG;
        }
        BN = sp.bn;
    }
    CUtensorMap ma, mb;
    GVT_CHECK(make_map(&ma, A, M, K, lda, TC_BM, f16));
    GVT_CHECK(make_map(&mb, B, N, K, ldb, pair ? BN / 2 : BN, f16));
    const float* rs = row_scale;
    const float* cs = col_scale;
    if (f16)
        return pair ? launch_tc_bn<true, true>(BN, ma, mb, C, ldc, M, N, K, rs, cs, err, stall_cycles, sp, s)
                    : launch_tc_bn<true, false>(BN, ma, mb, C, ldc, M, N, K, rs, cs, err, stall_cycles, sp, s);
    return pair ? launch_tc_bn<false, true>(BN, ma, mb, C, ldc, M, N, K, rs, cs, err, stall_cycles, sp, s)
                : launch_tc_bn<false, false>(BN, ma, mb, C, ldc, M, N, K, rs, cs, err, stall_cycles, sp, s);
}

gvt_status tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                        int64_t N, int64_t K, int* err, cudaStream_t s, int pair_mode, long long stall_cycles)
{
    return tc_gemm(A, lda, B, ldb, C, ldc, M, N, K, false, nullptr, nullptr, err, s, pair_mode, stall_cycles);
}

}  // namespace gvt
