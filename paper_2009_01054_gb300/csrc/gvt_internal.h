// Internal declarations of the GVT library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gvt.h"

namespace gvt {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
gvt_status cuda_fail(cudaError_t e, const char* what);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device; the
// attribute persists, so each (kernel, device) pays the driver call once.
gvt_status ensure_smem_attr(const void* func, int bytes);

#define GVT_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::gvt::cuda_fail(e_, #call);         \
    } while (0)

#define GVT_CHECK(call)                                                    \
    do {                                                                   \
        gvt_status s_ = (call);                                            \
        if (s_ != GVT_OK) return s_;                                       \
    } while (0)

// Count `n` kernel launches made just before and check their launch status.
void count_launches(int n);
long long gvt_launch_count_internal();
#define GVT_LAUNCHED(n, what)                                              \
    do {                                                                   \
        ::gvt::count_launches(n);                                          \
        GVT_CUDA(cudaGetLastError());                                      \
    } while (0)
#define GVT_LAUNCH_CHECK(what) GVT_LAUNCHED(1, what)

struct StatRec {
    int kind;
    cudaEvent_t e0, e1;
    double flops, bytes, useful;
};

// ---------------------------------------------------------------- device memory
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    gvt_status reserve(size_t nbytes, cudaStream_t s);   // grow-only
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Bump allocator over one growable device buffer: a call lays out its
// temporaries with take(), then commit() grows the buffer if needed.
struct Arena {
    DevBuf buf;
    size_t used = 0;
    void reset() { used = 0; }
    size_t take(size_t bytes) {  // returns offset, 256-byte aligned
        size_t off = (used + 255) & ~size_t(255);
        used = off + bytes;
        return off;
    }
    gvt_status commit(cudaStream_t s) { return buf.reserve(used, s); }
    char* base() const { return static_cast<char*>(buf.ptr); }
};

// A split copy of a kernel matrix kept across products while a solve holds its matrices fixed.
struct FactorCacheEntry {
    const void* ptr = nullptr;
    const int32_t* rowperm = nullptr;   // row and column relabelling of the split (NULL: none)
    const int32_t* colperm = nullptr;
    int64_t ld = 0, rows = 0, K = 0;
    int sq = -1;
    int parts = 3;
    bool f16 = false;
    bool valid = false;
    uint64_t used = 0;
    DevBuf buf;
};
constexpr int kFactorCacheEntries = 4;

}  // namespace gvt

struct gvt_handle {
    gvt::Arena ws;          // per-call workspace (S, transposes, partial sums)
    gvt::Arena solve_ws;    // solver vectors
    gvt::DevBuf status;     // device status words
    double* host_scalars = nullptr;  // pinned
    bool stats_on = false;
    int stage1_engine = 0;          // gvt_stage1_engine for FP32 products
    int tc_pairs = GVT_TC_PAIRS_AUTO;   // gvt_tc_pairs: tile form of the tensor-core GEMM
    long long tc_stall_cycles = 0;      // > 0: test stall of the GEMMs' timeout path (gvt_set_tc_stall_test)
    int stage_tiles = GVT_TILES_AUTO;   // gvt_stage_tiles: per-tile dense/sparse stages
    // a second stream on which a per-tile stage's sparse part runs beside its GEMM (created on first
    // use), with the events that fork it from and join it to the caller's stream
    cudaStream_t aux = nullptr;
    cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
    cudaStream_t cg_stream = nullptr;   // CG iterations (captured into graphs in steady state)
    cudaEvent_t cg_fork = nullptr, cg_join = nullptr;
    std::map<std::tuple<int, int64_t, int>, int> batch_tune;   // batched stage-1 tile choice
    std::vector<gvt::StatRec> recs;
    std::vector<cudaEvent_t> event_pool;
    int factor_cache_depth = 0;     // > 0 while a solve keeps its kernel matrices unchanged
    uint64_t factor_cache_tick = 0;
    gvt::FactorCacheEntry factor_cache[gvt::kFactorCacheEntries];
};

namespace gvt {
// The handle's auxiliary stream, forked from s: work queued on it after this call runs after
// everything queued on s so far.  aux_join(h, s) makes s wait for everything queued on it.
gvt_status aux_fork(gvt_handle* h, cudaStream_t s, cudaStream_t* aux);
gvt_status aux_join(gvt_handle* h, cudaStream_t s);

// While alive, the dense engines reuse split copies of kernel matrices across products (the
// caller guarantees the matrices do not change); the copies are dropped when the last scope ends.
struct FactorCacheScope {
    gvt_handle* h;
    explicit FactorCacheScope(gvt_handle* h_) : h(h_) { ++h->factor_cache_depth; }
    ~FactorCacheScope()
    {
        if (--h->factor_cache_depth == 0)
            for (auto& e : h->factor_cache) e.valid = false;
    }
};
}  // namespace gvt

namespace gvt {
// Bracket one stage launch with events when statistics are on.
struct StatScope {
    gvt_handle* h;
    cudaStream_t s;
    int kind;
    double flops, bytes, useful;
    cudaEvent_t e0 = nullptr;
    // useful < 0: the launch's useful flops are its algorithmic flops
    StatScope(gvt_handle* h_, cudaStream_t s_, int kind_, double flops_, double bytes_, double useful_ = -1.0);
    ~StatScope();
};
}  // namespace gvt

namespace gvt {

// Input or output pairs sorted (stably) by one component.
struct Order {
    int32_t* key = nullptr;    // sorted component values
    int32_t* other = nullptr;  // the other component, same order
    int32_t* perm = nullptr;   // original pair index
    int32_t* seg = nullptr;    // seg[k] = first sorted position with key >= k, k in [0, K]
    int64_t K = 0;             // id range of the key component
};

}  // namespace gvt

namespace gvt {
// Per-tile dense/sparse form of one stage of a Kronecker group (Zipf-like degrees make some tiles of
// W, and of the sampled output grid, dense and most others sparse).  Ids are relabelled by
// decreasing degree so that the dense tiles gather in one corner; dense tiles run on the
// tensor-core GEMM, the rest on the SIMT stages.  Built on the host once per plan and
// configuration; device arrays live in the plan's allocations.
struct HybridS1 {                   // stage 1: S = B W with W's columns x, rows k
    int ia = -1, ib = -1, parts = 0;
    int64_t X = 0, K = 0, Y = 0;
    int bn = 256;                   // x tile (the GEMM's N tile); k blocks are 64 wide
    int64_t nx = 0, nk = 0;
    int32_t* xperm = nullptr;       // x' -> x
    int32_t* xrank = nullptr;       // x -> x'
    int32_t* kperm = nullptr;       // k' -> k
    int32_t* krank = nullptr;       // k -> k'
    uint8_t* dense = nullptr;       // nx * nk tile flags
    int32_t* kb_off = nullptr;      // nx + 1 offsets into kb_list
    int32_t* kb_list = nullptr;     // dense k blocks of every x tile
    int32_t *seg_r = nullptr, *bcol_r = nullptr, *perm_r = nullptr;   // remainder entries, by x
    int64_t n_r = 0, n_dense_tiles = 0, n_dense_entries = 0;
    int mode = 0;                   // 0: SIMT, 1: dense GEMM, 2: per tile
    double cost[3] = {0, 0, 0};
};
struct HybridS2 {                   // stage 2: u_i = <A[a_i, :], S[s_i, :]> over the output pairs
    int oa = -1, ob = -1, parts = 0, eb = 4;
    int64_t MA = 0, YS = 0, X = 0;
    int bm = 128, bn = 256;         // output tile of the GEMM C' = A' S'^T
    int64_t na = 0, nb = 0;
    int32_t* aperm = nullptr;       // a' -> a
    int32_t* sperm = nullptr;       // s' -> s
    int32_t* tiles = nullptr;       // dense output tiles, (m tile, n tile) pairs
    int64_t n_tiles = 0;
    int32_t *arow_d = nullptr, *srow_d = nullptr, *perm_d = nullptr;  // outputs in dense tiles, relabelled
    int64_t n_d = 0;
    int32_t *arow_r = nullptr, *srow_r = nullptr, *perm_r = nullptr;  // remainder outputs, by a
    int32_t *arow_rl = nullptr, *srow_rl = nullptr;   // the remainder's rows relabelled (a', s')
    int64_t n_r = 0;
    int mode = 0;
    double cost[3] = {0, 0, 0};
};
}  // namespace gvt

struct gvt_plan {
    gvt_handle* h = nullptr;
    int64_t m_rows = 0, m_cols = 0, q_rows = 0, q_cols = 0;
    int64_t n_in = 0, n_out = 0;
    bool out_is_in = false;
    int32_t* d_in = nullptr;
    int32_t* t_in = nullptr;
    int32_t* d_out = nullptr;
    int32_t* t_out = nullptr;
    gvt::Order in_by[2];    // [FIRST], [SECOND]
    gvt::Order out_by[2];
    std::vector<void*> allocs;
    std::deque<gvt::HybridS1> hyb1;    // per-tile forms built so far (a deque: references stay valid)
    std::deque<gvt::HybridS2> hyb2;
};

namespace gvt {

// ---------------------------------------------------------------- sort / scan
// Workspace bytes needed by radix_sort_by_key for n elements.
size_t sort_workspace_bytes(int64_t n);
// Stable sort of `keys` (values in [0, K)) carrying the original index.
// out_key / out_perm: n each.  ws: sort_workspace_bytes(n) bytes.
gvt_status radix_sort_by_key(const int32_t* keys, int64_t n, int64_t K, int32_t* out_key,
                             int32_t* out_perm, void* ws, cudaStream_t s);
// seg[k] = lower_bound(sorted_key, k), k in [0, K].
gvt_status segment_offsets(const int32_t* sorted_key, int64_t n, int64_t K, int32_t* seg,
                           cudaStream_t s);
// out[i] = in[perm[i]]
gvt_status gather_i32(const int32_t* in, const int32_t* perm, int64_t n, int32_t* out,
                      cudaStream_t s);
// min and max of an int32 array into dev_minmax[0..1] (int32); n > 0.
gvt_status minmax_i32(const int32_t* x, int64_t n, int32_t* dev_minmax, cudaStream_t s);

// ---------------------------------------------------------------- stage kernels
enum FactorMode { FM_DENSE = 0, FM_SQUARE = 1 };

// One source of stage-1 entries: the input pairs in one sorted order.
// Entry j of column x (j in [seg[x], seg[x+1])) contributes coef*v[perm[j]] at
// row bcol[j] of W.
struct S1Source {
    const int32_t* seg;
    const int32_t* bcol;
    const int32_t* perm;
    double coef;
    int same;   // bcol is the segment key itself: every entry of segment x lands in cell (x, x)
};
constexpr int kMaxSources = 4;
struct S1Sources {
    S1Source src[kMaxSources];
    int count;
};

// S[y, x] = sum_src coef * sum_{j in seg_src[x]} Bt[bcol_j, y] * v[perm_j]   (y < Y, x < X)
// Bt is B transposed: Bt[t*ldb + y] = B[y, t].  mode squares B's entries.
template <class T>
gvt_status stage1_sparse(const T* Bt, int64_t ldb, int mode, const S1Sources& srcs, const T* v,
                        T* S, int64_t lds, int64_t Y, int64_t X, cudaStream_t s);
// B = identity: S[y, x] = sum_src coef * sum_{j in seg_src[x], bcol_j == y} v[perm_j]
// (S must be zeroed by the caller; entries with bcol >= Y are skipped).
template <class T>
gvt_status stage1_identity(const S1Sources& srcs, const T* v, T* S, int64_t lds, int64_t Y,
                           int64_t X, cudaStream_t s);

// Output pairs in one sorted order: row of A = arow[i], row of S = srow[i],
// destination u[perm[i]].
struct S2Outputs {
    const int32_t* arow;
    const int32_t* srow;
    const int32_t* perm;
    int64_t n;
};
// u[perm_i] += coef * sum_{x < X} A[arow_i, x] * S[srow_i, x]
template <class T>
gvt_status stage2_gather(const T* A, int64_t lda, int mode, const T* S, int64_t lds, int64_t X,
                        const S2Outputs& outs, double coef, T* u, cudaStream_t s);
// The same over FP16 rows of A and S scaled by powers of two (inverses ascale, sscale per row),
// dots accumulated in FP32; X, lda and lds multiples of 8, both bases 16-byte aligned.
gvt_status stage2_gather_f16(const void* A, int64_t lda, const float* ascale, const void* S, int64_t lds,
                             const float* sscale, int64_t X, const S2Outputs& outs, double coef, float* u,
                             cudaStream_t s);
// u[perm_i] += C[arow_i, srow_i] (the dense stage 2's sampled read-out)
gvt_status dense_gather(const float* C, int64_t ldc, const S2Outputs& outs, float* u, cudaStream_t s);
// A = identity: u[perm_i] += coef * S[srow_i, arow_i] (arow_i < X)
template <class T>
gvt_status stage2_identity(const T* S, int64_t lds, int64_t X, const S2Outputs& outs, double coef,
                           T* u, cudaStream_t s);

// One-sided terms (a factor is the all-ones operator).
// s[x] += coef * sum_{j in seg[x]} v[perm_j]   for x < K
template <class T>
gvt_status segment_sums(const int32_t* seg, const int32_t* perm, int64_t K, const T* v, double coef,
                        T* s_out, cudaStream_t s);
// One-sided groups on the same factor share one pass over it (up to kMaxOneSidedShare):
// z[g*ldz + r] = sum_{x < X} F[r, x] * svecs[g*lds + x], and u[i] += sum_g z_g[idx_g[i]].
constexpr int kMaxOneSidedShare = 4;
template <class T>
gvt_status gemv_rows_multi(const T* F, int64_t ldf, int mode, int64_t R, int64_t X, const T* svecs, int64_t lds,
                           int count, T* z, int64_t ldz, cudaStream_t s);
template <class T>
gvt_status gather_add_multi(const T* const* z, const int32_t* const* idx, int count, int64_t n, T* u,
                            cudaStream_t s);

// Bt[c*ldt + r] = B[r*ldb + c]
template <class T>
gvt_status transpose(const T* B, int64_t ldb, int64_t rows, int64_t cols, T* Bt, int64_t ldt,
                     cudaStream_t s);

gvt_status convert(const void* src, int sdt, void* dst, int ddt, int64_t n, cudaStream_t s);
gvt_status linear_kernel(const double* X, int64_t rx, const double* Y, int64_t ry, int64_t dim, void* K,
                         int64_t ldk, int dtype, cudaStream_t s);
gvt_status tanimoto_kernel(const uint32_t* X, int64_t rx, const uint32_t* Y, int64_t ry, int64_t words, void* K,
                           int64_t ldk, int dtype, cudaStream_t s);
gvt_status gaussian_kernel(const double* X, int64_t rx, const double* Y, int64_t ry, int64_t dim,
                           double gamma, void* K, int64_t ldk, int dtype, cudaStream_t s);

size_t dtype_size(int dt);

// ---------------------------------------------------------------- tensor-core stage 1
// Device error word of a handle (bounded waits in tensor-core kernels report here).
inline int* handle_err_word(gvt_handle* h) { return static_cast<int*>(h->status.ptr) + 16; }
// C[M x N] = row_scale[m] col_scale[n] (A B^T)[m, n] on the tensor cores; A, B both FP16 (f16) or
// both BF16, K-major; the scales may be NULL; pair_mode is a gvt_tc_pairs value.
// Sparse forms of the tensor-core GEMM (device arrays; one SM per tile, no split K):
//  * block-sparse B: the CTA of N tile j (bn columns) runs over the k-blocks
//    kb_list[kb_off[j] .. kb_off[j+1]) of each of the kb_parts K segments (kb_stride
//    k-blocks apart); an N tile with an empty list stores zeros;
//  * tile list: only the n_tiles output tiles tile_list[2b], tile_list[2b+1] = (m tile, n tile).
// One output tile of a grouped launch: rows a_row.. of A and b_row.. of B (128 and bn of them;
// rows past m_valid / n_valid are computed but not stored) over k-blocks 0 .. nkb-1, stored at
// C + c_off with row stride ldc; row and column scales indexed by A and B row.
struct TcGroupTile {
    int32_t a_row, b_row, nkb, m_valid, n_valid, pad;
    int64_t c_off, ldc;
};
struct TcSparse {
    const int* kb_list = nullptr;
    const int* kb_off = nullptr;
    int kb_parts = 1;
    int kb_stride = 0;
    const int* tile_list = nullptr;
    int64_t n_tiles = 0;
    int bn = 256;
    const TcGroupTile* group = nullptr;   // grouped tiles (n_tiles of them), instead of the lists
};
// stall_cycles > 0 (one-SM form only): the test stall of the timeout path (the GEMM's MMA thread
// waits that many cycles on a barrier nothing arrives on; the result is then invalid).
gvt_status tc_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                   int64_t N, int64_t K, bool f16, const float* row_scale, const float* col_scale, int* err,
                   cudaStream_t s, int pair_mode, long long stall_cycles = 0, const TcSparse* sparse = nullptr);
// C[M x N] (FP32, ld ldc) = A[M x K] B[N x K]^T, A and B BF16 K-major (K % 64 == 0).
gvt_status tc_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                        int64_t N, int64_t K, int* err, cudaStream_t s, int pair_mode, long long stall_cycles = 0);

// A split operand of the dense stages: rows x (parts * kp) 16-bit values ([hi|hi|lo] or
// [hi|lo|hi] when parts == 3, [hi] when parts == 1), and for FP16 splits the inverse
// power-of-two scale of every row.
struct DenseOperand {
    void* data = nullptr;
    float* inv_scale = nullptr;
    int64_t rows = 0;
    int64_t kp = 0;   // K rounded up to 64
    int parts = 3;
};
int64_t dense_kp(int64_t K);
size_t dense_operand_bytes(int64_t rows, int64_t K, int parts);
DenseOperand dense_operand_at(void* base, int64_t rows, int64_t K, int parts);
size_t dense_w_scratch_bytes(int64_t X, int64_t K);
// rows of a row-major FP32 matrix (entries squared if `square`), pattern_b: [hi|lo|hi] instead of [hi|hi|lo];
// row r taken from source row rowperm[r] and entry k from column colperm[k] when given
gvt_status dense_split_rows(const float* src, int64_t ld, int64_t rows, int64_t cols, int square, bool f16,
                            int pattern_b, const DenseOperand& dst, cudaStream_t s, const int32_t* rowperm = nullptr,
                            const int32_t* colperm = nullptr);
// W^T in relabelled rows x' (original column xperm[x']) holding only the entries of one source that
// fall in dense tiles (dense[(x' / bn) * nk + krank[bcol] / 64] != 0), at column krank[bcol], split
gvt_status dense_densify_tiles(const S1Source& src, const int32_t* xperm, const int32_t* krank, const uint8_t* dense,
                               int bn, int64_t nk, const float* v, int64_t X, bool f16, const DenseOperand& dst,
                               cudaStream_t s);
// S[y, x] += Sd[y, xrank[x]]
gvt_status dense_merge_cols(float* S, int64_t lds, const float* Sd, int64_t ldsd, const int32_t* xrank, int64_t Y,
                            int64_t X, cudaStream_t s);
// The merge followed by dense_split_rows of S (rows rowperm[r], all X columns) in one pass: S is
// merged in place and split into dst.  Only for rows that fit (dense_merge_split_fits).
bool dense_merge_split_fits(int64_t X);
gvt_status dense_merge_split(float* S, int64_t lds, const float* Sd, int64_t ldsd, const int32_t* xrank, int64_t Y,
                             int64_t X, bool f16, int pattern_b, const DenseOperand& dst, cudaStream_t s,
                             const int32_t* rowperm);
// W^T (X rows, [hi|lo|hi]) from the sources of a stage-1 group (keys[si][j] = column x of entry j)
gvt_status dense_split_w(const S1Sources& srcs, const int32_t* const keys[kMaxSources], int64_t n, const float* v,
                         int64_t X, bool f16, const DenseOperand& dst, float* wide_scratch, cudaStream_t s);
// C[a.rows x b.rows] = a b^T with the FP16 row scales applied
gvt_status dense_gemm(const DenseOperand& a, const DenseOperand& b, bool f16, float* C, int64_t ldc, int* err,
                      cudaStream_t s, int pair_mode, long long stall_cycles = 0, const TcSparse* sparse = nullptr);

// ---------------------------------------------------------------- per-tile dense/sparse stages
// The per-tile form of stage 1 (x component ia, inner component ib, Y rows of S) or of stage 2
// (A rows component oa, S rows component ob, inner length X) for `parts` 16-bit GEMM parts, with
// the mode the cost model picks; built on first use and kept in the plan.  Stage 2's sparse
// remainder reads `eb` bytes per row entry (4: FP32; 2: the FP16 operands of the single pass).
gvt_status hybrid_stage1(gvt_plan* p, int ia, int ib, int64_t Y, int parts, cudaStream_t s, const HybridS1** out);
gvt_status hybrid_stage2(gvt_plan* p, int oa, int ob, int64_t X, int parts, int eb, cudaStream_t s,
                         const HybridS2** out);

// ---------------------------------------------------------------- pairwise driver
// u = R_out K_desc R_in^T v for one column (all pointers device; T = float/double).
template <class T>
gvt_status pairwise_apply(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                          const gvt_matrix* N, const T* v, T* u, cudaStream_t s);

// ---------------------------------------------------------------- learned preconditioner
template <class T>
gvt_status precond_apply(gvt_precond* p, const T* r, T* z, cudaStream_t s);
int64_t precond_size(const gvt_precond* p);

// ---------------------------------------------------------------- vector kernels (CG)
template <class T>
gvt_status vec_zero(T* x, int64_t n, cudaStream_t s);

}  // namespace gvt

namespace gvt {
// ---------------------------------------------------------------- host-driven Krylov solvers
// (MINRES, multi-shift CG, the logistic Newton solver): dot products reduce to one partial
// sum per block, which the host adds in a fixed order, so runs are reproducible.
constexpr int kRedGrid = 512;      // blocks of a reduction launch
constexpr int kRedBlock = 256;     // threads per block

#ifdef __CUDACC__
// block sum of v into part[slot * gridDim.x + blockIdx.x]; may be called twice in a row
__device__ __forceinline__ void block_sum_slot(double v, double* __restrict__ part, int slot)
{
    __shared__ double sh[kRedBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kRedBlock / 32; ++i) t += sh[i];
        part[(int64_t)slot * gridDim.x + blockIdx.x] = t;
    }
}
#endif

// out[k] = the fixed-order sum of slot k's kRedGrid partials (k < slots); synchronises s
gvt_status host_reduce(const double* part_dev, int slots, std::vector<double>& host, double* out, cudaStream_t s);
}  // namespace gvt
