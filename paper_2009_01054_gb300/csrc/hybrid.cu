// Per-tile dense/sparse forms of the two GVT stages (Theorem 1) for a Kronecker
// group, built on the host once per plan and configuration.
//
// Theorem 1's cost, O(qbar n + m nhat) per term, is what the sparse SIMT stages
// pay; a dense GEMM over W (or over the whole output grid) pays for every cell
// instead.  With power-law degrees neither fits everywhere: the cells of
// high-degree drugs and targets are nearly all pairs, the rest nearly empty.
// Ids are therefore relabelled by decreasing degree, which gathers the dense
// cells into one corner, and the two operands are cut into tiles:
//  * stage 1: W^T tiles of bn relabelled columns x' by 64 relabelled rows k'
//    (one N tile of the GEMM by one k-block).  A tile with more entries than the
//    break-even count joins the block-sparse GEMM S' = B' W'^T (B' the stage-1
//    factor with its columns relabelled); the entries of the other tiles stay in
//    a compacted order for the sparse scatter-accumulate, which writes S; S' is
//    then added into S through the column relabelling.
//  * stage 2: output tiles of 128 relabelled rows a' by bn relabelled rows s' of
//    S.  Dense tiles go to the tile-list GEMM C' = A' S'^T (A' and S' with their
//    rows relabelled) and their outputs are read out of C'; the other outputs keep
//    the sampled gather-dot.
// The break-even counts and the choice between SIMT, dense and per-tile come from
// a cost model with rates measured on GB300 at the kernel-filling scale (20000 x
// 20000 ids, 10M pairs): the FP16x3 GEMM executes 1.3e15 flop/s; a sparse stage-1
// entry of the per-tile remainder takes its factor row (4 Y bytes, in 1024-row
// slices that stay in L2 during a pass) at about 1.0e13 B/s, and a sampled dot its
// two rows (about 5 X bytes, the A row shared by neighbouring outputs) at about
// 6.2e12 B/s (the remainder's rows belong to low-degree ids and rarely stay in L2).
// On the single pass stage 2's remainder reads the GEMM's FP16 operands instead (half
// the bytes, at the same rate), and the model counts their bytes.  Stage 1's remainder
// stays on FP32 factor rows: its time is set by the entries, not by their bytes
// (measured: FP16 rows made it slower).
#include <algorithm>
#include <numeric>
#include <vector>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr double kTcRate = 1.3e15;        // executed flop/s of the split GEMM
constexpr double kStage1Bw = 1.0e13;      // bytes/s of a sparse stage-1 entry's row stream
constexpr double kStage2Bw = 6.2e12;      // bytes/s of a sampled dot's row streams
constexpr double kPassBw = 4e12;          // split, densify and merge passes
constexpr double kFixed = 8e-6;           // per dense stage (launches, ring fill, epilogue)

template <class T>
gvt_status to_host(std::vector<T>& h, const T* d, int64_t n)
{
    h.resize((size_t)std::max<int64_t>(n, 0));
    if (n > 0) GVT_CUDA(cudaMemcpy(h.data(), d, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost));
    return GVT_OK;
}

template <class T>
gvt_status to_device(gvt_plan* p, const std::vector<T>& h, T** out)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("per-tile stages: device allocation failed");
        return GVT_ERR_ALLOC;
    }
    p->allocs.push_back(q);
    if (!h.empty()) GVT_CUDA(cudaMemcpy(q, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    *out = static_cast<T*>(q);
    return GVT_OK;
}

// ids ordered by decreasing degree (ties by id): perm[rank] = id, rank[id] = rank
void degree_order(const std::vector<int32_t>& seg, std::vector<int32_t>& perm, std::vector<int32_t>& rank)
{
    const int64_t n = (int64_t)seg.size() - 1;
    perm.resize((size_t)n);
    rank.resize((size_t)n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int32_t a, int32_t b) { return seg[a + 1] - seg[a] > seg[b + 1] - seg[b]; });
    for (int64_t r = 0; r < n; ++r) rank[perm[r]] = (int32_t)r;
}

}  // namespace

gvt_status hybrid_stage1(gvt_plan* p, int ia, int ib, int64_t Y, int parts, cudaStream_t s, const HybridS1** out)
{
    for (auto& h : p->hyb1)
        if (h.ia == ia && h.ib == ib && h.Y == Y && h.parts == parts) {
            *out = &h;
            return GVT_OK;
        }
    GVT_CUDA(cudaStreamSynchronize(s));
    HybridS1 H;
    H.ia = ia;
    H.ib = ib;
    H.Y = Y;
    H.parts = parts;
    const Order& ox = p->in_by[ia];
    const Order& ok = p->in_by[ib];
    H.X = ox.K;
    H.K = ok.K;
    const int64_t n = p->n_in;
    std::vector<int32_t> segx, segk, key, bcol, perm;
    GVT_CHECK(to_host(segx, ox.seg, H.X + 1));
    GVT_CHECK(to_host(segk, ok.seg, H.K + 1));
    GVT_CHECK(to_host(key, ox.key, n));
    GVT_CHECK(to_host(bcol, ox.other, n));
    GVT_CHECK(to_host(perm, ox.perm, n));
    std::vector<int32_t> xperm, xrank, kperm, krank;
    degree_order(segx, xperm, xrank);
    degree_order(segk, kperm, krank);
    const int bn = H.bn;
    H.nx = (H.X + bn - 1) / bn;
    H.nk = (H.K + 63) / 64;
    std::vector<int64_t> cnt((size_t)(H.nx * H.nk), 0);
    for (int64_t j = 0; j < n; ++j) cnt[(size_t)((xrank[key[j]] / bn) * H.nk + krank[bcol[j]] / 64)]++;
    // break-even entries of a tile: its GEMM time over the sparse stage's time per entry
    const double kp = (double)((H.K + 63) / 64 * 64);
    const double tile_t = 2.0 * Y * bn * 64.0 * parts / kTcRate;
    const double entry_t = 4.0 * Y / kStage1Bw;
    const double thr = tile_t / entry_t;
    std::vector<uint8_t> dense(cnt.size(), 0);
    std::vector<int32_t> kb_off((size_t)H.nx + 1, 0), kb_list;
    for (int64_t xt = 0; xt < H.nx; ++xt) {
        for (int64_t kb = 0; kb < H.nk; ++kb)
            if ((double)cnt[(size_t)(xt * H.nk + kb)] > thr) {
                dense[(size_t)(xt * H.nk + kb)] = 1;
                kb_list.push_back((int32_t)kb);
                H.n_dense_entries += cnt[(size_t)(xt * H.nk + kb)];
            }
        kb_off[(size_t)xt + 1] = (int32_t)kb_list.size();
    }
    H.n_dense_tiles = (int64_t)kb_list.size();
    // remainder: the entries of sparse tiles, in the same order by x
    std::vector<int32_t> seg_r((size_t)H.X + 1, 0), bcol_r, perm_r;
    bcol_r.reserve((size_t)(n - H.n_dense_entries));
    perm_r.reserve((size_t)(n - H.n_dense_entries));
    for (int64_t j = 0; j < n; ++j) {
        const int32_t x = key[j];
        if (dense[(size_t)((xrank[x] / bn) * H.nk + krank[bcol[j]] / 64)]) continue;
        bcol_r.push_back(bcol[j]);
        perm_r.push_back(perm[j]);
        seg_r[(size_t)x + 1]++;
    }
    for (int64_t x = 0; x < H.X; ++x) seg_r[(size_t)x + 1] += seg_r[(size_t)x];
    H.n_r = (int64_t)bcol_r.size();
    // costs of the three forms (seconds)
    const double split_t = (2.0 * parts * (double)(Y + H.X) * kp + 4.0 * (double)Y * H.K) / kPassBw + kFixed;
    H.cost[0] = (double)n * entry_t;
    H.cost[1] = (double)(H.nx * H.nk) * tile_t + split_t;
    H.cost[2] = (double)H.n_dense_tiles * tile_t + (double)H.n_r * entry_t + split_t +
                12.0 * (double)Y * H.X / kPassBw + 5e-6;
    H.mode = (int)(std::min_element(H.cost, H.cost + 3) - H.cost);
    GVT_CHECK(to_device(p, xperm, &H.xperm));
    GVT_CHECK(to_device(p, xrank, &H.xrank));
    GVT_CHECK(to_device(p, kperm, &H.kperm));
    GVT_CHECK(to_device(p, krank, &H.krank));
    GVT_CHECK(to_device(p, dense, &H.dense));
    GVT_CHECK(to_device(p, kb_off, &H.kb_off));
    GVT_CHECK(to_device(p, kb_list, &H.kb_list));
    GVT_CHECK(to_device(p, seg_r, &H.seg_r));
    GVT_CHECK(to_device(p, bcol_r, &H.bcol_r));
    GVT_CHECK(to_device(p, perm_r, &H.perm_r));
    p->hyb1.push_back(H);
    *out = &p->hyb1.back();
    return GVT_OK;
}

gvt_status hybrid_stage2(gvt_plan* p, int oa, int ob, int64_t X, int parts, int eb, cudaStream_t s,
                         const HybridS2** out)
{
    for (auto& h : p->hyb2)
        if (h.oa == oa && h.ob == ob && h.X == X && h.parts == parts && h.eb == eb) {
            *out = &h;
            return GVT_OK;
        }
    GVT_CUDA(cudaStreamSynchronize(s));
    HybridS2 H;
    H.oa = oa;
    H.ob = ob;
    H.X = X;
    H.parts = parts;
    H.eb = eb;
    const Order& oA = p->out_by[oa];
    const Order& oS = p->out_by[ob];
    H.MA = oA.K;
    H.YS = oS.K;
    const int64_t n = p->n_out;
    std::vector<int32_t> sega, segs, arow, srow, perm;
    GVT_CHECK(to_host(sega, oA.seg, H.MA + 1));
    GVT_CHECK(to_host(segs, oS.seg, H.YS + 1));
    GVT_CHECK(to_host(arow, oA.key, n));
    GVT_CHECK(to_host(srow, oA.other, n));
    GVT_CHECK(to_host(perm, oA.perm, n));
    std::vector<int32_t> aperm, arank, sperm, srank;
    degree_order(sega, aperm, arank);
    degree_order(segs, sperm, srank);
    H.na = (H.MA + H.bm - 1) / H.bm;
    H.nb = (H.YS + H.bn - 1) / H.bn;
    std::vector<int64_t> cnt((size_t)(H.na * H.nb), 0);
    for (int64_t i = 0; i < n; ++i) cnt[(size_t)((arank[arow[i]] / H.bm) * H.nb + srank[srow[i]] / H.bn)]++;
    const double kp = (double)((X + 63) / 64 * 64);
    const double tile_t = 2.0 * H.bm * H.bn * kp * parts / kTcRate;
    const double out_t = 1.25 * eb * X / kStage2Bw;   // the S row and a share of the A row
    const double thr = tile_t / out_t;
    std::vector<uint8_t> dense(cnt.size(), 0);
    std::vector<int32_t> tiles;
    // groups of 16 m tiles, m tile fastest within a group: the CTAs resident at one time share a
    // few A strips and B strips in L2 (the GEMM's own grid order)
    constexpr int64_t kGroupM = 16;
    for (int64_t g0 = 0; g0 < H.na; g0 += kGroupM)
        for (int64_t nt = 0; nt < H.nb; ++nt)
            for (int64_t mt = g0; mt < std::min(H.na, g0 + kGroupM); ++mt)
                if ((double)cnt[(size_t)(mt * H.nb + nt)] > thr) {
                    dense[(size_t)(mt * H.nb + nt)] = 1;
                    tiles.push_back((int32_t)mt);
                    tiles.push_back((int32_t)nt);
                }
    H.n_tiles = (int64_t)tiles.size() / 2;
    std::vector<int32_t> arow_d, srow_d, perm_d, arow_r, srow_r, perm_r, arow_rl, srow_rl;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t a = arank[arow[i]], b = srank[srow[i]];
        if (dense[(size_t)((a / H.bm) * H.nb + b / H.bn)]) {
            arow_d.push_back(a);
            srow_d.push_back(b);
            perm_d.push_back(perm[i]);
        } else {
            arow_r.push_back(arow[i]);
            srow_r.push_back(srow[i]);
            perm_r.push_back(perm[i]);
            arow_rl.push_back(a);
            srow_rl.push_back(b);
        }
    }
    H.n_d = (int64_t)arow_d.size();
    H.n_r = (int64_t)arow_r.size();
    const double split_t = (2.0 * parts * (double)(H.MA + H.YS) * kp) / kPassBw + kFixed;
    H.cost[0] = (double)n * out_t;
    H.cost[1] = (double)(H.na * H.nb) * tile_t + split_t + 4.0 * (double)H.MA * H.YS / kPassBw;
    H.cost[2] = (double)H.n_tiles * tile_t + (double)H.n_r * out_t + split_t + 5e-6;
    H.mode = (int)(std::min_element(H.cost, H.cost + 3) - H.cost);
    GVT_CHECK(to_device(p, aperm, &H.aperm));
    GVT_CHECK(to_device(p, sperm, &H.sperm));
    GVT_CHECK(to_device(p, tiles, &H.tiles));
    GVT_CHECK(to_device(p, arow_d, &H.arow_d));
    GVT_CHECK(to_device(p, srow_d, &H.srow_d));
    GVT_CHECK(to_device(p, perm_d, &H.perm_d));
    GVT_CHECK(to_device(p, arow_r, &H.arow_r));
    GVT_CHECK(to_device(p, srow_r, &H.srow_r));
    GVT_CHECK(to_device(p, perm_r, &H.perm_r));
    GVT_CHECK(to_device(p, arow_rl, &H.arow_rl));
    GVT_CHECK(to_device(p, srow_rl, &H.srow_rl));
    p->hyb2.push_back(H);
    *out = &p->hyb2.back();
    return GVT_OK;
}

}  // namespace gvt
