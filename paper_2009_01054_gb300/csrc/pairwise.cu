// Pairwise kernel matrix-vector products as sums of Kronecker terms
// (Corollary 1), each term evaluated with the two stages of the generalized
// vec trick (Theorem 1).
//
// A descriptor is compiled on the host into
//   * two-sided groups: terms with the same (A, B, out_a, out_b) share one
//     stage 2; their input recipes (in_a, in_b, coef) are summed into one
//     sparse W, so one stage 1 serves them (W is linear in v).  Groups whose
//     B factor and recipe coincide share S.
//   * one-sided groups (one factor is the all-ones operator 1):
//     u_i += (F s)[o(i)] with s the coefficient-weighted segment sums of v.
// The stage ordering of every dense x dense term is the cheaper of the two
// orderings of Theorem 1, min(qbar*n + m*nhat, mbar*n + q*nhat).
#include <algorithm>
#include <map>
#include <tuple>

#include "gvt_internal.h"

namespace gvt {
namespace {

bool is_dense(int f) { return f == GVT_FACTOR_M || f == GVT_FACTOR_N || f == GVT_FACTOR_M_SQ || f == GVT_FACTOR_N_SQ; }
int sq_mode(int f) { return (f == GVT_FACTOR_M_SQ || f == GVT_FACTOR_N_SQ) ? FM_SQUARE : FM_DENSE; }
// 0 = M, 1 = N
int base_matrix(int f, bool homogeneous)
{
    if (homogeneous) return 0;
    return (f == GVT_FACTOR_N || f == GVT_FACTOR_N_SQ) ? 1 : 0;
}

struct TwoSided {
    int fa, fb, oa, ob;
    std::map<std::pair<int, int>, double> recipe;   // (in_a, in_b) -> coef
};
struct OneSided {
    int f, oc;
    std::map<int, double> sources;                    // in comp -> coef
};

struct Compiled {
    std::vector<TwoSided> two;
    std::vector<OneSided> one;
};

// Engine choice of GVT_STAGES_AUTO (parts = 3) and GVT_STAGES_TC_F16X1 (parts = 1) for one
// stage: the dense GEMM over `parts` 16-bit parts (rows x cols outputs, inner length K) against
// the sparse SIMT stage doing simt_flops useful flops.  Rates measured on GB300 at m = q = 2000
// over pair densities 0.2 % to 20 %: SIMT stages about 4.5e12 useful flop/s, the split GEMM
// about 1.2e15 flop/s, the split and densify passes about 4e12 B/s, and about 8 us of fixed cost
// per dense stage (a dense stage measured 66 us there, the SIMT stage 74 us at 2 % density; for
// one Kronecker term the model switches at 1.8 % with three parts).
bool dense_pays(int64_t rows, int64_t cols, int64_t K, double simt_flops, int parts)
{
    const double kp = (double)dense_kp(K);
    const double t_dense = 2.0 * parts * rows * cols * kp / 1.2e15 +
                           (2.0 * parts * (double)(rows + cols) * kp + 4.0 * (double)rows * cols) / 4e12 + 8e-6;
    return t_dense < simt_flops / 4.5e12;
}

// Pairs below which the automatic engines keep the per-stage choice: the per-tile form's one-time
// host build (a sort of the ids by degree, a pass over the pairs) pays off on large samples.
constexpr int64_t kTilesMinPairs = int64_t(1) << 20;

int64_t out_range(const gvt_plan* p, int c) { return c == GVT_FIRST ? p->m_rows : p->q_rows; }
int64_t in_range(const gvt_plan* p, int c) { return c == GVT_FIRST ? p->m_cols : p->q_cols; }

gvt_status compile(const gvt_plan* p, const gvt_desc* d, const gvt_matrix* mats[2], bool tc, Compiled& out)
{
    if (d->n_terms < 1 || d->n_terms > GVT_MAX_TERMS) {
        set_error("descriptor: n_terms out of range");
        return GVT_ERR_INVALID_ARG;
    }
    const bool homo = d->homogeneous != 0;
    std::map<std::tuple<int, int, int, int>, size_t> two_idx;
    std::map<std::pair<int, int>, size_t> one_idx;
    for (int k = 0; k < d->n_terms; ++k) {
        gvt_term t = d->terms[k];
        auto comp_ok = [](int c) { return c == GVT_FIRST || c == GVT_SECOND; };
        if (t.factor_a < 0 || t.factor_a > GVT_FACTOR_IDENTITY || t.factor_b < 0 ||
            t.factor_b > GVT_FACTOR_IDENTITY || !comp_ok(t.out_a) || !comp_ok(t.out_b) ||
            !comp_ok(t.in_a) || !comp_ok(t.in_b)) {
            set_error("descriptor: bad factor or component in term " + std::to_string(k));
            return GVT_ERR_INVALID_ARG;
        }
        if (t.coef == 0.0) continue;
        const bool a1 = t.factor_a == GVT_FACTOR_ONES, b1 = t.factor_b == GVT_FACTOR_ONES;
        if (a1 && b1) {
            set_error("descriptor: a term with two all-ones factors is not supported");
            return GVT_ERR_UNSUPPORTED;
        }
        if (a1 || b1) {
            const int f = a1 ? t.factor_b : t.factor_a;
            const int oc = a1 ? t.out_b : t.out_a;
            const int ic = a1 ? t.in_b : t.in_a;
            if (!is_dense(f)) {
                set_error("descriptor: ones x identity terms are not supported");
                return GVT_ERR_UNSUPPORTED;
            }
            const gvt_matrix* F = mats[base_matrix(f, homo)];
            if (F->rows < out_range(p, oc) || F->cols < in_range(p, ic)) {
                set_error("descriptor: kernel matrix smaller than the id range of a one-sided term");
                return GVT_ERR_INVALID_ARG;
            }
            auto key = std::make_pair(f, oc);
            auto it = one_idx.find(key);
            if (it == one_idx.end()) {
                one_idx[key] = out.one.size();
                out.one.push_back(OneSided{f, oc, {}});
                it = one_idx.find(key);
            }
            out.one[it->second].sources[ic] += t.coef;
            continue;
        }
        if (t.factor_a == GVT_FACTOR_IDENTITY && t.factor_b == GVT_FACTOR_IDENTITY) {
            set_error("descriptor: identity x identity terms are not supported");
            return GVT_ERR_UNSUPPORTED;
        }
        // Ordering choice of Theorem 1 for dense x dense terms: swap the roles of
        // the two factors when mbar*n + q*nhat < qbar*n + m*nhat.
        if (is_dense(t.factor_a) && is_dense(t.factor_b)) {
            const gvt_matrix* A = mats[base_matrix(t.factor_a, homo)];
            const gvt_matrix* B = mats[base_matrix(t.factor_b, homo)];
            double c1 = (double)out_range(p, t.out_b) * p->n_in + (double)in_range(p, t.in_a) * p->n_out;
            double c2 = (double)out_range(p, t.out_a) * p->n_in + (double)in_range(p, t.in_b) * p->n_out;
            if (tc) {   // stage 1 on tensor cores is cheap: minimise the stage-2 length instead
                c1 = (double)in_range(p, t.in_a) * p->n_out;
                c2 = (double)in_range(p, t.in_b) * p->n_out;
            }
            (void)A; (void)B;
            if (c2 < c1) {
                std::swap(t.factor_a, t.factor_b);
                std::swap(t.out_a, t.out_b);
                std::swap(t.in_a, t.in_b);
            }
        }
        if (is_dense(t.factor_a)) {
            const gvt_matrix* A = mats[base_matrix(t.factor_a, homo)];
            if (A->rows < out_range(p, t.out_a) || A->cols < in_range(p, t.in_a)) {
                set_error("descriptor: left factor smaller than its id ranges");
                return GVT_ERR_INVALID_ARG;
            }
        }
        if (is_dense(t.factor_b)) {
            const gvt_matrix* B = mats[base_matrix(t.factor_b, homo)];
            if (B->rows < out_range(p, t.out_b) || B->cols < in_range(p, t.in_b)) {
                set_error("descriptor: right factor smaller than its id ranges");
                return GVT_ERR_INVALID_ARG;
            }
        }
        auto key = std::make_tuple(t.factor_a, t.factor_b, t.out_a, t.out_b);
        auto it = two_idx.find(key);
        if (it == two_idx.end()) {
            two_idx[key] = out.two.size();
            out.two.push_back(TwoSided{t.factor_a, t.factor_b, t.out_a, t.out_b, {}});
            it = two_idx.find(key);
        }
        out.two[it->second].recipe[{t.in_a, t.in_b}] += t.coef;
    }
    for (auto& g : out.two) {
        if (g.recipe.size() > (size_t)kMaxSources) {
            set_error("descriptor: more than 4 index recipes in one group");
            return GVT_ERR_UNSUPPORTED;
        }
        int64_t X = -1;
        for (auto& r : g.recipe) {
            const int64_t K = in_range(p, r.first.first);
            if (X >= 0 && K != X) {
                set_error("descriptor: merged terms have different column id ranges");
                return GVT_ERR_UNSUPPORTED;
            }
            X = K;
        }
    }
    return GVT_OK;
}

template <class T>
struct FactorView {
    const T* A = nullptr;   // row-major factor
    int64_t lda = 0;
    const T* Bt = nullptr;  // transposed factor for stage 1
    int64_t ldbt = 0;
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

template <class T>
gvt_status pairwise_apply(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                          const gvt_matrix* N, const T* v, T* u, cudaStream_t s)
{
    const bool homo = desc->homogeneous != 0;
    const gvt_matrix* mats[2] = {M, homo ? M : N};
    gvt_handle* h = plan->h;
    // engine of the dense x dense groups of FP32 products (FP64 products always run the SIMT stages)
    const int engine = sizeof(T) == 4 ? h->stage1_engine : (int)GVT_STAGE1_SIMT;
    const bool f16 = engine == GVT_STAGES_TC_F16X3 || engine == GVT_STAGES_AUTO || engine == GVT_STAGES_TC_F16X1;
    // 16-bit parts of every dense operand: the hi/lo split (three GEMM passes) or hi alone
    const int parts = engine == GVT_STAGES_TC_F16X1 ? 1 : 3;
    const bool chooses = engine == GVT_STAGES_AUTO || engine == GVT_STAGES_TC_F16X1;   // per-stage cost model
    Compiled C;
    GVT_CHECK(compile(plan, desc, mats, engine == GVT_STAGE1_TC_BF16X3, C));

    const int64_t n_out = plan->n_out;

    // ---- workspace layout
    Arena& ws = h->ws;
    ws.reset();
    size_t off_t[2] = {SIZE_MAX, SIZE_MAX};
    int64_t ldt[2] = {0, 0};
    bool need_t[2] = {false, false};
    for (auto& g : C.two)
        if (is_dense(g.fb)) need_t[base_matrix(g.fb, homo)] = true;
    for (int b = 0; b < 2; ++b) {
        if (!need_t[b]) continue;
        const gvt_matrix* B = mats[b];
        if (B->symmetric && B->rows == B->cols) continue;
        ldt[b] = round_up(B->rows, 4);
        off_t[b] = ws.take(sizeof(T) * (size_t)ldt[b] * (size_t)B->cols);
    }
    int64_t s_elems = 0;
    for (auto& g : C.two) {
        const int64_t X = in_range(plan, g.recipe.begin()->first.first);
        const int64_t Y = is_dense(g.fb) ? out_range(plan, g.ob) : out_range(plan, g.ob);
        s_elems = std::max(s_elems, Y * round_up(X, 4));
    }
    const size_t off_S = s_elems > 0 ? ws.take(sizeof(T) * (size_t)s_elems) : 0;
    int64_t one_elems = 0;
    for (auto& g : C.one) {
        const gvt_matrix* F = mats[base_matrix(g.f, homo)];
        one_elems = std::max(one_elems, kMaxOneSidedShare * (F->cols + F->rows));
    }
    const size_t off_one = one_elems > 0 ? ws.take(sizeof(T) * (size_t)one_elems) : 0;
    // ---- dense-stage decisions (same grouping as the execution loop below) and their workspace
    // 0: SIMT, 1: dense GEMM, 2: per tile (dense tiles on the GEMM, the rest SIMT)
    std::vector<char> tc1(C.two.size(), 0), tc2(C.two.size(), 0);
    size_t slot_bytes = 0, w_bytes = 0, s_bytes = 0, c_bytes = 0, wide_bytes = 0;
    int64_t sd_elems = 0;   // S' of a per-tile stage 1 (its dense part, relabelled columns)
    // per-tile forms: the cost-model engines on large samples, or on request
    const bool tiles_ok = chooses && sizeof(T) == 4 && h->stage_tiles != GVT_TILES_OFF &&
                          (h->stage_tiles == GVT_TILES_ON || std::min(plan->n_in, n_out) >= kTilesMinPairs);
    if (engine != GVT_STAGE1_SIMT) {
        std::vector<bool> seen(C.two.size(), false);
        for (size_t gi = 0; gi < C.two.size(); ++gi) {
            if (seen[gi]) continue;
            const TwoSided& g = C.two[gi];
            const int64_t X = in_range(plan, g.recipe.begin()->first.first);
            const int64_t Y = out_range(plan, g.ob);
            const int ib = g.recipe.begin()->first.second;
            bool same_ib = true;
            for (auto& r : g.recipe) same_ib = same_ib && in_range(plan, r.first.second) == in_range(plan, ib);
            const int64_t K = in_range(plan, ib);
            if (is_dense(g.fb) && same_ib && Y > 0 && X > 0 && K > 0) {   // stage 1 needs a dense B only
                const double entries = (double)g.recipe.size() * plan->n_in;
                tc1[gi] = chooses ? dense_pays(Y, X, K, 2.0 * Y * entries, parts) : 1;
                const int ia = g.recipe.begin()->first.first;
                if (tiles_ok && g.recipe.size() == 1 && ia != ib && 4 * dense_kp(K) <= 160 * 1024) {
                    const HybridS1* h1 = nullptr;
                    GVT_CHECK(hybrid_stage1(plan, ia, ib, Y, parts, s, &h1));
                    tc1[gi] = h->stage_tiles == GVT_TILES_ON ? 2 : (char)h1->mode;
                }
            }
            if (tc1[gi]) {
                slot_bytes = std::max(slot_bytes, dense_operand_bytes(Y, K, parts));
                w_bytes = std::max(w_bytes, dense_operand_bytes(X, K, parts));
                wide_bytes = std::max(wide_bytes, dense_w_scratch_bytes(X, K));
            }
            if (tc1[gi] == 2) sd_elems = std::max(sd_elems, Y * round_up(X, 4));
            for (size_t gj = gi; gj < C.two.size(); ++gj) {
                const TwoSided& g2 = C.two[gj];
                if (seen[gj] || g2.fb != g.fb || g2.recipe != g.recipe || out_range(plan, g2.ob) != Y) continue;
                seen[gj] = true;
                const int64_t mb = out_range(plan, g2.oa);
                if (!f16 || !is_dense(g2.fa) || mb <= 0) continue;
                tc2[gj] = chooses ? dense_pays(mb, Y, X, 2.0 * X * (double)n_out, parts) : 1;
                if (tiles_ok && g2.oa != g2.ob) {
                    const HybridS2* h2 = nullptr;
                    GVT_CHECK(hybrid_stage2(plan, g2.oa, g2.ob, X, parts, parts == 1 ? 2 : 4, s, &h2));
                    tc2[gj] = h->stage_tiles == GVT_TILES_ON ? 2 : (char)h2->mode;
                }
                if (!tc2[gj]) continue;
                slot_bytes = std::max(slot_bytes, dense_operand_bytes(mb, X, parts));
                s_bytes = std::max(s_bytes, dense_operand_bytes(Y, X, parts));
                c_bytes = std::max(c_bytes, sizeof(float) * (size_t)mb * (size_t)round_up(Y, 4));
            }
        }
    }
    const size_t off_slot0 = slot_bytes ? ws.take(slot_bytes) : 0;
    const size_t off_slot1 = slot_bytes ? ws.take(slot_bytes) : 0;
    const size_t off_w = w_bytes ? ws.take(w_bytes) : 0;
    const size_t off_s2 = s_bytes ? ws.take(s_bytes) : 0;
    const size_t off_c2 = c_bytes ? ws.take(c_bytes) : 0;
    const size_t off_wide = wide_bytes ? ws.take(wide_bytes) : 0;
    const size_t off_sd = sd_elems ? ws.take(sizeof(T) * (size_t)sd_elems) : 0;
    GVT_CHECK(ws.commit(s));
    char* base = ws.base();

    FactorView<T> fv[2];
    for (int b = 0; b < 2; ++b) {
        const gvt_matrix* F = mats[b];
        if (!F || !F->data) continue;
        fv[b].A = static_cast<const T*>(F->data);
        fv[b].lda = F->ld;
        if (need_t[b]) {
            if (off_t[b] == SIZE_MAX) {
                fv[b].Bt = fv[b].A;
                fv[b].ldbt = F->ld;
            } else {
                T* Bt = reinterpret_cast<T*>(base + off_t[b]);
                GVT_CHECK(transpose<T>(fv[b].A, F->ld, F->rows, F->cols, Bt, ldt[b], s));
                fv[b].Bt = Bt;
                fv[b].ldbt = ldt[b];
            }
        }
    }

    GVT_CHECK(vec_zero<T>(u, n_out, s));

    // ---- two-sided groups, grouped by shared stage 1
    std::vector<bool> done(C.two.size(), false);
    // Split factors live in two slots; a split stays valid for later groups (and for
    // stage 2) that need the same factor, square mode, extents and format.
    struct Slot {
        const void* ptr = nullptr;
        const int32_t* rowperm = nullptr;
        const int32_t* colperm = nullptr;
        int sq = -1, pattern = -1;
        int64_t rows = -1, K = -1;
        size_t off = 0;
        int64_t used = -1;
    } slots[2];   // (the parts count is fixed for the whole call)
    slots[0].off = off_slot0;
    slots[1].off = off_slot1;
    int64_t tick = 0;
    auto factor_operand = [&](const gvt_matrix* F, int sq, int64_t rows, int64_t K, DenseOperand& out,
                              const int32_t* rowperm = nullptr, const int32_t* colperm = nullptr) -> gvt_status {
        if (h->factor_cache_depth > 0) {   // a solve holds the matrices fixed: keep splits across products
            for (auto& e : h->factor_cache)
                if (e.valid && e.ptr == F->data && e.ld == F->ld && e.rows == rows && e.K == K && e.sq == sq &&
                    e.f16 == f16 && e.parts == parts && e.rowperm == rowperm && e.colperm == colperm) {
                    e.used = ++h->factor_cache_tick;
                    out = dense_operand_at(e.buf.ptr, rows, K, parts);
                    return GVT_OK;
                }
            FactorCacheEntry* lru = &h->factor_cache[0];   // an empty entry, else the least recently used
            for (auto& e : h->factor_cache)
                if (!e.valid ? lru->valid || e.used < lru->used : lru->valid && e.used < lru->used) lru = &e;
            lru->valid = false;
            GVT_CHECK(lru->buf.reserve(dense_operand_bytes(rows, K, parts), s));
            out = dense_operand_at(lru->buf.ptr, rows, K, parts);
            GVT_CHECK(dense_split_rows(static_cast<const float*>(F->data), F->ld, rows, K, sq, f16, 0, out, s,
                                       rowperm, colperm));
            lru->ptr = F->data;
            lru->rowperm = rowperm;
            lru->colperm = colperm;
            lru->ld = F->ld;
            lru->rows = rows;
            lru->K = K;
            lru->sq = sq;
            lru->f16 = f16;
            lru->parts = parts;
            lru->valid = true;
            lru->used = ++h->factor_cache_tick;
            return GVT_OK;
        }
        for (auto& sl : slots)
            if (sl.ptr == F->data && sl.sq == sq && sl.rows == rows && sl.K == K && sl.pattern == 0 &&
                sl.rowperm == rowperm && sl.colperm == colperm) {
                sl.used = ++tick;
                out = dense_operand_at(base + sl.off, rows, K, parts);
                return GVT_OK;
            }
        Slot& sl = slots[0].used <= slots[1].used ? slots[0] : slots[1];
        out = dense_operand_at(base + sl.off, rows, K, parts);
        GVT_CHECK(dense_split_rows(static_cast<const float*>(F->data), F->ld, rows, K, sq, f16, 0, out, s, rowperm,
                                   colperm));
        sl.ptr = F->data;
        sl.rowperm = rowperm;
        sl.colperm = colperm;
        sl.sq = sq;
        sl.rows = rows;
        sl.K = K;
        sl.pattern = 0;
        sl.used = ++tick;
        return GVT_OK;
    };
    T* S = reinterpret_cast<T*>(base + off_S);
    // S += S' of a per-tile stage 1 is left to the first reader of S: the per-tile stage 2 merges it
    // in the same pass that splits S, any other reader has it merged first
    struct PendingMerge {
        const float* Sd = nullptr;
        const int32_t* xrank = nullptr;
        int64_t Y = 0, X = 0, lds = 0;
    } pend;
    auto flush_merge = [&]() -> gvt_status {
        if (!pend.Sd) return GVT_OK;
        GVT_CHECK(dense_merge_cols(reinterpret_cast<float*>(S), pend.lds, pend.Sd, pend.lds, pend.xrank, pend.Y,
                                   pend.X, s));
        pend.Sd = nullptr;
        return GVT_OK;
    };
    for (size_t gi = 0; gi < C.two.size(); ++gi) {
        if (done[gi]) continue;
        const TwoSided& g = C.two[gi];
        const int64_t X = in_range(plan, g.recipe.begin()->first.first);
        const int64_t Y = out_range(plan, g.ob);
        const int64_t lds = round_up(X, 4);
        S1Sources srcs{};
        srcs.count = 0;
        for (auto& r : g.recipe) {
            const Order& o = plan->in_by[r.first.first];
            S1Source& sr = srcs.src[srcs.count++];
            sr.seg = o.seg;
            sr.bcol = (r.first.first == r.first.second) ? o.key : o.other;
            sr.perm = o.perm;
            sr.coef = r.second;
            sr.same = r.first.first == r.first.second ? 1 : 0;
        }
        const double E = (double)srcs.count * (double)plan->n_in;
        const double sz = (double)sizeof(T);
        if (tc1[gi] == 2) {
            // per tile: the sparse tiles' entries by the scatter-accumulate into S, the dense tiles on
            // the block-sparse GEMM into S' (relabelled columns), then S += S' through the relabelling
            const int ia = g.recipe.begin()->first.first, ib = g.recipe.begin()->first.second;
            const int64_t K = in_range(plan, ib);
            const HybridS1* h1 = nullptr;
            GVT_CHECK(hybrid_stage1(plan, ia, ib, Y, parts, s, &h1));
            const double fm = sq_mode(g.fb) ? 3.0 : 2.0;
            StatScope st(h, s, GVT_STAT_STAGE1, fm * Y * E,
                         sz * Y * (double)K + sz * Y * X + E * (8 + sz) + 4.0 * (X + 1));
            const FactorView<T>& B = fv[base_matrix(g.fb, homo)];
            S1Sources rem{};
            rem.count = 1;
            rem.src[0] = S1Source{h1->seg_r, h1->bcol_r, h1->perm_r, srcs.src[0].coef, 0};
            // the sparse part (streams factor rows from HBM) runs on the auxiliary stream beside the
            // GEMM (tensor cores); they write S and S', joined before the merge
            cudaStream_t sa = nullptr;
            GVT_CHECK(aux_fork(h, s, &sa));
            {
                const double fr = fm * Y * (double)h1->n_r;
                const double br = sz * Y * (double)K + sz * Y * X + h1->n_r * (8 + sz) + 4.0 * (X + 1);
                StatScope sk(h, sa, GVT_STAT_SPARSE_STAGE1, fr, br);
                GVT_CHECK(stage1_sparse<T>(B.Bt, B.ldbt, sq_mode(g.fb), rem, v, S, lds, Y, X, sa));
            }
            const gvt_matrix* Bm = mats[base_matrix(g.fb, homo)];
            DenseOperand a1, b1 = dense_operand_at(base + off_w, X, K, parts);
            GVT_CHECK(factor_operand(Bm, sq_mode(g.fb), Y, K, a1, nullptr, h1->kperm));
            GVT_CHECK(dense_densify_tiles(srcs.src[0], h1->xperm, h1->krank, h1->dense, h1->bn, h1->nk,
                                          reinterpret_cast<const float*>(v), X, f16, b1, s));
            TcSparse sp;
            sp.kb_list = h1->kb_list;
            sp.kb_off = h1->kb_off;
            sp.kb_parts = parts;
            sp.kb_stride = (int)(dense_kp(K) / 64);
            sp.bn = h1->bn;
            T* Sd = reinterpret_cast<T*>(base + off_sd);
            {
                StatScope sg(h, s, GVT_STAT_TC_GEMM, 2.0 * Y * h1->bn * 64.0 * parts * (double)h1->n_dense_tiles,
                             2.0 * parts * 64.0 * (double)h1->n_dense_tiles * (Y + h1->bn) + 4.0 * Y * X,
                             fm * Y * (double)h1->n_dense_entries);
                GVT_CHECK(dense_gemm(a1, b1, f16, reinterpret_cast<float*>(Sd), lds, handle_err_word(h), s,
                                     h->tc_pairs, h->tc_stall_cycles, &sp));
            }
            GVT_CHECK(aux_join(h, s));
            pend = PendingMerge{reinterpret_cast<const float*>(Sd), h1->xrank, Y, X, lds};
        } else if (tc1[gi]) {
            const int ib = g.recipe.begin()->first.second;
            const gvt_matrix* Bm = mats[base_matrix(g.fb, homo)];
            const int32_t* keys[kMaxSources] = {nullptr, nullptr, nullptr, nullptr};
            int k = 0;
            for (auto& r : g.recipe) keys[k++] = plan->in_by[r.first.first].key;
            const int64_t K = in_range(plan, ib);
            const double kp = (double)dense_kp(K);
            // the stage's algorithmic work (the same figures as the SIMT engine); the GEMM's own
            // executed flops are recorded under GVT_STAT_TC_GEMM
            StatScope st(h, s, GVT_STAT_STAGE1, (sq_mode(g.fb) ? 3.0 : 2.0) * Y * E,
                         sz * Y * (double)K + sz * Y * X + E * (8 + sz) + srcs.count * 4.0 * (X + 1));
            DenseOperand a1, b1 = dense_operand_at(base + off_w, X, K, parts);
            GVT_CHECK(factor_operand(Bm, sq_mode(g.fb), Y, K, a1));
            GVT_CHECK(dense_split_w(srcs, keys, plan->n_in, reinterpret_cast<const float*>(v), X, f16, b1,
                                    reinterpret_cast<float*>(base + off_wide), s));
            {
                StatScope sg(h, s, GVT_STAT_TC_GEMM, 2.0 * Y * X * parts * kp,
                             2.0 * parts * kp * (Y + X) + 4.0 * Y * X, (sq_mode(g.fb) ? 3.0 : 2.0) * Y * E);
                GVT_CHECK(dense_gemm(a1, b1, f16, reinterpret_cast<float*>(S), lds, handle_err_word(h), s, h->tc_pairs,
                                     h->tc_stall_cycles));
            }
        } else if (g.fb == GVT_FACTOR_IDENTITY) {
            GVT_CHECK(vec_zero<T>(S, Y * lds, s));
            StatScope st(h, s, GVT_STAT_STAGE1, E, sz * Y * X + E * (8 + sz));
            GVT_CHECK(stage1_identity<T>(srcs, v, S, lds, Y, X, s));
        } else {
            const FactorView<T>& B = fv[base_matrix(g.fb, homo)];
            const double bcols = (double)mats[base_matrix(g.fb, homo)]->cols;
            const double f1 = (sq_mode(g.fb) ? 3.0 : 2.0) * Y * E;
            const double b1 = sz * Y * bcols + sz * Y * X + E * (8 + sz) + srcs.count * 4.0 * (X + 1);
            StatScope st(h, s, GVT_STAT_STAGE1, f1, b1);
            StatScope sk(h, s, GVT_STAT_SPARSE_STAGE1, f1, b1);
            GVT_CHECK(stage1_sparse<T>(B.Bt, B.ldbt, sq_mode(g.fb), srcs, v, S, lds, Y, X, s));
        }
        // every group that reads this S (same B factor, out_b range and recipe); on the dense
        // engine S is split once, and a group whose stage-2 GEMM equals the previous one (same
        // A factor, square mode and rows: only the read-out positions differ) reuses its C
        bool s_split = false;
        const void* c_ptr = nullptr;
        int c_sq = -1;
        int64_t c_rows = -1;
        for (size_t gj = gi; gj < C.two.size(); ++gj) {
            const TwoSided& g2 = C.two[gj];
            if (done[gj] || g2.fb != g.fb || g2.recipe != g.recipe ||
                out_range(plan, g2.ob) != Y)
                continue;
            done[gj] = true;
            if (!(tc2[gj] == 2 && g2.fa != GVT_FACTOR_IDENTITY)) GVT_CHECK(flush_merge());
            const Order& oo = plan->out_by[g2.oa];
            S2Outputs outs{oo.key, (g2.oa == g2.ob) ? oo.key : oo.other, oo.perm, n_out};
            if (g2.fa == GVT_FACTOR_IDENTITY) {
                StatScope st(h, s, GVT_STAT_STAGE2, (double)n_out, (double)n_out * (12 + 3 * sz));
                GVT_CHECK(stage2_identity<T>(S, lds, X, outs, 1.0, u, s));
            } else if (tc2[gj] == 2) {
                // per tile: the dense output tiles on the tile-list GEMM C' = A' S'^T (rows relabelled)
                // and read out of C'; the other outputs by the sampled gather-dot
                const HybridS2* h2 = nullptr;
                GVT_CHECK(hybrid_stage2(plan, g2.oa, g2.ob, X, parts, parts == 1 ? 2 : 4, s, &h2));
                const int64_t mb = out_range(plan, g2.oa);
                const int64_t ldc2 = round_up(Y, 4);
                const double fm = sq_mode(g2.fa) ? 3.0 : 2.0;
                StatScope st(h, s, GVT_STAT_STAGE2, fm * X * n_out,
                             sz * ((double)mb * X + (double)Y * X) + (double)n_out * (12 + 2 * sz));
                const gvt_matrix* Fa = mats[base_matrix(g2.fa, homo)];
                DenseOperand a2, s2 = dense_operand_at(base + off_s2, Y, X, parts);
                // single pass: the remainder's dots read the GEMM's own FP16 operands (A' and S', rows
                // relabelled and scaled by powers of two), so the splits come first, S merged in the
                // same pass that splits it; otherwise the remainder reads S in FP32 once it is merged,
                // beside the splits and the GEMM
                const bool rem16 = h2->eb == 2 && h2->n_r > 0;
                auto split_operands = [&]() -> gvt_status {
                    GVT_CHECK(factor_operand(Fa, sq_mode(g2.fa), mb, X, a2, h2->aperm, nullptr));
                    if (pend.Sd && dense_merge_split_fits(X)) {
                        GVT_CHECK(dense_merge_split(reinterpret_cast<float*>(S), lds, pend.Sd, pend.lds, pend.xrank,
                                                    Y, X, f16, 1, s2, s, h2->sperm));
                        pend.Sd = nullptr;
                    } else {
                        GVT_CHECK(flush_merge());
                        GVT_CHECK(dense_split_rows(reinterpret_cast<const float*>(S), lds, Y, X, 0, f16, 1, s2, s,
                                                   h2->sperm, nullptr));
                    }
                    return GVT_OK;
                };
                if (rem16) GVT_CHECK(split_operands());
                else GVT_CHECK(flush_merge());
                // the remainder's sampled dots (HBM-bound) on the auxiliary stream beside the tile-list
                // GEMM; they add into disjoint outputs of u
                cudaStream_t sa = nullptr;
                GVT_CHECK(aux_fork(h, s, &sa));
                {
                    const FactorView<T>& A = fv[base_matrix(g2.fa, homo)];
                    const double fr = fm * X * (double)h2->n_r;
                    const double zb = rem16 ? 2.0 : sz;
                    const double br = zb * ((double)mb * X + (double)Y * X) + (double)h2->n_r * (12 + 2 * sz);
                    StatScope sk(h, sa, GVT_STAT_SPARSE_STAGE2, fr, br);
                    if (rem16)
                        GVT_CHECK(stage2_gather_f16(a2.data, a2.kp, a2.inv_scale, s2.data, s2.kp, s2.inv_scale, a2.kp,
                                                    S2Outputs{h2->arow_rl, h2->srow_rl, h2->perm_r, h2->n_r}, 1.0,
                                                    reinterpret_cast<float*>(u), sa));
                    else
                        GVT_CHECK(stage2_gather<T>(A.A, A.lda, sq_mode(g2.fa), S, lds, X,
                                                   S2Outputs{h2->arow_r, h2->srow_r, h2->perm_r, h2->n_r}, 1.0, u,
                                                   sa));
                }
                if (!rem16) GVT_CHECK(split_operands());
                s_split = false;   // s2 now holds the relabelled split
                float* C2 = reinterpret_cast<float*>(base + off_c2);
                TcSparse sp;
                sp.tile_list = h2->tiles;
                sp.n_tiles = h2->n_tiles;
                sp.bn = h2->bn;
                {
                    const double kp = (double)dense_kp(X);
                    StatScope sg(h, s, GVT_STAT_TC_GEMM, 2.0 * h2->bm * h2->bn * kp * parts * (double)h2->n_tiles,
                                 2.0 * parts * kp * (double)h2->n_tiles * (h2->bm + h2->bn) +
                                     4.0 * h2->bm * h2->bn * (double)h2->n_tiles,
                                 fm * X * (double)h2->n_d);
                    GVT_CHECK(dense_gemm(a2, s2, f16, C2, ldc2, handle_err_word(h), s, h->tc_pairs, h->tc_stall_cycles,
                                         &sp));
                }
                c_ptr = nullptr;
                GVT_CHECK(dense_gather(C2, ldc2, S2Outputs{h2->arow_d, h2->srow_d, h2->perm_d, h2->n_d},
                                       reinterpret_cast<float*>(u), s));
                GVT_CHECK(aux_join(h, s));
            } else if (tc2[gj]) {
                const int64_t mb = out_range(plan, g2.oa);
                const int64_t ldc2 = round_up(Y, 4);
                const double kp = (double)dense_kp(X);
                StatScope st(h, s, GVT_STAT_STAGE2, (sq_mode(g2.fa) ? 3.0 : 2.0) * X * n_out,
                             sz * ((double)mb * X + (double)Y * X) + (double)n_out * (12 + 2 * sz));
                DenseOperand a2, s2 = dense_operand_at(base + off_s2, Y, X, parts);
                const gvt_matrix* Fa = mats[base_matrix(g2.fa, homo)];
                float* C2 = reinterpret_cast<float*>(base + off_c2);
                if (!(c_ptr == Fa->data && c_sq == sq_mode(g2.fa) && c_rows == mb)) {
                    // useful flops of this GEMM: its own group's sampled dots and those of the later
                    // groups of this S that read the same C out (until another GEMM replaces it)
                    double c2_useful = 0.0;
                    for (size_t gk = gj; gk < C.two.size(); ++gk) {
                        const TwoSided& g3 = C.two[gk];
                        if ((gk != gj && done[gk]) || g3.fb != g.fb || g3.recipe != g.recipe ||
                            out_range(plan, g3.ob) != Y || g3.fa == GVT_FACTOR_IDENTITY || !tc2[gk])
                            continue;
                        const gvt_matrix* F3 = mats[base_matrix(g3.fa, homo)];
                        if (F3->data != Fa->data || sq_mode(g3.fa) != sq_mode(g2.fa) || out_range(plan, g3.oa) != mb)
                            break;
                        c2_useful += (sq_mode(g3.fa) ? 3.0 : 2.0) * X * (double)n_out;
                    }
                    GVT_CHECK(factor_operand(Fa, sq_mode(g2.fa), mb, X, a2));
                    if (!s_split) {
                        GVT_CHECK(dense_split_rows(reinterpret_cast<const float*>(S), lds, Y, X, 0, f16, 1, s2, s));
                        s_split = true;
                    }
                    StatScope sg(h, s, GVT_STAT_TC_GEMM, 2.0 * mb * Y * parts * kp,
                                 2.0 * parts * kp * (mb + Y) + 4.0 * mb * Y, c2_useful);
                    GVT_CHECK(dense_gemm(a2, s2, f16, C2, ldc2, handle_err_word(h), s, h->tc_pairs, h->tc_stall_cycles));
                    c_ptr = Fa->data;
                    c_sq = sq_mode(g2.fa);
                    c_rows = mb;
                }
                GVT_CHECK(dense_gather(C2, ldc2, outs, reinterpret_cast<float*>(u), s));
            } else {
                const FactorView<T>& A = fv[base_matrix(g2.fa, homo)];
                const double arows = (double)out_range(plan, g2.oa);
                const double f2 = (sq_mode(g2.fa) ? 3.0 : 2.0) * X * n_out;
                const double b2 = sz * (arows * X + (double)Y * X) + (double)n_out * (12 + 2 * sz);
                StatScope st(h, s, GVT_STAT_STAGE2, f2, b2);
                StatScope sk(h, s, GVT_STAT_SPARSE_STAGE2, f2, b2);
                GVT_CHECK(stage2_gather<T>(A.A, A.lda, sq_mode(g2.fa), S, lds, X, outs, 1.0, u, s));
            }
        }
        GVT_CHECK(flush_merge());
    }

    // ---- one-sided groups; those on the same factor (data and square mode) share one pass over it
    std::vector<bool> od(C.one.size(), false);
    for (size_t i = 0; i < C.one.size(); ++i) {
        if (od[i]) continue;
        const gvt_matrix* Fm = mats[base_matrix(C.one[i].f, homo)];
        const int sq = sq_mode(C.one[i].f);
        std::vector<size_t> L{i};
        od[i] = true;
        for (size_t j = i + 1; j < C.one.size() && (int)L.size() < kMaxOneSidedShare; ++j)
            if (!od[j] && mats[base_matrix(C.one[j].f, homo)]->data == Fm->data && sq_mode(C.one[j].f) == sq) {
                L.push_back(j);
                od[j] = true;
            }
        const int G = (int)L.size();
        int64_t R = 0;
        double nsrc = 0.0;
        for (size_t g : L) {
            R = std::max(R, out_range(plan, C.one[g].oc));
            nsrc += (double)C.one[g].sources.size();
        }
        const int64_t Xc = Fm->cols;
        T* sv = reinterpret_cast<T*>(base + off_one);
        T* z = sv + (size_t)G * Xc;
        const double sz = (double)sizeof(T);
        StatScope st(h, s, GVT_STAT_ONE_SIDED,
                     nsrc * plan->n_in + G * ((sq ? 3.0 : 2.0) * R * (double)Xc) + (double)G * n_out,
                     nsrc * plan->n_in * (4 + sz) + sz * (R * (double)Xc + G * ((double)Xc + R)) +
                         (double)n_out * (G * 4 + 2 * sz));
        GVT_CHECK(vec_zero<T>(sv, (int64_t)G * Xc, s));
        const T* zs[kMaxOneSidedShare];
        const int32_t* idxs[kMaxOneSidedShare];
        for (int k = 0; k < G; ++k) {
            const OneSided& g = C.one[L[k]];
            for (auto& src : g.sources) {
                const Order& o = plan->in_by[src.first];
                GVT_CHECK(segment_sums<T>(o.seg, o.perm, in_range(plan, src.first), v, src.second,
                                          sv + (size_t)k * Xc, s));
            }
            zs[k] = z + (size_t)k * R;
            idxs[k] = (g.oc == GVT_FIRST) ? plan->d_out : plan->t_out;
        }
        GVT_CHECK(gemv_rows_multi<T>(static_cast<const T*>(Fm->data), Fm->ld, sq, R, Xc, sv, Xc, G, z, R, s));
        GVT_CHECK(gather_add_multi<T>(zs, idxs, G, n_out, u, s));
    }
    return GVT_OK;
}

template gvt_status pairwise_apply<float>(gvt_plan*, const gvt_desc*, const gvt_matrix*,
                                          const gvt_matrix*, const float*, float*, cudaStream_t);
template gvt_status pairwise_apply<double>(gvt_plan*, const gvt_desc*, const gvt_matrix*,
                                           const gvt_matrix*, const double*, double*, cudaStream_t);

}  // namespace gvt
