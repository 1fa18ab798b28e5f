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
    const bool tc = sizeof(T) == 4 && h->stage1_engine == GVT_STAGE1_TC_BF16X3;
    Compiled C;
    GVT_CHECK(compile(plan, desc, mats, tc, C));

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
        one_elems = std::max(one_elems, F->cols + F->rows);
    }
    const size_t off_one = one_elems > 0 ? ws.take(sizeof(T) * (size_t)one_elems) : 0;
    size_t tc_bytes = 0;
    if (tc)
        for (auto& g : C.two)
            if (is_dense(g.fa) && is_dense(g.fb)) {
                const int ib = g.recipe.begin()->first.second;
                const int64_t X = in_range(plan, g.recipe.begin()->first.first);
                tc_bytes = std::max(tc_bytes, dense_stage1_workspace(out_range(plan, g.ob), in_range(plan, ib), X));
            }
    const size_t off_tc = tc_bytes > 0 ? ws.take(tc_bytes) : 0;
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
    // the dense stage 1's BF16 split of its factor stays valid in the workspace for the
    // next group with the same factor, square mode and extents
    const void* split_of = nullptr;
    int split_sq = -1;
    int64_t split_Y = -1, split_K = -1;
    T* S = reinterpret_cast<T*>(base + off_S);
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
        }
        const double E = (double)srcs.count * (double)plan->n_in;
        const double sz = (double)sizeof(T);
        bool same_ib = true;   // every source's W row ids share one id range (the K of the GEMM)
        for (auto& r : g.recipe)
            same_ib = same_ib && in_range(plan, r.first.second) == in_range(plan, g.recipe.begin()->first.second);
        if (tc && is_dense(g.fa) && is_dense(g.fb) && same_ib) {
            const int ib = g.recipe.begin()->first.second;
            const gvt_matrix* Bm = mats[base_matrix(g.fb, homo)];
            const int32_t* keys[kMaxSources] = {nullptr, nullptr, nullptr, nullptr};
            int k = 0;
            for (auto& r : g.recipe) keys[k++] = plan->in_by[r.first.first].key;
            const int64_t K = in_range(plan, ib);
            StatScope st(h, s, GVT_STAT_STAGE1, 2.0 * 3.0 * Y * (double)((K + 63) / 64 * 64) * X,
                         2.0 * (3.0 * (Y + X) * ((K + 63) / 64 * 64)) + sz * Y * X + E * (8 + sz));
            const int reuse = split_of == Bm->data && split_sq == sq_mode(g.fb) && split_Y == Y && split_K == K;
            GVT_CHECK(dense_stage1(reinterpret_cast<const float*>(Bm->data), Bm->ld, Y, K, sq_mode(g.fb), srcs, keys,
                                   plan->n_in, reinterpret_cast<const float*>(v), X, reinterpret_cast<float*>(S), lds,
                                   base + off_tc, reuse, handle_err_word(h), s));
            split_of = Bm->data;
            split_sq = sq_mode(g.fb);
            split_Y = Y;
            split_K = K;
        } else if (g.fb == GVT_FACTOR_IDENTITY) {
            GVT_CHECK(vec_zero<T>(S, Y * lds, s));
            StatScope st(h, s, GVT_STAT_STAGE1, E, sz * Y * X + E * (8 + sz));
            GVT_CHECK(stage1_identity<T>(srcs, v, S, lds, Y, X, s));
        } else {
            const FactorView<T>& B = fv[base_matrix(g.fb, homo)];
            const double bcols = (double)mats[base_matrix(g.fb, homo)]->cols;
            StatScope st(h, s, GVT_STAT_STAGE1, (sq_mode(g.fb) ? 3.0 : 2.0) * Y * E,
                         sz * Y * bcols + sz * Y * X + E * (8 + sz) + srcs.count * 4.0 * (X + 1));
            GVT_CHECK(stage1_dense<T>(B.Bt, B.ldbt, sq_mode(g.fb), srcs, v, S, lds, Y, X, s));
        }
        // every group that reads this S (same B factor, out_b range and recipe)
        for (size_t gj = gi; gj < C.two.size(); ++gj) {
            const TwoSided& g2 = C.two[gj];
            if (done[gj] || g2.fb != g.fb || g2.recipe != g.recipe ||
                out_range(plan, g2.ob) != Y)
                continue;
            done[gj] = true;
            const Order& oo = plan->out_by[g2.oa];
            S2Outputs outs{oo.key, (g2.oa == g2.ob) ? oo.key : oo.other, oo.perm, n_out};
            if (g2.fa == GVT_FACTOR_IDENTITY) {
                StatScope st(h, s, GVT_STAT_STAGE2, (double)n_out, (double)n_out * (12 + 3 * sz));
                GVT_CHECK(stage2_identity<T>(S, lds, X, outs, 1.0, u, s));
            } else {
                const FactorView<T>& A = fv[base_matrix(g2.fa, homo)];
                const double arows = (double)out_range(plan, g2.oa);
                StatScope st(h, s, GVT_STAT_STAGE2, (sq_mode(g2.fa) ? 3.0 : 2.0) * X * n_out,
                             sz * (arows * X + (double)Y * X) + (double)n_out * (12 + 2 * sz));
                GVT_CHECK(stage2_dense<T>(A.A, A.lda, sq_mode(g2.fa), S, lds, X, outs, 1.0, u, s));
            }
        }
    }

    // ---- one-sided groups
    for (auto& g : C.one) {
        const gvt_matrix* Fm = mats[base_matrix(g.f, homo)];
        T* sv = reinterpret_cast<T*>(base + off_one);
        T* z = sv + Fm->cols;
        const double sz = (double)sizeof(T);
        const int64_t R = out_range(plan, g.oc);
        const double Xc = (double)Fm->cols;
        StatScope st(h, s, GVT_STAT_ONE_SIDED,
                     (double)g.sources.size() * plan->n_in + (sq_mode(g.f) ? 3.0 : 2.0) * R * Xc + n_out,
                     (double)g.sources.size() * plan->n_in * (4 + sz) + sz * (R * Xc + Xc + R) +
                         (double)n_out * (4 + 3 * sz));
        GVT_CHECK(vec_zero<T>(sv, Fm->cols, s));
        for (auto& src : g.sources) {
            const Order& o = plan->in_by[src.first];
            GVT_CHECK(segment_sums<T>(o.seg, o.perm, in_range(plan, src.first), v, src.second, sv, s));
        }
        GVT_CHECK(gemv_rows<T>(static_cast<const T*>(Fm->data), Fm->ld, sq_mode(g.f), R,
                               Fm->cols, sv, z, s));
        const int32_t* idx = (g.oc == GVT_FIRST) ? plan->d_out : plan->t_out;
        GVT_CHECK(gather_add<T>(z, idx, n_out, u, s));
    }
    return GVT_OK;
}

template gvt_status pairwise_apply<float>(gvt_plan*, const gvt_desc*, const gvt_matrix*,
                                          const gvt_matrix*, const float*, float*, cudaStream_t);
template gvt_status pairwise_apply<double>(gvt_plan*, const gvt_desc*, const gvt_matrix*,
                                           const gvt_matrix*, const double*, double*, cudaStream_t);

}  // namespace gvt
