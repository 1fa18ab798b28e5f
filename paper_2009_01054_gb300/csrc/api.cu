// C ABI entry points: handles, plans, descriptors and products.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "gvt_internal.h"

namespace gvt {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};
}

void set_error(const std::string& msg) { g_last_error = msg; }

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long gvt_launch_count_internal() { return g_launches.load(std::memory_order_relaxed); }

StatScope::StatScope(gvt_handle* h_, cudaStream_t s_, int kind_, double flops_, double bytes_, double useful_)
    : h(h_), s(s_), kind(kind_), flops(flops_), bytes(bytes_), useful(useful_ < 0.0 ? flops_ : useful_)
{
    if (!h || !h->stats_on) return;
    if (h->event_pool.size() < 2) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); break; }
            h->event_pool.push_back(e);
        }
        if (h->event_pool.size() < 2) return;
    }
    e0 = h->event_pool.back();
    h->event_pool.pop_back();
    cudaEventRecord(e0, s);
}

StatScope::~StatScope()
{
    if (!e0) return;
    // nested scopes may have used the pool up since the constructor: create the end event then
    if (h->event_pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            h->event_pool.push_back(e0);   // drop this record
            return;
        }
        h->event_pool.push_back(e);
    }
    cudaEvent_t e1 = h->event_pool.back();
    h->event_pool.pop_back();
    cudaEventRecord(e1, s);
    h->recs.push_back(StatRec{kind, e0, e1, flops, bytes, useful});
}

gvt_status aux_fork(gvt_handle* h, cudaStream_t s, cudaStream_t* aux)
{
    if (!h->aux) {
        GVT_CUDA(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        GVT_CUDA(cudaEventCreateWithFlags(&h->aux_fork, cudaEventDisableTiming));
        GVT_CUDA(cudaEventCreateWithFlags(&h->aux_join, cudaEventDisableTiming));
    }
    GVT_CUDA(cudaEventRecord(h->aux_fork, s));
    GVT_CUDA(cudaStreamWaitEvent(h->aux, h->aux_fork, 0));
    *aux = h->aux;
    return GVT_OK;
}

gvt_status aux_join(gvt_handle* h, cudaStream_t s)
{
    GVT_CUDA(cudaEventRecord(h->aux_join, h->aux));
    GVT_CUDA(cudaStreamWaitEvent(s, h->aux_join, 0));
    return GVT_OK;
}

gvt_status cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GVT_ERR_ALLOC : GVT_ERR_CUDA;
}

gvt_status ensure_smem_attr(const void* func, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> raised;   // (kernel, device) -> limit set
    int dev = 0;
    GVT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    int& have = raised[{func, dev}];
    if (have >= bytes) return GVT_OK;
    GVT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    have = bytes;
    return GVT_OK;
}

gvt_status DevBuf::reserve(size_t nbytes, cudaStream_t s)
{
    if (nbytes <= bytes) return GVT_OK;
    size_t want = nbytes + nbytes / 4;
    if (ptr) {
        GVT_CUDA(cudaStreamSynchronize(s));
        GVT_CUDA(cudaFree(ptr));
        ptr = nullptr;
        bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        set_error("workspace allocation of " + std::to_string(want) + " bytes failed");
        return GVT_ERR_ALLOC;
    }
    bytes = want;
    return GVT_OK;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

}  // namespace gvt

using namespace gvt;

namespace {

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

gvt_status check_matrix(const gvt_matrix* A, int dtype, const char* name, bool required)
{
    if (!A) {
        if (!required) return GVT_OK;
        set_error(std::string(name) + " is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    if (!A->data || A->rows < 0 || A->cols < 0 || A->ld < A->cols) {
        set_error(std::string(name) + ": bad data pointer, shape or leading dimension");
        return GVT_ERR_INVALID_ARG;
    }
    if (A->dtype != dtype) {
        set_error(std::string(name) + ": dtype differs from the call's dtype");
        return GVT_ERR_INVALID_ARG;
    }
    return GVT_OK;
}

gvt_status plan_alloc(gvt_plan* p, void** out, size_t bytes)
{
    *out = nullptr;
    if (bytes == 0) bytes = 4;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("plan allocation failed");
        return GVT_ERR_ALLOC;
    }
    p->allocs.push_back(*out);
    return GVT_OK;
}

template <class P>
gvt_status plan_alloc_t(gvt_plan* p, P** out, size_t count)
{
    void* ptr;
    GVT_CHECK(plan_alloc(p, &ptr, count * sizeof(**out)));
    *out = static_cast<P*>(ptr);
    return GVT_OK;
}

gvt_status build_order(gvt_plan* p, const int32_t* keyc, const int32_t* otherc, int64_t n, int64_t K,
                       Order& o, void* sort_ws, cudaStream_t s)
{
    o.K = K;
    GVT_CHECK(plan_alloc_t(p, &o.key, (size_t)n));
    GVT_CHECK(plan_alloc_t(p, &o.other, (size_t)n));
    GVT_CHECK(plan_alloc_t(p, &o.perm, (size_t)n));
    GVT_CHECK(plan_alloc_t(p, &o.seg, (size_t)K + 1));
    GVT_CHECK(radix_sort_by_key(keyc, n, K, o.key, o.perm, sort_ws, s));
    GVT_CHECK(gather_i32(otherc, o.perm, n, o.other, s));
    GVT_CHECK(segment_offsets(o.key, n, K, o.seg, s));
    return GVT_OK;
}

const int64_t kMaxCount = (int64_t(1) << 31) - 1;

template <class T>
gvt_status apply_cols(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* N,
                      const void* v, void* u, int64_t k_cols, cudaStream_t s)
{
    for (int64_t c = 0; c < k_cols; ++c) {
        const T* vc = static_cast<const T*>(v) + c * plan->n_in;
        T* uc = static_cast<T*>(u) + c * plan->n_out;
        GVT_CHECK(pairwise_apply<T>(plan, desc, M, N, vc, uc, s));
    }
    return GVT_OK;
}

gvt_status pairwise_entry(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* N,
                          const void* v, void* u, int64_t k_cols, int32_t dtype, void* stream)
{
    if (!plan || !desc) {
        set_error("plan or descriptor is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    if (dtype != GVT_F64 && dtype != GVT_F32) {
        set_error("products support GVT_F64 and GVT_F32");
        return GVT_ERR_UNSUPPORTED;
    }
    if (k_cols < 0) {
        set_error("k_cols < 0");
        return GVT_ERR_INVALID_ARG;
    }
    const bool homo = desc->homogeneous != 0;
    GVT_CHECK(check_matrix(M, dtype, "M", true));
    GVT_CHECK(check_matrix(N, dtype, "N", !homo));
    if (homo && (plan->m_rows != plan->q_rows || plan->m_cols != plan->q_cols)) {
        set_error("homogeneous kernel on a plan whose drug and target id ranges differ");
        return GVT_ERR_INVALID_ARG;
    }
    if ((plan->n_in > 0 && !v && k_cols > 0) || (plan->n_out > 0 && !u && k_cols > 0)) {
        set_error("v or u is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    if (k_cols == 0 || plan->n_out == 0) return GVT_OK;
    cudaStream_t s = as_stream(stream);
    if (dtype == GVT_F64) return apply_cols<double>(plan, desc, M, N, v, u, k_cols, s);
    return apply_cols<float>(plan, desc, M, N, v, u, k_cols, s);
}

}  // namespace

extern "C" {

const char* gvt_last_error(void) { return gvt::g_last_error.c_str(); }

int32_t gvt_version(void) { return 10000; }

gvt_status gvt_create(gvt_handle** out)
{
    if (!out) {
        set_error("gvt_create: out is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    gvt_handle* h = new (std::nothrow) gvt_handle();
    if (!h) {
        set_error("gvt_create: host allocation failed");
        return GVT_ERR_ALLOC;
    }
    if (h->status.reserve(256, nullptr) != GVT_OK || cudaMemset(h->status.ptr, 0, h->status.bytes) != cudaSuccess) {
        cudaGetLastError();
        h->status.release();
        delete h;
        set_error("gvt_create: device status buffer allocation failed");
        return GVT_ERR_ALLOC;
    }
    if (cudaMallocHost(&h->host_scalars, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        h->status.release();
        delete h;
        set_error("gvt_create: pinned allocation failed");
        return GVT_ERR_ALLOC;
    }
    *out = h;
    return GVT_OK;
}

gvt_status gvt_destroy(gvt_handle* h)
{
    if (!h) return GVT_OK;
    cudaDeviceSynchronize();
    for (auto& r : h->recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    h->ws.buf.release();
    h->solve_ws.buf.release();
    h->status.release();
    for (auto& e : h->factor_cache) e.buf.release();
    if (h->host_scalars) cudaFreeHost(h->host_scalars);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux_fork) cudaEventDestroy(h->aux_fork);
    if (h->aux_join) cudaEventDestroy(h->aux_join);
    if (h->cg_stream) cudaStreamDestroy(h->cg_stream);
    if (h->cg_fork) cudaEventDestroy(h->cg_fork);
    if (h->cg_join) cudaEventDestroy(h->cg_join);
    delete h;
    return GVT_OK;
}

gvt_status gvt_plan_create(gvt_handle* h, int64_t m_rows, int64_t m_cols, int64_t q_rows, int64_t q_cols,
                           const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                           const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                           void* stream, gvt_plan** out)
{
    if (!h || !out) {
        set_error("gvt_plan_create: handle or out is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const bool same = (d_out == nullptr && t_out == nullptr);
    if (same) n_out = n_in;
    if (m_rows < 0 || m_cols < 0 || q_rows < 0 || q_cols < 0 || m_rows > kMaxCount ||
        m_cols > kMaxCount || q_rows > kMaxCount || q_cols > kMaxCount) {
        set_error("gvt_plan_create: bad kernel matrix shape");
        return GVT_ERR_INVALID_ARG;
    }
    if (n_in < 0 || n_out < 0 || n_in > kMaxCount || n_out > kMaxCount) {
        set_error("gvt_plan_create: pair counts must be in [0, 2^31)");
        return GVT_ERR_INVALID_ARG;
    }
    if ((n_in > 0 && (!d_in || !t_in)) || (!same && n_out > 0 && (!d_out || !t_out))) {
        set_error("gvt_plan_create: NULL index array");
        return GVT_ERR_INVALID_ARG;
    }
    if (!same && ((d_out == nullptr) != (t_out == nullptr))) {
        set_error("gvt_plan_create: pass both output arrays or neither");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t s = as_stream(stream);
    gvt_plan* p = new (std::nothrow) gvt_plan();
    if (!p) {
        set_error("gvt_plan_create: host allocation failed");
        return GVT_ERR_ALLOC;
    }
    p->h = h;
    p->m_rows = m_rows; p->m_cols = m_cols; p->q_rows = q_rows; p->q_cols = q_cols;
    p->n_in = n_in; p->n_out = n_out; p->out_is_in = same;

    auto fail = [&](gvt_status st) { gvt_plan_destroy(p); return st; };
    gvt_status st;
    if ((st = plan_alloc_t(p, &p->d_in, (size_t)n_in)) != GVT_OK) return fail(st);
    if ((st = plan_alloc_t(p, &p->t_in, (size_t)n_in)) != GVT_OK) return fail(st);
    if (n_in > 0) {
        if (cudaMemcpyAsync(p->d_in, d_in, 4 * n_in, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(p->t_in, t_in, 4 * n_in, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "copy input pairs"));
    }
    if (same) {
        p->d_out = p->d_in;
        p->t_out = p->t_in;
    } else {
        if ((st = plan_alloc_t(p, &p->d_out, (size_t)n_out)) != GVT_OK) return fail(st);
        if ((st = plan_alloc_t(p, &p->t_out, (size_t)n_out)) != GVT_OK) return fail(st);
        if (n_out > 0 &&
            (cudaMemcpyAsync(p->d_out, d_out, 4 * n_out, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
             cudaMemcpyAsync(p->t_out, t_out, 4 * n_out, cudaMemcpyDeviceToDevice, s) != cudaSuccess))
            return fail(cuda_fail(cudaGetLastError(), "copy output pairs"));
    }

    // ---- validation: every id inside its kernel matrix dimension
    {
        int32_t* mm = h->status.as<int32_t>();
        struct Chk { const int32_t* a; int64_t n; int64_t bound; const char* name; };
        Chk chks[4] = {
            {p->d_in, n_in, same ? std::min(m_cols, m_rows) : m_cols, "d_in"},
            {p->t_in, n_in, same ? std::min(q_cols, q_rows) : q_cols, "t_in"},
            {same ? nullptr : p->d_out, n_out, m_rows, "d_out"},
            {same ? nullptr : p->t_out, n_out, q_rows, "t_out"}};
        for (auto& c : chks) {
            if (!c.a || c.n == 0) continue;
            if ((st = minmax_i32(c.a, c.n, mm, s)) != GVT_OK) return fail(st);
            int32_t hmm[2];
            if (cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "index validation"));
            if (hmm[0] < 0 || (int64_t)hmm[1] >= c.bound) {
                set_error(std::string("gvt_plan_create: ") + c.name + " has an index outside [0, " +
                          std::to_string(c.bound) + ") (min " + std::to_string(hmm[0]) + ", max " +
                          std::to_string(hmm[1]) + ")");
                return fail(GVT_ERR_INDEX_OOB);
            }
        }
    }

    // ---- sorted orders
    {
        const int64_t nmax = std::max(n_in, n_out);
        void* sort_ws = nullptr;
        const size_t wsb = sort_workspace_bytes(nmax);
        if (cudaMalloc(&sort_ws, wsb) != cudaSuccess) {
            cudaGetLastError();
            set_error("gvt_plan_create: sort workspace allocation failed");
            return fail(GVT_ERR_ALLOC);
        }
        st = build_order(p, p->d_in, p->t_in, n_in, m_cols, p->in_by[0], sort_ws, s);
        if (st == GVT_OK) st = build_order(p, p->t_in, p->d_in, n_in, q_cols, p->in_by[1], sort_ws, s);
        if (st == GVT_OK && !same) {
            st = build_order(p, p->d_out, p->t_out, n_out, m_rows, p->out_by[0], sort_ws, s);
            if (st == GVT_OK)
                st = build_order(p, p->t_out, p->d_out, n_out, q_rows, p->out_by[1], sort_ws, s);
        }
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(sort_ws);
        if (st != GVT_OK) return fail(st);
        if (e != cudaSuccess) return fail(cuda_fail(e, "plan sort"));
    }
    if (same) {
        p->out_by[0] = p->in_by[0];
        p->out_by[1] = p->in_by[1];
    }
    *out = p;
    return GVT_OK;
}

gvt_status gvt_plan_destroy(gvt_plan* p)
{
    if (!p) return GVT_OK;
    cudaDeviceSynchronize();
    for (void* a : p->allocs) cudaFree(a);
    delete p;
    return GVT_OK;
}

gvt_status gvt_plan_sizes(const gvt_plan* p, int64_t* n_in, int64_t* n_out)
{
    if (!p) {
        set_error("plan is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    if (n_in) *n_in = p->n_in;
    if (n_out) *n_out = p->n_out;
    return GVT_OK;
}

gvt_status gvt_desc_make(int32_t kind, gvt_desc* out)
{
    if (!out) {
        set_error("gvt_desc_make: out is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    out->kind = kind;
    const int F = GVT_FIRST, S = GVT_SECOND;
    auto add = [&](double c, int fa, int fb, int oa, int ob, int ia, int ib) {
        out->terms[out->n_terms++] = gvt_term{c, fa, fb, oa, ob, ia, ib};
    };
    const int M = GVT_FACTOR_M, N = GVT_FACTOR_N, M2 = GVT_FACTOR_M_SQ, N2 = GVT_FACTOR_N_SQ;
    const int ONE = GVT_FACTOR_ONES, I = GVT_FACTOR_IDENTITY;
    switch (kind) {
    case GVT_KERNEL_KRONECKER:
    case GVT_KERNEL_GAUSSIAN:      // D kron T
        add(1, M, N, F, S, F, S);
        break;
    case GVT_KERNEL_LINEAR:        // D kron 1 + 1 kron T
        add(1, M, ONE, F, S, F, S);
        add(1, ONE, N, F, S, F, S);
        break;
    case GVT_KERNEL_POLY2D:        // Q(D kron D)Q^T + 2 D kron T + PQ(T kron T)Q^T P^T
        add(1, M2, ONE, F, S, F, S);
        add(2, M, N, F, S, F, S);
        add(1, ONE, N2, F, S, F, S);
        break;
    case GVT_KERNEL_CARTESIAN:     // D kron I + I kron T
        add(1, M, I, F, S, F, S);
        add(1, I, N, F, S, F, S);
        break;
    case GVT_KERNEL_SYMMETRIC:     // (I + P)(D kron D): the P term reads the input pair swapped
        out->homogeneous = 1;
        add(1, M, M, F, S, F, S);
        add(1, M, M, F, S, S, F);
        break;
    case GVT_KERNEL_ANTISYMMETRIC: // (I - P)(D kron D), the sign of Table 4b
        out->homogeneous = 1;
        add(1, M, M, F, S, F, S);
        add(-1, M, M, F, S, S, F);
        break;
    case GVT_KERNEL_RANKING:       // (I - P)(D kron 1)(I - P): four one-sided terms
        out->homogeneous = 1;
        add(1, M, ONE, F, S, F, S);
        add(-1, M, ONE, F, S, S, F);
        add(-1, M, ONE, S, F, F, S);
        add(1, M, ONE, S, F, S, F);
        break;
    case GVT_KERNEL_MLPK:          // (I + P)(I - Q)(D kron D)(I - Q)^T(I + P): ten terms
        out->homogeneous = 1;
        add(1, M2, ONE, F, S, F, S);    // k(d,dbar)^2        = Q(DxD)Q^T
        add(1, M2, ONE, F, S, S, F);    // k(d,dbar')^2       = Q(DxD)Q^T P
        add(1, M2, ONE, S, F, F, S);    // k(d',dbar)^2       = PQ(DxD)Q^T
        add(1, M2, ONE, S, F, S, F);    // k(d',dbar')^2      = PQ(DxD)Q^T P
        add(2, M, M, F, S, F, S);       // 2 k(d,dbar)k(d',dbar')   = 2(DxD)
        add(2, M, M, F, S, S, F);       // 2 k(d,dbar')k(d',dbar)   = 2P(DxD)
        add(-2, M, M, F, F, F, S);      // -2 k(d,dbar)k(d,dbar')   = -2Q(DxD)
        add(-2, M, M, S, S, F, S);      // -2 k(d',dbar)k(d',dbar') = -2PQ(DxD)
        add(-2, M, M, F, S, F, F);      // -2 k(d,dbar)k(d',dbar)   = -2(DxD)Q^T
        add(-2, M, M, F, S, S, S);      // -2 k(d,dbar')k(d',dbar') = -2(DxD)Q^T P
        break;
    default:
        set_error("gvt_desc_make: unknown kernel kind");
        return GVT_ERR_INVALID_ARG;
    }
    (void)N2;
    return GVT_OK;
}

gvt_status gvt_matvec(gvt_plan* plan, const gvt_matrix* M, const gvt_matrix* N, const void* v, void* u,
                      int64_t k_cols, int32_t dtype, void* stream)
{
    gvt_desc d;
    gvt_desc_make(GVT_KERNEL_KRONECKER, &d);
    return pairwise_entry(plan, &d, M, N, v, u, k_cols, dtype, stream);
}

gvt_status gvt_pairwise_kernel_matvec(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M,
                                      const gvt_matrix* N, const void* v, void* u, int64_t k_cols,
                                      int32_t dtype, void* stream)
{
    return pairwise_entry(plan, desc, M, N, v, u, k_cols, dtype, stream);
}

gvt_status gvt_predict(gvt_plan* plan, const gvt_desc* desc, const gvt_matrix* M, const gvt_matrix* N,
                       const void* a, void* p, int64_t k_cols, int32_t dtype, void* stream)
{
    return pairwise_entry(plan, desc, M, N, a, p, k_cols, dtype, stream);
}

gvt_status gvt_gaussian_kernel(gvt_handle* h, const double* X, int64_t rows_x, const double* Y,
                               int64_t rows_y, int64_t dim, double gamma, void* K, int64_t ldk,
                               int32_t out_dtype, void* stream)
{
    if (!h || (rows_x > 0 && (!X || !K)) || (rows_y > 0 && !Y) || rows_x < 0 || rows_y < 0 || dim < 0 ||
        ldk < rows_y) {
        set_error("gvt_gaussian_kernel: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    if ((rows_x + 31) / 32 > 65535) {
        set_error("gvt_gaussian_kernel: too many rows");
        return GVT_ERR_UNSUPPORTED;
    }
    return gaussian_kernel(X, rows_x, Y, rows_y, dim, gamma, K, ldk, out_dtype, as_stream(stream));
}

gvt_status gvt_linear_kernel(gvt_handle* h, const double* X, int64_t rows_x, const double* Y, int64_t rows_y,
                             int64_t dim, void* K, int64_t ldk, int32_t out_dtype, void* stream)
{
    if (!h || (rows_x > 0 && (!X || !K)) || (rows_y > 0 && !Y) || rows_x < 0 || rows_y < 0 || dim < 0 ||
        ldk < rows_y) {
        set_error("gvt_linear_kernel: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    if ((rows_x + 31) / 32 > 65535) {
        set_error("gvt_linear_kernel: too many rows");
        return GVT_ERR_UNSUPPORTED;
    }
    return linear_kernel(X, rows_x, Y, rows_y, dim, K, ldk, out_dtype, as_stream(stream));
}

gvt_status gvt_tanimoto_kernel(gvt_handle* h, const uint32_t* X, int64_t rows_x, const uint32_t* Y,
                               int64_t rows_y, int64_t words, void* K, int64_t ldk, int32_t out_dtype,
                               void* stream)
{
    if (!h || (rows_x > 0 && (!X || !K)) || (rows_y > 0 && !Y) || rows_x < 0 || rows_y < 0 || words < 0 ||
        ldk < rows_y) {
        set_error("gvt_tanimoto_kernel: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    if ((rows_x + 31) / 32 > 65535 || words > (int64_t)1 << 26) {
        set_error("gvt_tanimoto_kernel: too many rows or words");
        return GVT_ERR_UNSUPPORTED;
    }
    return tanimoto_kernel(X, rows_x, Y, rows_y, words, K, ldk, out_dtype, as_stream(stream));
}

gvt_status gvt_factor_cache_begin(gvt_handle* h)
{
    if (!h) {
        set_error("gvt_factor_cache_begin: NULL handle");
        return GVT_ERR_INVALID_ARG;
    }
    ++h->factor_cache_depth;
    return GVT_OK;
}

gvt_status gvt_factor_cache_end(gvt_handle* h)
{
    if (!h || h->factor_cache_depth <= 0) {
        set_error("gvt_factor_cache_end: NULL handle or no open scope");
        return GVT_ERR_INVALID_ARG;
    }
    if (--h->factor_cache_depth == 0)
        for (auto& e : h->factor_cache) e.valid = false;
    return GVT_OK;
}

gvt_status gvt_set_tc_pairs(gvt_handle* h, int32_t mode)
{
    if (!h || mode < GVT_TC_PAIRS_AUTO || mode > GVT_TC_PAIRS_ON) {
        set_error("gvt_set_tc_pairs: bad handle or mode");
        return GVT_ERR_INVALID_ARG;
    }
    h->tc_pairs = mode;
    return GVT_OK;
}

gvt_status gvt_set_stage1_engine(gvt_handle* h, int32_t engine)
{
    if (!h || engine < GVT_STAGE1_SIMT || engine > GVT_STAGES_TC_F16X1) {
        set_error("gvt_set_stage1_engine: bad handle or engine");
        return GVT_ERR_INVALID_ARG;
    }
    h->stage1_engine = engine;
    return GVT_OK;
}

gvt_status gvt_check_device_errors(gvt_handle* h, void* stream)
{
    if (!h) {
        set_error("gvt_check_device_errors: handle is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t s = as_stream(stream);
    int word = 0;
    GVT_CUDA(cudaMemcpyAsync(&word, handle_err_word(h), sizeof(int), cudaMemcpyDeviceToHost, s));
    GVT_CUDA(cudaStreamSynchronize(s));
    if (word != 0) {
        GVT_CUDA(cudaMemsetAsync(handle_err_word(h), 0, sizeof(int), s));
        GVT_CUDA(cudaStreamSynchronize(s));
        set_error("a bounded wait in a tensor-core kernel expired; its results are invalid");
        return (gvt_status)word;
    }
    return GVT_OK;
}

gvt_status gvt_tc_gemm_bf16(gvt_handle* h, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                            int64_t ldc, int64_t M, int64_t N, int64_t K, void* stream)
{
    if (!h || (M > 0 && N > 0 && (!A || !B || !C))) {
        set_error("gvt_tc_gemm_bf16: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    return tc_gemm_bf16(A, lda, B, ldb, C, ldc, M, N, K, handle_err_word(h), as_stream(stream), h->tc_pairs,
                        h->tc_stall_cycles);
}

gvt_status gvt_set_stage_tiles(gvt_handle* h, int32_t mode)
{
    if (!h || mode < GVT_TILES_AUTO || mode > GVT_TILES_ON) {
        set_error("gvt_set_stage_tiles: bad handle or mode");
        return GVT_ERR_INVALID_ARG;
    }
    h->stage_tiles = mode;
    return GVT_OK;
}

gvt_status gvt_set_tc_stall_test(gvt_handle* h, int64_t cycles)
{
    if (!h || cycles < 0 || cycles > 4000000000ll) {
        set_error("gvt_set_tc_stall_test: bad handle or cycle count (0 .. 4e9)");
        return GVT_ERR_INVALID_ARG;
    }
    h->tc_stall_cycles = cycles;
    return GVT_OK;
}

gvt_status gvt_convert(const void* src, int32_t src_dtype, void* dst, int32_t dst_dtype, int64_t n,
                       void* stream)
{
    if (n < 0 || (n > 0 && (!src || !dst))) {
        set_error("gvt_convert: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    return convert(src, src_dtype, dst, dst_dtype, n, as_stream(stream));
}

gvt_status gvt_stats_enable(gvt_handle* h, int32_t on)
{
    if (!h) {
        set_error("gvt_stats_enable: handle is NULL");
        return GVT_ERR_INVALID_ARG;
    }
    for (auto& r : h->recs) {
        cudaEventSynchronize(r.e1);
        h->event_pool.push_back(r.e0);
        h->event_pool.push_back(r.e1);
    }
    h->recs.clear();
    h->stats_on = on != 0;
    return GVT_OK;
}

gvt_status gvt_stats_read(gvt_handle* h, gvt_kernel_stats* out)
{
    if (!h || !out) {
        set_error("gvt_stats_read: NULL argument");
        return GVT_ERR_INVALID_ARG;
    }
    for (int k = 0; k < GVT_STAT_COUNT; ++k) out[k] = gvt_kernel_stats{0, 0.0, 0.0, 0.0, 0.0};
    for (auto& r : h->recs) {
        GVT_CUDA(cudaEventSynchronize(r.e1));
        float ms = 0.f;
        GVT_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
        gvt_kernel_stats& o = out[r.kind];
        o.launches += 1;
        o.ms += ms;
        o.flops += r.flops;
        o.bytes += r.bytes;
        o.useful_flops += r.useful;
    }
    return GVT_OK;
}

int64_t gvt_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
