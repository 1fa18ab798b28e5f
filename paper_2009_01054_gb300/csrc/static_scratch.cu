// gvt_matvec_static: the Kronecker product u = R(dhat,that)(M kron N)R(d,t)^T v
// without any device allocation.
//
// Some callers cannot call cudaMalloc: applications whose framework owns all
// device memory through its own pool (a cudaMalloc would fail or fragment the
// pool), and latency-bound loops in which cudaMalloc / cudaFree, which can
// synchronise the device, are not allowed.  gvt_matvec needs a plan and a
// handle, both of which allocate.  This entry point needs neither: its only
// scratch -- the intermediate S of the two-stage product and one error word --
// lives in a fixed-size __device__ array of this library, which every device
// that loads the library keeps until the process exits.
//
// Without a plan there are no sorted segments, so stage 1 accumulates S with
// atomic adds (sums in run-dependent order, within rounding of gvt_matvec) and
// stage 2 reads S rows directly.
#include <mutex>

#include "gvt_internal.h"

namespace gvt {
namespace {

constexpr size_t kStaticBytes = GVT_STATIC_SCRATCH_BYTES;
constexpr size_t kStaticHeader = 256;   // error word(s), then S
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  The first call
// on a device looks it up with cudaGetSymbolAddress (a host-side use of the
// symbol's name would only give a host stand-in, not a device address).
gvt_status static_scratch(void** out)
{
    int dev = 0;
    GVT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gvt_matvec_static: device ordinal out of range");
        return GVT_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            if (e == cudaSuccess) e = cudaErrorInvalidSymbol;
            return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return GVT_OK;
}

__global__ void static_zero_kernel(unsigned long long* __restrict__ words, int64_t n_words)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words;
         i += (int64_t)gridDim.x * blockDim.x)
        words[i] = 0ull;
}

// Stage 1: S[y, d_j] += N[y, t_j] * v_j for every input pair, one warp per pair.
// Pairs with an id outside M's columns or N's columns are counted in *bad and skipped.
template <class T>
__global__ void static_stage1_kernel(const T* __restrict__ N, int64_t ldn, int n_sym,
                                     const int32_t* __restrict__ d, const int32_t* __restrict__ t,
                                     int64_t n, const T* __restrict__ v, int64_t X, int64_t Y,
                                     int64_t t_range, T* __restrict__ S, unsigned int* __restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += nw) {
        const int32_t dj = d[j], tj = t[j];
        if (dj < 0 || dj >= X || tj < 0 || tj >= t_range) {
            if (lane == 0) atomicAdd(bad, 1u);
            continue;
        }
        const T vj = v[j];
        for (int64_t y = lane; y < Y; y += 32) {
            const T b = n_sym ? N[(int64_t)tj * ldn + y] : N[y * ldn + tj];
            atomicAdd(&S[y * X + dj], b * vj);
        }
    }
}

// Stage 2: u_i = <M[dhat_i, :X], S[that_i, :]>, one warp per output pair.
template <class T>
__global__ void static_stage2_kernel(const T* __restrict__ M, int64_t ldm, int64_t m_rows,
                                     const int32_t* __restrict__ d, const int32_t* __restrict__ t,
                                     int64_t n, const T* __restrict__ S, int64_t X, int64_t Y,
                                     T* __restrict__ u, unsigned int* __restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int32_t a = d[i], b = t[i];
        if (a < 0 || a >= m_rows || b < 0 || b >= Y) {
            if (lane == 0) {
                atomicAdd(bad, 1u);
                u[i] = T(0);
            }
            continue;
        }
        const T* mrow = M + (int64_t)a * ldm;
        const T* srow = S + (int64_t)b * X;
        T acc = T(0);
        for (int64_t x = lane; x < X; x += 32) acc = fma(mrow[x], srow[x], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) u[i] = acc;
    }
}

unsigned warp_grid(int64_t n)
{
    int64_t g = (n + 7) / 8;   // 8 warps per 256-thread block
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

template <class T>
gvt_status run_static(int64_t m_rows, int64_t m_cols, int64_t q_rows, int64_t q_cols,
                      const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                      const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                      const gvt_matrix* M, const gvt_matrix* N, const T* v, T* u, cudaStream_t s)
{
    const int64_t X = m_cols, Y = q_rows;
    // Y * X elements must fit the scratch after its header; compare by division so that large
    // declared sizes cannot wrap the product.
    const uint64_t cap_elems = (kStaticBytes - kStaticHeader) / sizeof(T);
    if (X > 0 && (uint64_t)Y > cap_elems / (uint64_t)X) {
        set_error("gvt_matvec_static: q_rows * m_cols = " + std::to_string(Y) + " * " + std::to_string(X) +
                  " elements exceed the static scratch of " + std::to_string(kStaticBytes - kStaticHeader) +
                  " bytes");
        return GVT_ERR_INVALID_ARG;
    }
    const size_t s_bytes = sizeof(T) * (size_t)X * (size_t)Y;
    void* base = nullptr;
    GVT_CHECK(static_scratch(&base));
    unsigned int* bad = static_cast<unsigned int*>(base);
    T* S = reinterpret_cast<T*>(static_cast<char*>(base) + kStaticHeader);
    // The array keeps the previous call's contents: clear the error word and S.
    const int64_t words = (int64_t)((kStaticHeader + s_bytes + 7) / 8);
    static_zero_kernel<<<warp_grid(words * 4), 256, 0, s>>>(static_cast<unsigned long long*>(base), words);
    GVT_LAUNCH_CHECK("static zero");
    // Column t of N: row t when N is symmetric, else a strided column read.
    const int n_sym = (N->symmetric && N->rows == N->cols) ? 1 : 0;
    static_stage1_kernel<T><<<warp_grid(n_in), 256, 0, s>>>(
        static_cast<const T*>(N->data), N->ld, n_sym, d_in, t_in, n_in, v, X, Y, q_cols, S, bad);
    GVT_LAUNCH_CHECK("static stage 1");
    static_stage2_kernel<T><<<warp_grid(n_out), 256, 0, s>>>(
        static_cast<const T*>(M->data), M->ld, m_rows, d_out, t_out, n_out, S, X, Y, u, bad);
    GVT_LAUNCH_CHECK("static stage 2");
    unsigned int hbad = 0;
    GVT_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
    GVT_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        set_error("gvt_matvec_static: " + std::to_string(hbad) +
                  " pair(s) with an index outside the kernel matrices were skipped");
        return GVT_ERR_INDEX_OOB;
    }
    return GVT_OK;
}

}  // namespace
}  // namespace gvt

using namespace gvt;

extern "C" gvt_status gvt_matvec_static(int64_t m_rows, int64_t m_cols, int64_t q_rows, int64_t q_cols,
                                        const int32_t* d_in, const int32_t* t_in, int64_t n_in,
                                        const int32_t* d_out, const int32_t* t_out, int64_t n_out,
                                        const gvt_matrix* M, const gvt_matrix* N, const void* v, void* u,
                                        int32_t dtype, void* stream)
{
    if (!M || !N || !M->data || !N->data || m_rows < 0 || m_cols < 0 || q_rows < 0 || q_cols < 0 ||
        n_in < 0 || n_out < 0) {
        set_error("gvt_matvec_static: bad argument");
        return GVT_ERR_INVALID_ARG;
    }
    if (dtype != GVT_F64 && dtype != GVT_F32) {
        set_error("gvt_matvec_static: dtype must be GVT_F64 or GVT_F32");
        return GVT_ERR_UNSUPPORTED;
    }
    if (M->dtype != dtype || N->dtype != dtype || M->rows < m_rows || M->cols < m_cols ||
        N->rows < q_rows || N->cols < q_cols) {
        set_error("gvt_matvec_static: M or N has the wrong dtype or is smaller than the id ranges");
        return GVT_ERR_INVALID_ARG;
    }
    if (d_out == nullptr && t_out == nullptr) {
        d_out = d_in;
        t_out = t_in;
        n_out = n_in;
    }
    if ((n_in > 0 && (!d_in || !t_in || !v)) || (n_out > 0 && (!d_out || !t_out || !u))) {
        set_error("gvt_matvec_static: NULL array");
        return GVT_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == GVT_F64)
        return run_static<double>(m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in, d_out, t_out, n_out, M,
                                  N, static_cast<const double*>(v), static_cast<double*>(u), s);
    return run_static<float>(m_rows, m_cols, q_rows, q_cols, d_in, t_in, n_in, d_out, t_out, n_out, M, N,
                             static_cast<const float*>(v), static_cast<float*>(u), s);
}
