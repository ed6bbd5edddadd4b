// gl_common.cuh -- internal declarations of the GB300 Ginzburg-Landau Jacobian
// solver: complex helpers, the sliced-ELL layout, device buffers, error state,
// and the primitives (scan, deterministic reductions) shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/gl.h"

namespace gl {

// ---------------------------------------------------------------- errors
// GL_VERBOSE=1 in the environment: setup decisions are reported on stderr
inline bool verbose() {
    static const bool v = [] {
        const char *e = std::getenv("GL_VERBOSE");
        return e && e[0] && e[0] != '0';
    }();
    return v;
}
void set_error(const std::string &msg);
const char *last_error();

struct Error {
    gl_status code;
    std::string msg;
};

#define GL_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            throw ::gl::Error{e_ == cudaErrorMemoryAllocation ? GL_ERR_OOM : GL_ERR_CUDA,        \
                              std::string(#call) + ": " + cudaGetErrorString(e_)};               \
    } while (0)

#define GL_LAUNCH_CHECK() GL_CUDA(cudaGetLastError())

#define GL_REQUIRE(cond, code, msg)                                                              \
    do {                                                                                         \
        if (!(cond)) throw ::gl::Error{code, msg};                                               \
    } while (0)

// ---------------------------------------------------------------- device memory
// Owning device buffer (cudaMalloc / cudaFree), move-only.
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr, o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count) GL_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------- complex helpers
template <typename R>
struct CT;
template <>
struct CT<double> {
    using type = double2;
};
template <>
struct CT<float> {
    using type = float2;
};
template <typename R>
using cplx_t = typename CT<R>::type;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename C>
__host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C>
__host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
template <typename C>
__host__ __device__ __forceinline__ C cmulc(C a, C b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
template <typename C, typename R>
__host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
template <typename C>
__host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// acc += a * b (complex fused multiply-add)
template <typename C>
__host__ __device__ __forceinline__ void cfma(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 to32(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to64(float2 a) { return make_double2(a.x, a.y); }

// ---------------------------------------------------------------- CSR (canonical numbering)
struct CsrDev {
    int64_t n = 0, m = 0, nnz = 0;
    DBuf<int64_t> rp;
    DBuf<int32_t> ci;
    DBuf<double2> v;
};

// ---------------------------------------------------------------- sliced ELL
// Rows are grouped in slices of SELL_C = 32 consecutive rows (one warp).  Slice s
// stores width_s x 32 entries column-major: entry k of row (32 s + lane) sits at
// sptr[s] + 32 k + lane, so a warp reads 32 consecutive values per k.  Padding
// entries point at the row itself with value 0.
constexpr int SELL_C = 32;

template <typename C>
struct SellView {
    int64_t nrows;
    int64_t nslices;
    const int64_t *sptr;  // nslices + 1 entry offsets
    const int32_t *col;
    const C *val;
};

template <typename C>
struct Sell {
    int64_t nrows = 0, nslices = 0, nnz_stored = 0, nnz_real = 0;
    DBuf<int64_t> sptr;
    DBuf<int32_t> col;
    DBuf<C> val;
    SellView<C> view() const { return SellView<C>{nrows, nslices, sptr.get(), col.get(), val.get()}; }
    size_t bytes() const { return sptr.bytes() + col.bytes() + val.bytes(); }
};

// ---------------------------------------------------------------- grouped CSR
// Rows stored contiguously (CSR, off-diagonals only) and processed by groups of
// G lanes of a warp (G in {1, 2, 4, 8, 16, 32}); a group walks its row with
// stride G (coalesced) and reduces with warp shuffles.  Used for the long rows of
// the coarse levels and of the restriction.
template <typename C>
struct CsrGView {
    int64_t nrows;
    const int64_t *rp;
    const int32_t *col;
    const C *val;
};

template <typename C>
struct CsrG {
    int64_t nrows = 0, nnz = 0;
    int G = 1;
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<C> val;
    CsrGView<C> view() const { return CsrGView<C>{nrows, rp.get(), col.get(), val.get()}; }
};

// ---------------------------------------------------------------- launch helpers
constexpr int NUM_SMS_HINT = 152;
inline int grid_for(int64_t n, int block, int cap = 1 << 20) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Deterministic reductions: every reducing kernel writes one partial per block to
// a fixed-size array; the consumer sums the partials in index order.
constexpr int RED_BLOCKS = 4 * NUM_SMS_HINT;  // fixed grid of reducing vector kernels
constexpr int RED_THREADS = 256;

// block-wide sum of a double (all threads get the result in thread 0)
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += sh[i];
    }
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------- primitives (gl_prims.cu)
// exclusive scan of n int64 values (in and out may alias); out[n] = total when
// out has n + 1 entries and with_total is set.
void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, bool with_total, cudaStream_t s);
// sum of n int64 values to host (synchronises s)
int64_t reduce_sum_i64(const int64_t *in, int64_t n, cudaStream_t s);
// max of n doubles to host (synchronises s)
double reduce_max_abs(const double *in, int64_t n, cudaStream_t s);
// count of nonzero bytes (synchronises s)
int64_t count_nonzero_u8(const uint8_t *in, int64_t n, cudaStream_t s);
// per-row sort of int32 keys carrying a payload of complex values, rows given by rp
void sort_rows_by_col(int64_t nrows, const int64_t *rp, int32_t *ci, double2 *v, int64_t max_row, cudaStream_t s);

// device scratch that primitives reuse (grown on demand, per host thread)
struct Scratch {
    DBuf<uint8_t> buf;
    void *get(size_t bytes) {
        if (buf.n < bytes) buf.alloc(bytes + bytes / 2 + 1024);
        return buf.get();
    }
};
Scratch &scratch();

}  // namespace gl
