// gl_prims.cu -- device-wide primitives used by the setup kernels: exclusive
// scan, deterministic sums/maxima, and per-row sorting of short sparse rows.
#include "gl_common.cuh"
#include "gl_profile.cuh"

namespace gl {

namespace {
thread_local std::string g_err;
}
void set_error(const std::string &msg) { g_err = msg; }
const char *last_error() { return g_err.c_str(); }

Profiler &profiler() {
    static Profiler p;
    return p;
}

Scratch &scratch() {
    static thread_local Scratch s;
    return s;
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_T = 256, SCAN_E = 4, SCAN_TILE = SCAN_T * SCAN_E;

// per-tile exclusive scan; writes the tile total to sums[blockIdx.x]
__global__ void k_scan_tile(const int64_t *in, int64_t *out, int64_t n, int64_t *sums) {
    __shared__ int64_t sh[SCAN_T];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_E;
    int64_t v[SCAN_E], run = 0;
    for (int e = 0; e < SCAN_E; ++e) {
        int64_t i = base + e;
        v[e] = (i < n) ? in[i] : 0;
        run += v[e];
    }
    sh[threadIdx.x] = run;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {  // Hillis-Steele on thread totals
        int64_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t excl = sh[threadIdx.x] - run;
    for (int e = 0; e < SCAN_E; ++e) {
        int64_t i = base + e;
        if (i < n) out[i] = excl;
        excl += v[e];
    }
    if (threadIdx.x == SCAN_T - 1) sums[blockIdx.x] = sh[SCAN_T - 1];
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *offs) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t add = offs[blockIdx.x];
    for (int e = threadIdx.x; e < SCAN_TILE; e += SCAN_T) {
        int64_t i = base + e;
        if (i < n) out[i] += add;
    }
}

__global__ void k_set_total(int64_t *out, int64_t n, const int64_t *last_in_copy, const int64_t *last_out) {
    out[n] = *last_out + *last_in_copy;
}

__global__ void k_copy1(const int64_t *src, int64_t *dst) { *dst = *src; }

static void scan_rec(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    DBuf<int64_t> sums(tiles + 1);
    k_scan_tile<<<(unsigned)tiles, SCAN_T, 0, s>>>(in, out, n, sums.get());
    GL_LAUNCH_CHECK();
    if (tiles > 1) {
        scan_rec(sums.get(), sums.get(), tiles, s);
        k_scan_add<<<(unsigned)tiles, SCAN_T, 0, s>>>(out, n, sums.get());
        GL_LAUNCH_CHECK();
    }
    // keep sums alive until the kernels using it are done
    GL_CUDA(cudaStreamSynchronize(s));
}

void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, bool with_total, cudaStream_t s) {
    if (n <= 0) {
        if (with_total) GL_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    DBuf<int64_t> last(1);
    if (with_total) {
        k_copy1<<<1, 1, 0, s>>>(in + n - 1, last.get());
        GL_LAUNCH_CHECK();
    }
    scan_rec(in, out, n, s);
    if (with_total) {
        k_set_total<<<1, 1, 0, s>>>(out, n, last.get(), out + n - 1);
        GL_LAUNCH_CHECK();
        GL_CUDA(cudaStreamSynchronize(s));
    }
}

// ------------------------------------------------------------------ reductions
__global__ void k_sum_i64(const int64_t *in, int64_t n, int64_t *part) {
    __shared__ int64_t sh[256];
    int64_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += in[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

int64_t reduce_sum_i64(const int64_t *in, int64_t n, cudaStream_t s) {
    const int G = 256;
    DBuf<int64_t> part(G);
    k_sum_i64<<<G, 256, 0, s>>>(in, n, part.get());
    GL_LAUNCH_CHECK();
    std::vector<int64_t> h(G);
    GL_CUDA(cudaMemcpyAsync(h.data(), part.get(), G * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    int64_t t = 0;
    for (auto x : h) t += x;
    return t;
}

__global__ void k_max_abs(const double *in, int64_t n, double *part) {
    __shared__ double sh[256];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fmax(acc, fabs(in[i]));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

double reduce_max_abs(const double *in, int64_t n, cudaStream_t s) {
    const int G = 256;
    DBuf<double> part(G);
    k_max_abs<<<G, 256, 0, s>>>(in, n, part.get());
    GL_LAUNCH_CHECK();
    std::vector<double> h(G);
    GL_CUDA(cudaMemcpyAsync(h.data(), part.get(), G * sizeof(double), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    double t = 0;
    for (auto x : h) t = std::fmax(t, x);
    return t;
}

__global__ void k_count_u8(const uint8_t *in, int64_t n, int64_t *part) {
    __shared__ int64_t sh[256];
    int64_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += in[i] ? 1 : 0;
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

int64_t count_nonzero_u8(const uint8_t *in, int64_t n, cudaStream_t s) {
    const int G = 256;
    DBuf<int64_t> part(G);
    k_count_u8<<<G, 256, 0, s>>>(in, n, part.get());
    GL_LAUNCH_CHECK();
    std::vector<int64_t> h(G);
    GL_CUDA(cudaMemcpyAsync(h.data(), part.get(), G * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    int64_t t = 0;
    for (auto x : h) t += x;
    return t;
}

// ------------------------------------------------------------------ per-row sort
// Short rows (<= 32): one thread per row, insertion sort.  Longer rows: one block
// per row, bitonic sort of (key, index) in shared memory, then payload gather.
__global__ void k_sort_rows_small(int64_t nrows, const int64_t *rp, int32_t *ci, double2 *v) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int64_t lo = rp[r], hi = rp[r + 1];
    if (hi - lo > 32) return;
    for (int64_t a = lo + 1; a < hi; ++a) {
        int32_t k = ci[a];
        double2 val = v[a];
        int64_t b = a - 1;
        while (b >= lo && ci[b] > k) {
            ci[b + 1] = ci[b];
            v[b + 1] = v[b];
            --b;
        }
        ci[b + 1] = k;
        v[b + 1] = val;
    }
}

__global__ void k_sort_rows_large(int64_t nrows, const int64_t *rp, int32_t *ci, double2 *v, int cap) {
    extern __shared__ unsigned char smem[];
    int64_t *key = reinterpret_cast<int64_t *>(smem);  // (col << 32 | original slot)
    double2 *tmp = reinterpret_cast<double2 *>(key + cap);
    int64_t r = blockIdx.x;
    int64_t lo = rp[r], hi = rp[r + 1];
    int len = (int)(hi - lo);
    if (len <= 32) return;
    int p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x)
        key[i] = (i < len) ? (((int64_t)ci[lo + i]) << 32 | (int64_t)i) : INT64_MAX;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = ((i & k) == 0);
                    int64_t a = key[i], b = key[ixj];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += blockDim.x) tmp[i] = v[lo + (key[i] & 0xffffffff)];
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        ci[lo + i] = (int32_t)(key[i] >> 32);
        v[lo + i] = tmp[i];
    }
}

void sort_rows_by_col(int64_t nrows, const int64_t *rp, int32_t *ci, double2 *v, int64_t max_row, cudaStream_t s) {
    if (nrows <= 0) return;
    k_sort_rows_small<<<grid_for(nrows, 128), 128, 0, s>>>(nrows, rp, ci, v);
    GL_LAUNCH_CHECK();
    if (max_row > 32) {
        int cap = 1;
        while (cap < max_row) cap <<= 1;
        size_t sm = (size_t)cap * (sizeof(int64_t) + sizeof(double2));
        GL_REQUIRE(sm <= 200 * 1024, GL_ERR_CAPACITY, "sort_rows_by_col: row too long");
        GL_CUDA(cudaFuncSetAttribute(k_sort_rows_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_sort_rows_large<<<(unsigned)nrows, 256, sm, s>>>(nrows, rp, ci, v, cap);
        GL_LAUNCH_CHECK();
    }
}

}  // namespace gl
