// gl_peaks.cu -- measured peaks of this GPU for the rooflines: the FP64 or FP32
// fused multiply-add rate, from a kernel of independent FMA chains timed with
// CUDA events (no datasheet figure), and the latencies that bound one phase of
// the coarse-level Gauss-Seidel sweeps (a release/acquire hand-off between two
// CTAs, a dependent L2 load, a GPU-scope fence after a store).  The FP64 Jacobian
// and coarse sweeps of the FP64 solve and the double-FP32 Jacobian of the mixed
// solve are bounded by the pipes rather than by HBM on this GPU; the coarse
// sweeps by the latencies.
#include <algorithm>
#include <vector>

#include "gl_internal.cuh"

namespace gl {

constexpr int PEAK_CHAINS = 8;  // independent accumulators per thread

template <typename R>
__global__ void __launch_bounds__(256) k_fma_peak(int64_t reps, R a, R b, R *sink) {
    R acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int64_t r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = fma(acc[k], a, b);
    }
    R t = 0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) t += acc[k];
    if (t == (R)-12345.0) *sink = t;  // keeps the chains live
}

template <typename R>
static double fma_peak_gflops(cudaStream_t s) {
    int dev = 0, nsm = 0, per_sm = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<R>, 256, 0));
    const int grid = nsm * std::max(per_sm, 1);
    DBuf<R> sink(1);
    cudaEvent_t e0, e1;
    GL_CUDA(cudaEventCreate(&e0));
    GL_CUDA(cudaEventCreate(&e1));
    // grow the repetition count until one launch takes at least 20 ms
    int64_t reps = 1 << 12;
    double best = 0;
    for (int trial = 0; trial < 12; ++trial) {
        k_fma_peak<R><<<grid, 256, 0, s>>>(reps, (R)0.999999, (R)1e-7, sink.get());
        GL_CUDA(cudaEventRecord(e0, s));
        k_fma_peak<R><<<grid, 256, 0, s>>>(reps, (R)0.999999, (R)1e-7, sink.get());
        GL_CUDA(cudaEventRecord(e1, s));
        GL_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        GL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double flops = 2.0 * (double)grid * 256 * PEAK_CHAINS * (double)reps;
        best = std::max(best, flops / (ms * 1e-3) / 1e9);
        if (ms >= 20.f) break;
        reps *= 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// ---- latencies
// Every spin below gives up after SPIN_NS of the global timer and sets *err.
constexpr unsigned long long SPIN_NS = 1000000000ull;
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acq(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ bool wait_geq(const unsigned long long *p, unsigned long long want, int *err) {
    const unsigned long long t0 = gtimer();
    for (unsigned k = 0;; ++k) {
        if (ld_acq(p) >= want) return true;
        if ((k & 63u) == 63u && gtimer() - t0 > SPIN_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
}

// CTA 0 and CTA `partner` (one CTA per SM: the launch asks for more than half
// an SM's shared memory; cooperative, so both are resident) pass a counter back
// and forth `rounds` times with release stores and acquiring loads, as the
// neighbour-flag sweep does; CTA 0 records the mean one-way hand-off in ns.
// flags[0], flags[1]: the two counters, starting at base.
__global__ void k_pingpong(int partner, int rounds, unsigned long long base, unsigned long long *flags,
                           double *out, int *err) {
    extern __shared__ char keep_alone[];  // only sizes the launch
    if (threadIdx.x != 0) return;
    if (blockIdx.x == 0) {
        const unsigned long long t0 = gtimer();
        for (int i = 1; i <= rounds; ++i) {
            st_rel(flags, base + i);
            if (!wait_geq(flags + 1, base + i, err)) return;
        }
        out[partner] = (double)(gtimer() - t0) / (2.0 * rounds);
        keep_alone[0] = 0;
    } else if ((int)blockIdx.x == partner) {
        for (int i = 1; i <= rounds; ++i) {
            if (!wait_geq(flags, base + i, err)) return;
            st_rel(flags + 1, base + i);
        }
    }
}

// one thread: `reps` dependent L2 loads along a chain through `next` (out[0], ns
// per load), then `reps` stores each followed by a GPU-scope fence (out[1])
__global__ void k_chase(const unsigned *next, int reps, unsigned *scratch, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned j = 0;
    for (int i = 0; i < reps; ++i) j = __ldcg(next + j);  // brings the chain into L2
    unsigned long long t0 = gtimer();
    for (int i = 0; i < reps; ++i) j = __ldcg(next + j);
    unsigned long long t1 = gtimer();
    out[0] = (double)(t1 - t0) / reps;
    t0 = gtimer();
    for (int i = 0; i < reps; ++i) {
        scratch[(i * 32 + j) & 4095] = (unsigned)i;
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    t1 = gtimer();
    out[1] = (double)(t1 - t0) / reps;
    scratch[4096] = j;
}
// next[i] = (i * 40505 + 7) mod n over n = 2^18 words (1 MiB): a full-period
// linear congruential chain (a = 1 mod 4, c odd), consecutive loads on lines far
// apart
__global__ void k_chase_init(unsigned *next, unsigned n) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) next[i] = (unsigned)(((unsigned long long)i * 40505ull + 7ull) % n);
}

static void sync_latency(double *res, cudaStream_t s) {
    int dev = 0, nsm = 0, smem_max = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GL_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int smem = smem_max / 2 + 1024;  // at most one CTA per SM
    GL_CUDA(cudaFuncSetAttribute(k_pingpong, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    GL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pingpong, 32, smem));
    GL_REQUIRE(per_sm == 1, GL_ERR_CUDA, "hand-off probe: expected one CTA per SM");
    const int rounds = 200;
    DBuf<unsigned long long> flags(2);
    DBuf<double> out(nsm);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(flags.get(), 0, 2 * sizeof(unsigned long long), s));
    GL_CUDA(cudaMemsetAsync(out.get(), 0, nsm * sizeof(double), s));
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    for (int p = 1; p < nsm; ++p) {
        unsigned long long base = (unsigned long long)(p - 1) * rounds;
        unsigned long long *fp = flags.get();
        double *op = out.get();
        int *ep = err.get();
        void *args[] = {&p, (void *)&rounds, &base, &fp, &op, &ep};
        GL_CUDA(cudaLaunchCooperativeKernel((void *)k_pingpong, dim3(nsm), dim3(32), args, smem, s));
    }
    std::vector<double> h(nsm);
    int e = 0;
    GL_CUDA(cudaMemcpyAsync(h.data(), out.get(), nsm * sizeof(double), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaMemcpyAsync(&e, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(e == 0, GL_ERR_TIMEOUT, "hand-off probe: a wait ran out");
    std::vector<double> v(h.begin() + 1, h.end());
    std::sort(v.begin(), v.end());
    res[0] = v[v.size() / 2];
    res[1] = v.back();
    const unsigned n = 1u << 18;
    DBuf<unsigned> next(n), scratch(4097);
    DBuf<double> o2(2);
    k_chase_init<<<(n + 255) / 256, 256, 0, s>>>(next.get(), n);
    k_chase<<<1, 32, 0, s>>>(next.get(), 4096, scratch.get(), o2.get());
    GL_LAUNCH_CHECK();
    double hh[2];
    GL_CUDA(cudaMemcpyAsync(hh, o2.get(), sizeof(hh), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    res[2] = hh[0];
    res[3] = hh[1];
}

}  // namespace gl

extern "C" gl_status gl_measure_sync_latency(double *ns4, void *stream) {
    try {
        gl::set_error("");
        GL_REQUIRE(ns4, GL_ERR_ARG, "NULL argument");
        gl::sync_latency(ns4, reinterpret_cast<cudaStream_t>(stream));
        return GL_OK;
    } catch (const gl::Error &e) {
        gl::set_error(e.msg);
        return e.code;
    } catch (const std::exception &e) {
        gl::set_error(e.what());
        return GL_ERR_CUDA;
    }
}

extern "C" gl_status gl_measure_fma_peak(int precision, double *gflops, void *stream) {
    try {
        gl::set_error("");
        GL_REQUIRE(gflops, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(precision == GL_FP64 || precision == GL_MIXED, GL_ERR_ARG, "precision must be GL_FP64 or GL_MIXED");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        *gflops = precision == GL_FP64 ? gl::fma_peak_gflops<double>(s) : gl::fma_peak_gflops<float>(s);
        return GL_OK;
    } catch (const gl::Error &e) {
        gl::set_error(e.msg);
        return e.code;
    } catch (const std::exception &e) {
        gl::set_error(e.what());
        return GL_ERR_CUDA;
    }
}
