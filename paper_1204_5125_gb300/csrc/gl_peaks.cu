// gl_peaks.cu -- measured arithmetic peaks of this GPU for the rooflines: the
// FP64 or FP32 fused multiply-add rate, from a kernel of independent FMA chains
// timed with CUDA events (no datasheet figure).  The FP64 Jacobian and coarse
// sweeps of the FP64 solve and the double-FP32 Jacobian of the mixed solve are
// bounded by these pipes rather than by HBM on this GPU.
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

}  // namespace gl

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
