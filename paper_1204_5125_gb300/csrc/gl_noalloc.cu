// gl_noalloc.cu -- gl_jacobian_apply_noalloc: the Jacobian apply of an existing
// mesh without any device allocation.
//
// gl_jacobian_apply keeps its three reordering buffers (psi, phi and y in the
// red-black solve ordering) in per-mesh memory that it allocates with
// cudaMalloc on first use.  Some callers cannot let a call allocate:
// applications that manage a fixed device-memory budget or their own pool (an
// allocation behind their back can fail or fragment it), and latency-critical
// loops (cudaMalloc/cudaFree can synchronise the device).  This entry point
// takes the three buffers from one file-scope __device__ array instead, of a
// fixed size that every GPU loading the library holds until the process exits.
//
// Notes for callers:
//   * capacity: n <= GL_NOALLOC_MAX_NODES nodes (the array holds 3 n complex
//     doubles); larger meshes are rejected with GL_ERR_CAPACITY;
//   * the array is shared by every call on a device and keeps the last call's
//     contents; nothing in it needs to start at zero (every slot is written
//     before it is read within a call), but two calls whose work overlaps on
//     the GPU (different streams, or different host threads) race on it;
//   * the first call on each device looks up the device address of the array
//     (cudaGetSymbolAddress) with that device current; that first call should
//     come before any stream capture on the device.
#include <mutex>

#include "gl_internal.cuh"

// maximum number of mesh nodes this entry point accepts (3 x 16 B per node)
#define GL_NOALLOC_MAX_NODES (1 << 18)

namespace {

static __device__ __align__(256) double2 g_noalloc_scratch[3 * (size_t)GL_NOALLOC_MAX_NODES];

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
double2 *g_ptr[MAX_DEVICES] = {nullptr};

// device address of the scratch array on the current device (looked up once)
double2 *scratch_address() {
    int dev = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_REQUIRE(dev >= 0 && dev < MAX_DEVICES, gl_status::GL_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        GL_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_ptr[dev] = static_cast<double2 *>(p);
    }
    return g_ptr[dev];
}

}  // namespace

extern "C" gl_status gl_jacobian_apply_noalloc(gl_mesh m, const void *psi, const void *phi, void *y, void *stream) {
    try {
        gl::set_error("");
        GL_REQUIRE(m && psi && phi && y, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(y != psi && y != phi, GL_ERR_ARG, "y must not alias psi or phi");
        if (m->n > GL_NOALLOC_MAX_NODES)
            throw gl::Error{GL_ERR_CAPACITY, "gl_jacobian_apply_noalloc: mesh has " + std::to_string(m->n) +
                                                 " nodes, the static scratch holds at most " +
                                                 std::to_string(GL_NOALLOC_MAX_NODES)};
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        double2 *base = scratch_address();
        int64_t n = m->n;
        double2 *t_psi = base, *t_phi = base + n, *t_y = base + 2 * n;
        gl::permute_in(n, m->perm.get(), static_cast<const double2 *>(psi), t_psi, s);
        gl::permute_in(n, m->perm.get(), static_cast<const double2 *>(phi), t_phi, s);
        gl::jacobian_apply_p(m, t_psi, t_phi, t_y, s);
        gl::permute_out(n, m->perm.get(), t_y, static_cast<double2 *>(y), s);
        return GL_OK;
    } catch (const gl::Error &e) {
        gl::set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        gl::set_error("host allocation failed");
        return GL_ERR_OOM;
    } catch (const std::exception &e) {
        gl::set_error(e.what());
        return GL_ERR_CUDA;
    }
}
