// gl_ops.cu -- the fused sliced-ELL operators of the discrete GL problem in the
// solve ordering (red nodes first, then black):
//   Jacobian (Sec. 3): y_i = (K phi)_i + (-1 + 2|psi_i|^2) phi_i + psi_i^2 conj(phi_i)
//   residual (Eq. discr ginla): r_i = (K psi)_i - psi_i (1 - |psi_i|^2)
// with K = D^-1 K-hat (Remark rmk:dk) stored as off-diagonals + diagonal.
#include "gl_internal.cuh"
#include "gl_kernels.cuh"

namespace gl {

__global__ void k_gather(int64_t n, const int32_t *__restrict__ perm, const double2 *__restrict__ nat,
                         double2 *__restrict__ sol) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) sol[p] = nat[perm[p]];
}
__global__ void k_scatter(int64_t n, const int32_t *__restrict__ perm, const double2 *__restrict__ sol,
                          double2 *__restrict__ nat) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) nat[perm[p]] = sol[p];
}

void permute_in(int64_t n, const int32_t *perm, const double2 *nat, double2 *sol, cudaStream_t s) {
    k_gather<<<grid_for(n, 256), 256, 0, s>>>(n, perm, nat, sol);
    GL_LAUNCH_CHECK();
}
void permute_out(int64_t n, const int32_t *perm, const double2 *sol, double2 *nat, cudaStream_t s) {
    k_scatter<<<grid_for(n, 256), 256, 0, s>>>(n, perm, sol, nat);
    GL_LAUNCH_CHECK();
}

// y = J(psi) phi, FP64
__global__ void k_jacobian64(int64_t n, SellView<double2> K, const double *__restrict__ kdiag,
                             const double2 *__restrict__ psi, const double2 *__restrict__ phi,
                             double2 *__restrict__ y) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double2 acc = sell_row<double2, double2>(K, p, phi);
    y[p] = jacobian_epilogue(acc, kdiag[p], psi[p], phi[p]);
}

// the same from the FP64 lattice tables (meshes whose stored K matches them)
__global__ void k_jacobian_lat64(int64_t n, LatticeView64 L, const double *__restrict__ kdiag,
                                 const double2 *__restrict__ psi, const double2 *__restrict__ phi,
                                 double2 *__restrict__ y) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double2 acc = lattice_row64(L, p, phi);
    y[p] = jacobian_epilogue(acc, kdiag[p], psi[p], phi[p]);
}

// y = J(psi) phi with the FP32 operator and FP32 arithmetic (FP64 in/out)
__global__ void k_jacobian32(int64_t n, SellView<float2> K, const float *__restrict__ kdiag,
                             const double2 *__restrict__ psi, const double2 *__restrict__ phi,
                             double2 *__restrict__ y) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < w; ++k) {
        int64_t q = beg + (int64_t)k * SELL_C + lane;
        cfma(acc, K.val[q], to32(phi[K.col[q]]));
    }
    float2 r = jacobian_epilogue(acc, kdiag[p], to32(psi[p]), to32(phi[p]));
    y[p] = to64(r);
}

// r = GL(psi), FP64
__global__ void k_residual64(int64_t n, SellView<double2> K, const double *__restrict__ kdiag,
                             const double2 *__restrict__ psi, double2 *__restrict__ r) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double2 acc = sell_row<double2, double2>(K, p, psi);
    double2 ps = psi[p];
    double a2 = ps.x * ps.x + ps.y * ps.y;
    // (K psi)_i - psi_i (1 - |psi_i|^2) = offdiag + (K_ii - 1 + |psi_i|^2) psi_i
    double d = kdiag[p] - 1.0 + a2;
    r[p] = mk(acc.x + d * ps.x, acc.y + d * ps.y);
}

// Newton right-hand side (Eq. Newton system): r <- -r in place, with per-block
// partials of ||r||_R^2 = sum |V_i| |r_i|^2
__global__ void k_negate_norm(int64_t n, const double *__restrict__ vol, double2 *__restrict__ r, double *part) {
    __shared__ double sh[32];
    double a = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = r[i];
        a += vol[i] * (v.x * v.x + v.y * v.y);
        r[i] = make_double2(-v.x, -v.y);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_sum_parts_sqrt(const double *part, int np, double *out) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) *out = sqrt(t);
}
// psi <- psi + d
__global__ void k_axpy64(int64_t n, const double2 *__restrict__ d, double2 *__restrict__ psi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) psi[i] = cadd(psi[i], d[i]);
}

double newton_rhs(const gl_mesh_s *m, double2 *r, double *part, double *scal, cudaStream_t s) {
    k_negate_norm<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->n, m->vol.get(), r, part);
    k_sum_parts_sqrt<<<1, 1024, 0, s>>>(part, RED_BLOCKS, scal);
    GL_LAUNCH_CHECK();
    double g = 0;
    GL_CUDA(cudaMemcpyAsync(&g, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return g;
}
void newton_update(int64_t n, const double2 *d, double2 *psi, cudaStream_t s) {
    k_axpy64<<<grid_for(n, 256), 256, 0, s>>>(n, d, psi);
    GL_LAUNCH_CHECK();
}

void jacobian_apply_p(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s) {
    k_jacobian64<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, m->K.view(), m->kdiag.get(), psi, phi, y);
    GL_LAUNCH_CHECK();
}
// the same matrix-free from the lattice stencil's FP64 tables (meshes whose stored
// K matches them to 16 ulp of its largest entry: the same operator up to rounding)
void jacobian_apply_lat64_p(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s) {
    GL_REQUIRE(m->lat64_ok, GL_ERR_ARG, "the mesh has no FP64 lattice stencil (odd N, or K does not match it)");
    k_jacobian_lat64<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, lattice_view64(m), m->kdiag.get(), psi, phi, y);
    GL_LAUNCH_CHECK();
}
void jacobian_apply_p32(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s) {
    k_jacobian32<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, m->K32.view(), m->kdiag32.get(), psi, phi, y);
    GL_LAUNCH_CHECK();
}
void residual_p(const gl_mesh_s *m, const double2 *psi, double2 *r, cudaStream_t s) {
    k_residual64<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, m->K.view(), m->kdiag.get(), psi, r);
    GL_LAUNCH_CHECK();
}

}  // namespace gl
