// gl_solve.cu -- preconditioned MINRES (Paige & Saunders 1975) for the Newton
// system J(psi) x = b (Eq. Newton system) in the real inner product
// <x, y>_R = Re sum_i |V_i| conj(x_i) y_i (Eq. disc inner2), in which J is
// self-adjoint (Sec. 3) and R_k (Eq. prec2) is self-adjoint positive definite.
//
// The Lanczos/Givens scalars live on the device; every reduction writes one
// partial per block of a fixed grid and is summed in index order, so results do
// not depend on scheduling.  A device status word stops all kernels once the
// solve has converged or failed.  A solve is one CUDA graph that loops on the
// device (a WHILE conditional node over bodies of six iterations, the later
// ones in IF nodes that the previous iteration's scalar kernel opens), so the
// host waits once; options.device_loop = 0 replays the body graph from the host
// instead, reading the status word between replays.
//
// GL_MIXED: FP64 defect correction x <- x + e around inner MINRES solves of
// J e = r whose vectors, Jacobian applies and V-cycles are FP32 (dots and
// scalars FP64, coarsest solve FP64); the FP64 true residual decides.
#include <chrono>
#include <memory>

#include "gl_internal.cuh"
#include "gl_kernels.cuh"
#include "gl_profile.cuh"

namespace gl {

struct MinresDev {
    double gamma, gamma_old, eta, eta0, c, c_old, s, s_old;
    double delta, a1, a2, a3, c_new, eta_prev, gamma_cur;
    double bnorm, tol, est, true_rel;
    double rho0;      // ||b - J x0||_D / ||b||_D: scales the recurrence's estimate to be relative to b
    int it, maxit, check_true, status, lucky, use_true, replays;
    double stall;     // > 0: stop with ST_STALL once the estimate is below stall * tol while the true
                      // residual is still above tol (0: never)
};
enum { ST_RUN = 0, ST_CONV = 1, ST_BREAK = 2, ST_NAN = 3, ST_MAXIT = 4, ST_STALL = 5, ST_TIMEOUT = 6 };
static_assert(ST_TIMEOUT == STATUS_TIMEOUT, "the sweeps write STATUS_TIMEOUT into the status word");

template <typename T>
struct SolveOps;
template <>
struct SolveOps<double> {
    using C = double2;
    static SellView<C> K(const gl_mesh_s *m) { return m->K.view(); }
    static const double *kdiag(const gl_mesh_s *m) { return m->kdiag.get(); }
    static const double *vol(const gl_mesh_s *m) { return m->volp.get(); }
};
template <>
struct SolveOps<float> {
    using C = float2;
    static SellView<C> K(const gl_mesh_s *m) { return m->K32.view(); }
    static const float *kdiag(const gl_mesh_s *m) { return m->kdiag32.get(); }
    static const float *vol(const gl_mesh_s *m) { return m->volp32.get(); }
};

template <typename C>
__device__ __forceinline__ double redot(C a, C b) {  // Re(conj(a) b)
    return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}

// ------------------------------------------------------------------ vector kernels
// v = b - J x ; partials of <b, b>_R and <v, v>_R
template <typename C, typename R>
__global__ void __launch_bounds__(RED_THREADS) k_init_resid(int64_t n, SellView<C> K, const R *kd, const R *vol,
                                                            const C *psi, const C *b, const C *x, C *v,
                                                            double *part) {
    __shared__ double sh[32];
    double ab = 0, av = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        C acc = sell_row<C, C>(K, p, x);
        C jx = jacobian_epilogue(acc, kd[p], psi[p], x[p]);
        C bb = b[p];
        C vv = csub(bb, jx);
        v[p] = vv;
        ab += (double)vol[p] * redot(bb, bb);
        av += (double)vol[p] * redot(vv, vv);
    }
    double t = block_sum(ab, sh);
    double u = block_sum(av, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        part[RED_BLOCKS + blockIdx.x] = u;
    }
}

// partials of <x, y>_R
template <typename C, typename R>
__global__ void __launch_bounds__(RED_THREADS) k_dot(int64_t n, const R *vol, const C *x, const C *y, double *part,
                                                     const int *stop) {
    __shared__ double sh[32];
    if (*stop) return;
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        a += (double)vol[p] * redot(x[p], y[p]);
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// q = J z (z not yet normalised) ; partials of <J z, z>_R
template <typename C, typename R>
__global__ void __launch_bounds__(RED_THREADS) k_jz(int64_t n, SellView<C> K, const R *kd, const R *vol, const C *psi,
                                                    const C *z, C *q, double *part, const int *stop) {
    __shared__ double sh[32];
    if (*stop) return;
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        C acc = sell_row<C, C>(K, p, z);
        C zz = z[p];
        C jz = jacobian_epilogue(acc, kd[p], psi[p], zz);
        q[p] = jz;
        a += (double)vol[p] * redot(jz, zz);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// the same from the FP64 lattice tables (the matrix-free stencil of a lattice mesh)
__global__ void __launch_bounds__(RED_THREADS) k_jz_lat64(int64_t n, LatticeView64 L, const double *kd,
                                                          const double2 *psi, const double2 *z, double2 *q,
                                                          double *part, const int *stop) {
    __shared__ double sh[32];
    if (*stop) return;
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double2 acc = lattice_row64(L, p, z);
        const double2 zz = z[p];
        const double2 jz = jacobian_epilogue(acc, kd[p], psi[p], zz);
        q[p] = jz;
        a += L.vol[p] * redot(jz, zz);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ------------------------------------------------------------------ double-float Jacobian apply
// In the mixed-precision solve (FP64 MINRES, FP32 V-cycle) every z that meets
// the Jacobian is the FP64 image of the V-cycle's FP32 output, so its FP32 copy
// is exact.  On even-N lattices J z is then formed with FP32 arithmetic only
// (far faster than FP64 on this GPU) from double-float data (hi + lo):
//   (J z)_i = 2^b_i sum_k a_ik (z_i - u_ik z_k) + (r_i - 1 + 2|psi_i|^2) z_i + psi_i^2 conj(z_i)
// with a = |K-hat| / h^d and the unit phase u = exp(-i theta) tabulated per axis
// (gl_lattice.cu), K_ik = -2^b_i a_ik u_ik (|V_i| = h^d 2^-b_i, b_i boundary
// coordinates: an exact power-of-2 factor) and r_i = K_ii - sum_k |K_ik|.  The
// differences z_i - u z_k are formed with Knuth's error-free TwoSum after an
// FMA-based TwoProd, so a smooth z cancels without error, and products and sums
// accumulate in the compensated form of Ogita, Rump and Oishi's Dot2 (an FP32
// running sum and an FP32 compensation collecting the exact rounding errors):
// about 48 significant bits, against 53 in FP64.  The solve watches for the
// consequence (see k_scal_true) and finishes with the FP64 apply if it stalls.
// per-solve coefficients of the local part: d = r - 1 + 2|psi|^2 and psi^2
__global__ void k_jz_coef(int64_t n, const double *__restrict__ rem, const double2 *__restrict__ psi,
                          float2 *__restrict__ d, float4 *__restrict__ p2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 ps = psi[i];
    d[i] = split_df(rem[i] - 1.0 + 2.0 * (ps.x * ps.x + ps.y * ps.y));
    float2 re = split_df(ps.x * ps.x - ps.y * ps.y), im = split_df(2.0 * ps.x * ps.y);
    p2[i] = make_float4(re.x, re.y, im.x, im.y);
}

// q = J z from the exact FP32 copy z of the V-cycle output; partials of <J z, z>_R
__global__ void __launch_bounds__(RED_THREADS) k_jz_latdf(int64_t n, LatticeDfView L, double hd,
                                                          const float2 *__restrict__ d, const float4 *__restrict__ p2,
                                                          const float2 *__restrict__ z, double2 *__restrict__ q,
                                                          double *part, const int *stop) {
    __shared__ double sh[32];
    if (*stop) return;
    float as = 0.f, ac = 0.f;
    const uint32_t N = (uint32_t)L.N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = p >= L.nred ? 1u : 0u;
        uint32_t v = 2u * (uint32_t)(p - (c ? L.nred : 0));
        const uint32_t r = L.dN.div(v), k = L.dN.div(r);
        uint32_t i = v - r * N;
        const uint32_t j = r - k * N;
        if (((i + j + k) & 1u) != c) {
            ++v;
            ++i;
        }
        const int64_t other = c ? 0 : L.nred;
        const int b = (i == 0 || i == N - 1) + (j == 0 || j == N - 1) + (L.dim == 3 && (k == 0 || k == N - 1));
        const float2 zp = z[p];
        float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
        // + a (z_p - u z_u) for the edge to node u; conj: the -e edge
        auto edge = [&](int64_t idx, uint32_t u, bool conj) {
            const float2 a = L.a[idx];
            const float4 t = L.u[idx];
            const float2 ur = make_float2(t.x, t.y);
            const float2 ui = conj ? make_float2(-t.z, -t.w) : make_float2(t.z, t.w);
            const float2 zu = z[(int64_t)(u >> 1) + other];
            float ws = 0.f, wc = 0.f, vs = 0.f, vc = 0.f;
            dot2_df(ws, wc, ur, zu.x);
            dot2_df(ws, wc, ui, -zu.y);
            dot2_df(vs, vc, ur, zu.y);
            dot2_df(vs, vc, ui, zu.x);
            float tr = zp.x, er = 0.f, ti = zp.y, ei = 0.f;
            dot2_add(tr, er, -ws);
            er = __fadd_rn(er, -wc);
            dot2_add(ti, ei, -vs);
            ei = __fadd_rn(ei, -vc);
            dot2_df(rs, rc, a, tr);
            rc = __fmaf_rn(a.x, er, rc);
            dot2_df(is, ic, a, ti);
            ic = __fmaf_rn(a.x, ei, ic);
        };
        {
            const int64_t idx = j + (int64_t)N * k;
            if (i + 1 < N) edge(idx, v + 1, false);
            if (i > 0) edge(idx, v - 1, true);
        }
        {
            const int64_t idx = L.per_axis + i + (int64_t)N * k;
            if (j + 1 < N) edge(idx, v + N, false);
            if (j > 0) edge(idx, v - N, true);
        }
        if (L.dim == 3) {
            const int64_t idx = 2 * L.per_axis + i + (int64_t)N * j;
            if (k + 1 < N) edge(idx, v + N * N, false);
            if (k > 0) edge(idx, v - N * N, true);
        }
        // row scale 2^b (exact), then + d z + psi^2 conj(z)
        const float sb = (float)(1 << b);
        rs *= sb;
        rc *= sb;
        is *= sb;
        ic *= sb;
        const float2 dd = d[p];
        const float4 pp = p2[p];
        const float2 pr = make_float2(pp.x, pp.y), pi = make_float2(pp.z, pp.w);
        dot2_df(rs, rc, dd, zp.x);
        dot2_df(rs, rc, pr, zp.x);
        dot2_df(rs, rc, pi, zp.y);
        dot2_df(is, ic, dd, zp.y);
        dot2_df(is, ic, pi, zp.x);
        dot2_df(is, ic, pr, -zp.y);
        q[p] = make_double2((double)rs + (double)rc, (double)is + (double)ic);
        // |V_p| Re(conj(q_p) z_p) / h^d = 2^-b Re(conj(q_p) z_p)
        float ts = 0.f, tc = 0.f;
        dot2_df(ts, tc, make_float2(rs, rc), zp.x);
        dot2_df(ts, tc, make_float2(is, ic), zp.y);
        const float isb = 1.f / sb;
        dot2_add(as, ac, ts * isb);
        ac = __fadd_rn(ac, tc * isb);
    }
    double t = block_sum(((double)as + (double)ac) * hd, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_round32(int64_t n, const double2 *a, float2 *b) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) b[p] = to32(a[p]);
}

// y = J(psi) phi by the double-float lattice kernel the GL_MIXED_PRECOND solve
// runs, for phi rounded to FP32 (in the solve that rounding is exact); solve
// ordering, synchronises s
void jacobian_apply_pdf(gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s) {
    mesh_ensure_fp32(m, s);
    GL_REQUIRE(m->lat_ok, GL_ERR_ARG,
               "the double-FP32 Jacobian needs a mesh with an even number of nodes per side (checked lattice stencil)");
    const int64_t n = m->n;
    DBuf<float2> d(n), z(n);
    DBuf<float4> p2(n);
    DBuf<double> part(RED_BLOCKS);
    DBuf<int> stop(1);
    GL_CUDA(cudaMemsetAsync(stop.get(), 0, sizeof(int), s));
    const int G = grid_for(n, 256);
    note_launch(3);
    k_jz_coef<<<G, 256, 0, s>>>(n, m->lat_krem.get(), psi, d.get(), p2.get());
    k_round32<<<G, 256, 0, s>>>(n, phi, z.get());
    k_jz_latdf<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, lattice_df_view(m), m->lat_hd, d.get(), p2.get(), z.get(), y,
                                                  part.get(), stop.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
}

// v_new = q / gamma - (delta / gamma) v - (gamma / gamma_old) v_old
template <typename C, typename R>
__global__ void k_vnew(int64_t n, const MinresDev *S, const C *q, const C *v, const C *v_old, C *v_new) {
    if (S->status) return;
    // the scalars once per thread (a fixed grid: FP64 divisions are costly here),
    // four rows per step with every load issued first
    R ig = (R)(1.0 / S->gamma), dg = (R)(S->delta / S->gamma), go = (R)(S->gamma / S->gamma_old);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; p + 3 * stride < n; p += 4 * stride) {
        C a[4], b[4], c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = q[p + u * stride];
            b[u] = v[p + u * stride];
            c[u] = v_old[p + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v_new[p + u * stride] =
                mk(a[u].x * ig - dg * b[u].x - go * c[u].x, a[u].y * ig - dg * b[u].y - go * c[u].y);
    }
    for (; p < n; p += stride) {
        C a = q[p], b = v[p], c = v_old[p];
        v_new[p] = mk(a.x * ig - dg * b.x - go * c.x, a.y * ig - dg * b.y - go * c.y);
    }
}

// the mixed-precision form's two passes around the FP32 V-cycle, each fused
// with its neighbour: v_new of k_vnew also written as the V-cycle's FP32 input,
// and the V-cycle's FP32 output widened to z_new inside the <v_new, z_new>_R dot
__global__ void k_vnew_mp(int64_t n, const MinresDev *S, const double2 *q, const double2 *v, const double2 *v_old,
                          double2 *v_new, float2 *v32) {
    if (S->status) return;
    double ig = 1.0 / S->gamma, dg = S->delta / S->gamma, go = S->gamma / S->gamma_old;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; p + 3 * stride < n; p += 4 * stride) {
        double2 a[4], b[4], c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = q[p + u * stride];
            b[u] = v[p + u * stride];
            c[u] = v_old[p + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 r =
                make_double2(a[u].x * ig - dg * b[u].x - go * c[u].x, a[u].y * ig - dg * b[u].y - go * c[u].y);
            v_new[p + u * stride] = r;
            v32[p + u * stride] = to32(r);
        }
    }
    for (; p < n; p += stride) {
        double2 a = q[p], b = v[p], c = v_old[p];
        double2 r = make_double2(a.x * ig - dg * b.x - go * c.x, a.y * ig - dg * b.y - go * c.y);
        v_new[p] = r;
        v32[p] = to32(r);
    }
}
__global__ void __launch_bounds__(RED_THREADS) k_widen_dot(int64_t n, const double *vol, const double2 *v,
                                                           const float2 *z32, double2 *z, double *part,
                                                           const int *stop) {
    __shared__ double sh[32];
    if (*stop) return;
    double a = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // four rows per step, every load issued before the first use
    for (; p + 3 * stride < n; p += 4 * stride) {
        float2 zr[4];
        double2 vv[4];
        double vo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            zr[u] = z32[p + u * stride];
            vv[u] = v[p + u * stride];
            vo[u] = vol[p + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 zz = to64(zr[u]);
            z[p + u * stride] = zz;
            a += vo[u] * redot(vv[u], zz);
        }
    }
    for (; p < n; p += stride) {
        double2 zz = to64(z32[p]);
        z[p] = zz;
        a += vol[p] * redot(v[p], zz);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// w_new = (z / gamma - a3 w_old - a2 w) / a1 ; x += c_new eta w_new.  The
// scalars are folded once per thread (z (1 / (gamma a1)) - (a3 / a1) w_old -
// (a2 / a1) w): three FP64 operations per component instead of four, which
// matters because this stream is bound by GB300's FP64 pipe, not by HBM.
template <typename C, typename R>
__global__ void k_update(int64_t n, const MinresDev *S, const C *z, const C *w_old, const C *w, C *w_new, C *x) {
    if (S->status) return;
    const double ia1 = 1.0 / S->a1;
    const R sz = (R)(ia1 / S->gamma_cur), s3 = (R)(S->a3 * ia1), s2 = (R)(S->a2 * ia1);
    const R ce = (R)(S->c_new * S->eta_prev);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    auto upd = [&](C zz, C wo, C ww, C xx, int64_t q) {
        const C wn = mk(zz.x * sz - s3 * wo.x - s2 * ww.x, zz.y * sz - s3 * wo.y - s2 * ww.y);
        w_new[q] = wn;
        x[q] = mk(xx.x + ce * wn.x, xx.y + ce * wn.y);
    };
    for (; p + 3 * stride < n; p += 4 * stride) {
        C zz[4], wo[4], ww[4], xx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            zz[u] = z[p + u * stride];
            wo[u] = w_old[p + u * stride];
            ww[u] = w[p + u * stride];
            xx[u] = x[p + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) upd(zz[u], wo[u], ww[u], xx[u], p + u * stride);
    }
    for (; p < n; p += stride) upd(z[p], w_old[p], w[p], x[p], p);
}

// partials of ||b - J x||_D^2, only when the scalar kernel asked for a check
template <typename C, typename R>
__global__ void __launch_bounds__(RED_THREADS) k_true_resid(int64_t n, SellView<C> K, const R *kd, const R *vol,
                                                            const C *psi, const C *b, const C *x, double *part,
                                                            const MinresDev *S, int force) {
    __shared__ double sh[32];
    if (!force && (S->status || !S->check_true)) return;
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        C acc = sell_row<C, C>(K, p, x);
        C jx = jacobian_epilogue(acc, kd[p], psi[p], x[p]);
        C r = csub(b[p], jx);
        a += (double)vol[p] * redot(r, r);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ------------------------------------------------------------------ scalar kernels (one block)
__device__ double sum_parts(const double *part, double *sh) {
    double a = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) a += part[i];
    return block_sum(a, sh);
}

__global__ void k_scal_init(MinresDev *S, const double *part) {
    __shared__ double sh[32];
    double bb = sum_parts(part, sh);
    double vv = sum_parts(part + RED_BLOCKS, sh);
    if (threadIdx.x) return;
    double tol = S->tol;
    int use_true = S->use_true;
    S->it = 0;
    S->replays = 0;
    S->status = ST_RUN;
    S->check_true = 0;
    S->lucky = 0;
    S->bnorm = sqrt(bb);
    S->true_rel = (S->bnorm > 0) ? sqrt(vv) / S->bnorm : 0.0;
    // the tolerance is relative to b, the recurrence's estimate to r0 = b - J x0:
    // scaled by ||r0||_D / ||b||_D (exactly 1 from x0 = 0)
    S->rho0 = S->true_rel;
    S->est = 1.0;
    if (!(S->bnorm > 0)) {
        S->status = ST_CONV;
        S->est = 0;
    } else if (use_true && S->true_rel <= tol) {
        S->status = ST_CONV;
    } else if (!isfinite(S->true_rel)) {
        S->status = ST_NAN;
    } else if (S->maxit <= 0) {
        S->status = ST_MAXIT;
    }
}

// solve parameters, written before the captured init phase reads them
__global__ void k_set_params(MinresDev *S, double tol, int maxit, int use_true, double stall) {
    S->tol = tol;
    S->maxit = maxit;
    S->use_true = use_true;
    S->stall = stall;
}

__global__ void k_scal_gamma0(MinresDev *S, const double *part) {
    __shared__ double sh[32];
    double g2 = sum_parts(part, sh);
    if (threadIdx.x || S->status) return;
    if (!isfinite(g2)) {
        S->status = ST_NAN;
        return;
    }
    if (g2 < 0) {
        S->status = ST_BREAK;
        return;
    }
    double g = sqrt(g2);
    S->gamma = g;
    S->gamma_old = 1.0;
    S->eta = S->eta0 = g;
    S->c = S->c_old = 1.0;
    S->s = S->s_old = 0.0;
    if (g == 0) S->status = ST_CONV;
}

__global__ void k_scal_delta(MinresDev *S, const double *part) {
    __shared__ double sh[32];
    double d = sum_parts(part, sh);
    if (threadIdx.x || S->status) return;
    S->delta = d / (S->gamma * S->gamma);
}

__global__ void k_scal_givens(MinresDev *S, const double *part) {
    __shared__ double sh[32];
    double g2 = sum_parts(part, sh);
    if (threadIdx.x || S->status) return;
    if (!isfinite(g2) || !isfinite(S->delta)) {
        S->status = ST_NAN;
        return;
    }
    if (g2 < 0) {
        S->status = ST_BREAK;
        return;
    }
    double gn = sqrt(g2);
    double g = S->gamma, d = S->delta;
    double a0 = S->c * d - S->c_old * S->s * g;
    double a1 = sqrt(a0 * a0 + gn * gn);
    double a2 = S->s * d + S->c_old * S->c * g;
    double a3 = S->s_old * g;
    double cn = a0 / a1, sn = gn / a1;
    S->a1 = a1;
    S->a2 = a2;
    S->a3 = a3;
    S->c_new = cn;
    S->eta_prev = S->eta;
    S->gamma_cur = g;
    S->eta = -sn * S->eta;
    S->gamma_old = g;
    S->gamma = gn;
    S->c_old = S->c;
    S->c = cn;
    S->s_old = S->s;
    S->s = sn;
    S->it += 1;
    S->est = S->rho0 * fabs(S->eta) / S->eta0;
    S->lucky = (gn == 0);
    S->check_true = (S->est <= S->tol) || S->lucky;
}

// Conditional-node handles of the device-side MINRES loop (all unused when n = 0):
// h[0] the WHILE node around a body of ITER_UNROLL iterations, h[k] (k >= 1) the
// IF node around iteration k of the body.
struct Gates {
    cudaGraphConditionalHandle h[6];
    int n;
};

// after iteration k of a loop body: the IF nodes of the body's later iterations
// open only while the solve runs; every gate this iteration can reach is
// written, so no value is left from an earlier body
__device__ void set_gates(MinresDev *S, const Gates &g, int k) {
    const unsigned run = S->status == ST_RUN ? 1u : 0u;
    for (int j = k + 1; j < g.n; ++j) cudaGraphSetConditional(g.h[j], run);
}

__global__ void k_loop_begin(cudaGraphConditionalHandle h, const MinresDev *S) {
    cudaGraphSetConditional(h, S->status == ST_RUN ? 1u : 0u);
}

// end of a loop body: another body while the solve runs, at most maxit / 6 + 2
// bodies (then ST_MAXIT), so the loop ends whatever the state
__global__ void k_loop_next(cudaGraphConditionalHandle h, MinresDev *S) {
    S->replays += 1;
    bool run = S->status == ST_RUN;
    if (run && S->replays >= S->maxit / 6 + 2) {
        S->status = ST_MAXIT;
        run = false;
    }
    cudaGraphSetConditional(h, run ? 1u : 0u);
}

__global__ void k_scal_true(MinresDev *S, const double *part, Gates g, int k) {
    __shared__ double sh[32];
    double r2 = sum_parts(part, sh);
    if (threadIdx.x) return;
    if (S->status) {
        set_gates(S, g, k);
        return;
    }
    if (S->check_true) {
        if (S->use_true) {
            S->true_rel = sqrt(r2) / S->bnorm;
            if (!isfinite(S->true_rel))
                S->status = ST_NAN;
            else if (S->true_rel <= S->tol)
                S->status = ST_CONV;
            else if (S->stall > 0 && S->est <= S->stall * S->tol)
                S->status = ST_STALL;  // the recurrence has run far past what the true residual shows
        } else {
            S->status = ST_CONV;  // inner solves stop on the estimate alone
        }
        if (!S->status && S->lucky) S->status = ST_MAXIT;  // Krylov space exhausted above tol
    }
    if (!S->status && S->it >= S->maxit) S->status = ST_MAXIT;
    set_gates(S, g, k);
}

__global__ void k_scal_final(MinresDev *S, const double *part) {
    __shared__ double sh[32];
    double r2 = sum_parts(part, sh);
    if (threadIdx.x) return;
    if (S->bnorm > 0) S->true_rel = sqrt(r2) / S->bnorm;
}

// ------------------------------------------------------------------ MINRES driver
// The initial phase and a body of ITER_UNROLL iterations are captured once as
// CUDA graphs and replayed; every kernel turns into a no-op once the status word
// is set, so a replay past convergence costs only launch latency.  The three v,
// two z and three w buffers rotate, so the body holds a multiple of 6 iterations
// and starts every replay with the same buffer roles.
constexpr int ITER_UNROLL = 6;
static_assert(ITER_UNROLL == 6, "k_loop_next bounds the device loop by maxit / 6 + 2 bodies");

struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> slots;  // profiler event slots recorded inside the graph
    int64_t launches = 0;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        slots.clear();
        launches = 0;
    }
};

struct GraphKey {
    const void *m = nullptr, *psi = nullptr, *b = nullptr, *x = nullptr;
    int64_t prec_uid = -1, generation = -1, mesh_version = -1;
    int vc32 = 0, df = 0, loop = 0;
    bool operator==(const GraphKey &o) const {
        return m == o.m && psi == o.psi && b == o.b && x == o.x && prec_uid == o.prec_uid &&
               generation == o.generation && mesh_version == o.mesh_version && vc32 == o.vc32 && df == o.df &&
               loop == o.loop;
    }
};

template <typename T>
struct MinresWork {
    using C = cplx_t<T>;
    DBuf<C> v[3], z[2], w[3], q;
    DBuf<float2> jd;      // double-float Jacobian coefficients (mixed-precision solve)
    DBuf<float4> jp2;
    DBuf<double> part;
    DBuf<MinresDev> S;
    int64_t n = 0;
    cudaStream_t cap = nullptr, cap_body = nullptr, cap_if = nullptr;
    GraphKey key;
    Graph init, body;
    // the device-side loop: the whole solve in one graph; launches of its initial
    // phase and of one iteration (counted at capture)
    Graph loop;
    int64_t loop_init_launches = 0, loop_iter_launches = 0;
    void ensure(int64_t nn) {
        if (!cap) GL_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        if (!cap_body) GL_CUDA(cudaStreamCreateWithFlags(&cap_body, cudaStreamNonBlocking));
        if (!cap_if) GL_CUDA(cudaStreamCreateWithFlags(&cap_if, cudaStreamNonBlocking));
        if (n == nn) return;
        init.reset();
        body.reset();
        loop.reset();
        key = GraphKey{};
        for (auto &b : v) b.alloc(nn);
        for (auto &b : z) b.alloc(nn);
        for (auto &b : w) b.alloc(nn);
        q.alloc(nn);
        part.alloc(2 * RED_BLOCKS);
        S.alloc(1);
        jd.release();
        jp2.release();
        n = nn;
    }
    void ensure_df() {
        if (jd.n != (size_t)n) {
            jd.alloc(n);
            jp2.alloc(n);
        }
    }
};

struct MinresResult {
    int status, iters;
    double est, true_rel;
};

// vc32: run the V-cycle in FP32 even when the Krylov vectors are FP64
template <typename T>
static void precond_apply_any(gl_prec_s *p, const cplx_t<T> *v, cplx_t<T> *z, const int *stop, bool vc32,
                              cudaStream_t s);
template <>
void precond_apply_any<double>(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, bool vc32,
                               cudaStream_t s) {
    if (vc32)
        precond_apply_p64_via32(p, v, z, stop, s);
    else
        precond_apply_p(p, v, z, stop, s);
}
template <>
void precond_apply_any<float>(gl_prec_s *p, const float2 *v, float2 *z, const int *stop, bool, cudaStream_t s) {
    precond_apply_p32(p, v, z, stop, s);
}

// b = 0 has the solution x = 0 whatever the initial guess
template <typename C>
__global__ void k_zero_if_bzero(int64_t n, const MinresDev *S, C *x) {
    if (S->bnorm > 0) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = mk(decltype(x[0].x)(0), decltype(x[0].x)(0));
}

template <typename C>
__global__ void k_copy_if(int64_t n, const C *a, C *b, const int *stop) {
    if (*stop) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// captures whatever `enqueue` launches on a private stream into g
template <typename F>
static void capture(Graph &g, cudaStream_t cs, F &&enqueue) {
    g.reset();
    Profiler &pr = profiler();
    int64_t l0 = pr.launches.load();
    pr.capture = &g.slots;
    cudaGraph_t graph = nullptr;
    GL_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue(cs);
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        pr.capture = nullptr;
        throw;
    }
    GL_CUDA(cudaStreamEndCapture(cs, &graph));
    pr.capture = nullptr;
    g.launches = pr.launches.load() - l0;
    pr.launches.fetch_sub(g.launches);
    GL_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
    GL_CUDA(cudaGraphDestroy(graph));
}

static void replay(Graph &g, cudaStream_t s) {
    GL_CUDA(cudaGraphLaunch(g.exec, s));
    note_launch((int)g.launches);
}
static void harvest(Graph &g) {
    Profiler &pr = profiler();
    if (pr.active) pr.harvest(g.slots);
    pr.harvest_direct();
}

// Enqueues the initial phase of MINRES (v_1 = b - J x_0, z_1 = R v_1,
// gamma_1) on `cs`; the parameters tol/maxit/use_true are read from S.
template <typename T>
static void enqueue_init(gl_mesh_s *m, gl_prec_s *p, const cplx_t<T> *psi, const cplx_t<T> *b, cplx_t<T> *x,
                         bool vc32, bool df, MinresWork<T> &W, cudaStream_t cs) {
    using O = SolveOps<T>;
    using C = cplx_t<T>;
    int64_t n = m->n;
    MinresDev *S = W.S.get();
    const int *stop = &S->status;
    double *part = W.part.get();
    int G = grid_for(n, 256);
    C *v0 = W.v[0].get(), *v1 = W.v[1].get(), *z0 = W.z[0].get();
    C *w0 = W.w[0].get(), *w1 = W.w[1].get();
    GL_CUDA(cudaMemsetAsync(v0, 0, n * sizeof(C), cs));
    GL_CUDA(cudaMemsetAsync(w0, 0, n * sizeof(C), cs));
    GL_CUDA(cudaMemsetAsync(w1, 0, n * sizeof(C), cs));
    if constexpr (std::is_same<T, double>::value) {
        if (df) {
            note_launch();
            k_jz_coef<<<G, 256, 0, cs>>>(n, m->lat_krem.get(), psi, W.jd.get(), W.jp2.get());
        }
    }
    note_launch(3);
    k_init_resid<C, T><<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, O::K(m), O::kdiag(m), O::vol(m), psi, b, x, v1, part);
    k_scal_init<<<1, 1024, 0, cs>>>(S, part);
    k_zero_if_bzero<C><<<G, 256, 0, cs>>>(n, S, x);
    GL_LAUNCH_CHECK();
    if (p) {
        precond_apply_any<T>(p, v1, z0, stop, vc32, cs);
    } else {
        note_launch();
        k_copy_if<C><<<G, 256, 0, cs>>>(n, v1, z0, stop);
    }
    note_launch(2);
    k_dot<C, T><<<RED_BLOCKS, RED_THREADS, 0, cs>>>(n, O::vol(m), v1, z0, part, stop);
    k_scal_gamma0<<<1, 1024, 0, cs>>>(S, part);
    GL_LAUNCH_CHECK();
}

// Enqueues ITER_UNROLL MINRES iterations on `cs` (buffer roles rotate inside
// and return to the starting roles at the end).  With `gates` (the device-side
// loop; cs captures into the loop body) iterations 1.. each sit in an IF node,
// captured on cs_child, which the previous iteration opens only while the solve
// runs.
template <typename T>
static void enqueue_body(gl_mesh_s *m, gl_prec_s *p, const cplx_t<T> *psi, const cplx_t<T> *b, cplx_t<T> *x,
                         bool vc32, bool df, MinresWork<T> &W, cudaStream_t cs, const Gates *gates = nullptr,
                         cudaStream_t cs_child = nullptr) {
    using O = SolveOps<T>;
    using C = cplx_t<T>;
    int64_t n = m->n;
    MinresDev *S = W.S.get();
    const int *stop = &S->status;
    double *part = W.part.get();
    auto K = O::K(m);
    auto kd = O::kdiag(m);
    auto vol = O::vol(m);
    int G = grid_for(n, 256);
    C *v_old = W.v[0].get(), *v = W.v[1].get(), *v_new = W.v[2].get();
    C *z = W.z[0].get(), *z_new = W.z[1].get();
    C *w_old = W.w[0].get(), *w = W.w[1].get(), *w_new = W.w[2].get();
    const Gates nog{{}, 0};
    const Gates &g = gates ? *gates : nog;
    for (int k = 0; k < ITER_UNROLL; ++k) {
        cudaStream_t ks = cs;
        cudaGraph_t child = nullptr;
        if (gates && k > 0) {
            cudaStreamCaptureStatus cst;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            GL_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = g.h[k];
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            cudaGraphNode_t inode;
            GL_CUDA(cudaGraphAddNode(&inode, cg, deps, nullptr, ndeps, &cp));
            child = cp.conditional.phGraph_out[0];
            GL_CUDA(cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
            GL_CUDA(cudaStreamBeginCaptureToGraph(cs_child, child, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
            ks = cs_child;
        }
        try {
        {
            // algorithmic bytes of the fused Jacobian + dot: off-diagonals, K_ii,
            // |V|, psi, z (own row; neighbours cached) and the written q
            int64_t nnz = (sizeof(T) == 8) ? m->K.nnz_real : m->K32.nnz_real;
            bool use_df = false;
            if constexpr (std::is_same<T, double>::value) use_df = df;
            if (use_df) {
                // z32 (8 B), d and psi^2 (24 B) and the written q (16 B) per row; the
                // neighbours' z and the tables from cache
                // FP32 operations of the error-free transformations, counted from the
                // kernel: about 84 per stored neighbour and 100 per row, as flop
                // equivalents (2 per operation: each takes an FMA issue slot)
                ProfScope ps("jz", (double)n * (8 + 24 + 16), ks,
                             2.0 * (84.0 * (double)m->K.nnz_real + 100.0 * (double)n));
                k_jz_latdf<<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, lattice_df_view(m), m->lat_hd, W.jd.get(),
                                                               W.jp2.get(), p->mp_out.get(), (double2 *)W.q.get(),
                                                               part, stop);
            } else {
                bool lat64 = false;
                if constexpr (std::is_same<T, double>::value) lat64 = m->lat64_ok && p && p->lattice64;
                if (lat64) {
                    // own z, K_ii, |V|, psi and the written q per row (48 + 16 B); the
                    // neighbours' z and the tables from cache; per row the six
                    // complex FMAs, the 1 / |V| scaling, the local terms and the dot
                    if constexpr (std::is_same<T, double>::value) {
                        ProfScope ps("jz", (double)n * (3 * sizeof(C) + 2 * sizeof(T)), ks,
                                     8.0 * (double)nnz + 28.0 * (double)n);
                        k_jz_lat64<<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, lattice_view64(m), kd, psi, z, W.q.get(),
                                                                      part, stop);
                    }
                } else {
                    double jb = (double)nnz * (sizeof(C) + 4) + (double)n * (2 * sizeof(T) + 3 * sizeof(C));
                    // a complex FMA (8 flops) per stored entry; per row the local terms
                    // (K_ii - 1 + 2|psi|^2) z + psi^2 conj(z) (20) and the dot (5)
                    ProfScope ps("jz", jb, ks, 8.0 * (double)nnz + 25.0 * (double)n);
                    k_jz<C, T><<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, K, kd, vol, psi, z, W.q.get(), part, stop);
                }
            }
        }
        note_launch(2);
        k_scal_delta<<<1, 1024, 0, ks>>>(S, part);
        bool fused = false;
        if constexpr (std::is_same<T, double>::value) fused = vc32 && p;
        if (fused) {
            // FP32 V-cycle between the two fused passes
            k_vnew_mp<<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, S, (const double2 *)W.q.get(), (const double2 *)v,
                                                          (const double2 *)v_old, (double2 *)v_new,
                                                          p->mp_in.get());
            precond_apply_p32(p, p->mp_in.get(), p->mp_out.get(), stop, ks);
            note_launch(5);
            k_widen_dot<<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, m->volp.get(), (const double2 *)v_new,
                                                            p->mp_out.get(), (double2 *)z_new, part, stop);
        } else {
            k_vnew<C, T><<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, S, W.q.get(), v, v_old, v_new);
            if (p) {
                precond_apply_any<T>(p, v_new, z_new, stop, vc32, ks);
            } else {
                note_launch();
                k_copy_if<C><<<G, 256, 0, ks>>>(n, v_new, z_new, stop);
            }
            note_launch(5);
            k_dot<C, T><<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, vol, v_new, z_new, part, stop);
        }
        k_scal_givens<<<1, 1024, 0, ks>>>(S, part);
        k_update<C, T><<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, S, z, w_old, w, w_new, x);
        k_true_resid<C, T><<<RED_BLOCKS, RED_THREADS, 0, ks>>>(n, K, kd, vol, psi, b, x, part, S, 0);
        k_scal_true<<<1, 1024, 0, ks>>>(S, part, g, k);
        GL_LAUNCH_CHECK();
        } catch (...) {
            if (child) {
                cudaGraph_t dummy = nullptr;
                cudaStreamEndCapture(cs_child, &dummy);
            }
            throw;
        }
        if (child) GL_CUDA(cudaStreamEndCapture(cs_child, &child));
        C *t = v_old;
        v_old = v;
        v = v_new;
        v_new = t;
        t = z;
        z = z_new;
        z_new = t;
        t = w_old;
        w_old = w;
        w = w_new;
        w_new = t;
    }
}

// Runs MINRES on J x = b with x as the initial guess (overwritten).  use_true:
// stop on the FP64 true residual (FP64 path) or on the estimate alone (inner).
template <typename T>
static MinresResult minres(gl_mesh_s *m, gl_prec_s *p, const cplx_t<T> *psi, const cplx_t<T> *b, cplx_t<T> *x,
                           double tol, int maxit, bool use_true, bool vc32, MinresWork<T> &W, cudaStream_t s,
                           bool df = false, bool device_loop = true) {
    using O = SolveOps<T>;
    using C = cplx_t<T>;
    int64_t n = m->n;
    W.ensure(n);
    if (df) W.ensure_df();
    MinresDev *S = W.S.get();
    double *part = W.part.get();
    // The device-side loop (the whole solve in one graph: the initial phase, then a
    // WHILE node over bodies of ITER_UNROLL iterations whose later iterations sit in
    // IF nodes) whenever no kernel class is being timed (the profiler's event
    // nodes cannot sit in conditional bodies) and R_inf does not nest its own loop.
    const bool timing_class = profiler().active && !profiler().name.empty();
    const bool loop = device_loop && !timing_class && !(p && p->rinf);
    GraphKey key{m, psi, b, x, p ? p->uid : -1, profiler().generation, m->version, vc32 ? 1 : 0, df ? 1 : 0,
                 loop ? 1 : 0};
    if (!(key == W.key) || (loop ? !W.loop.exec : (!W.init.exec || !W.body.exec))) {
        W.key = key;
        if (loop) {
            capture(W.loop, W.cap, [&](cudaStream_t cs) {
                Profiler &pr = profiler();
                const int64_t l0 = pr.launches.load();
                enqueue_init<T>(m, p, psi, b, x, vc32, df, W, cs);
                const int64_t l1 = pr.launches.load();
                cudaStreamCaptureStatus cst;
                cudaGraph_t cg = nullptr;
                const cudaGraphNode_t *deps = nullptr;
                size_t ndeps = 0;
                GL_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
                Gates g{};
                g.n = ITER_UNROLL;
                GL_CUDA(cudaGraphConditionalHandleCreate(&g.h[0], cg, 0, cudaGraphCondAssignDefault));
                note_launch();
                k_loop_begin<<<1, 1, 0, cs>>>(g.h[0], S);
                GL_LAUNCH_CHECK();
                GL_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
                cudaGraphNodeParams cp = {};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = g.h[0];
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t wnode;
                GL_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                GL_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
                for (int k = 1; k < ITER_UNROLL; ++k)
                    GL_CUDA(cudaGraphConditionalHandleCreate(&g.h[k], body, 0, cudaGraphCondAssignDefault));
                GL_CUDA(cudaStreamBeginCaptureToGraph(W.cap_body, body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal));
                const int64_t l2 = pr.launches.load();
                try {
                    enqueue_body<T>(m, p, psi, b, x, vc32, df, W, W.cap_body, &g, W.cap_if);
                    k_loop_next<<<1, 1, 0, W.cap_body>>>(g.h[0], S);
                    GL_LAUNCH_CHECK();
                } catch (...) {
                    cudaStreamEndCapture(W.cap_body, &body);
                    throw;
                }
                GL_CUDA(cudaStreamEndCapture(W.cap_body, &body));
                W.loop_init_launches = l1 - l0 + 1;  // + k_loop_begin
                W.loop_iter_launches = (pr.launches.load() - l2) / ITER_UNROLL;
            });
        } else {
            capture(W.init, W.cap, [&](cudaStream_t cs) { enqueue_init<T>(m, p, psi, b, x, vc32, df, W, cs); });
            capture(W.body, W.cap, [&](cudaStream_t cs) { enqueue_body<T>(m, p, psi, b, x, vc32, df, W, cs); });
        }
    }
    // Stall test: with the double-FP32 Jacobian the ~48-bit apply limits the true
    // residual, so a recurrence three decades past tol hands over to FP64; in
    // FP64 a true residual that stays above tol while the recurrence runs nine
    // decades past it has reached the attainable accuracy (the rounding floor of
    // J applied to the iterate), and further iterations only repeat the test.
    k_set_params<<<1, 1, 0, s>>>(S, tol, maxit, use_true ? 1 : 0, !use_true ? 0.0 : (df ? 1e-3 : 1e-9));
    GL_LAUNCH_CHECK();
    MinresDev h;
    if (loop) {
        GL_CUDA(cudaGraphLaunch(W.loop.exec, s));
        GL_CUDA(cudaMemcpyAsync(&h, S, sizeof(MinresDev), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        // the kernels that ran: the initial phase and one iteration's launches per iteration
        note_launch((int)(W.loop_init_launches + (int64_t)h.it * W.loop_iter_launches + h.replays));
        GL_REQUIRE(h.status != ST_RUN, GL_ERR_TIMEOUT, "MINRES status word was not updated");
    } else {
    replay(W.init, s);
    int64_t polls = 0, max_polls = (int64_t)maxit / ITER_UNROLL + 3;
    bool init_timed = false;  // the initial phase's profiler events are summed once per solve
    for (;;) {
        GL_CUDA(cudaMemcpyAsync(&h, S, sizeof(MinresDev), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        if (!init_timed) {
            harvest(W.init);
            init_timed = true;
        }
        if (h.status != ST_RUN) break;
        GL_REQUIRE(polls++ <= max_polls, GL_ERR_TIMEOUT, "MINRES status word was not updated");
        replay(W.body, s);
        GL_CUDA(cudaMemcpyAsync(&h, S, sizeof(MinresDev), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        harvest(W.body);
        if (h.status != ST_RUN) break;
    }
    }
    if (use_true) {
        note_launch(2);
        k_true_resid<C, T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, O::K(m), O::kdiag(m), O::vol(m), psi, b, x, part, S,
                                                              1);
        k_scal_final<<<1, 1024, 0, s>>>(S, part);
        GL_LAUNCH_CHECK();
        GL_CUDA(cudaMemcpyAsync(&h, S, sizeof(MinresDev), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
    }
    return MinresResult{h.status, h.it, h.est, h.true_rel};
}

static gl_status status_of(int st) {
    switch (st) {
        case ST_CONV: return GL_OK;
        case ST_BREAK: return GL_ERR_BREAKDOWN;
        case ST_NAN: return GL_ERR_NAN;
        case ST_TIMEOUT: return GL_ERR_TIMEOUT;
        default: return GL_ERR_NOT_CONVERGED;
    }
}

// ------------------------------------------------------------------ mixed precision
__global__ void k_resid64_scaled(int64_t n, SellView<double2> K, const double *kd, const double *vol,
                                 const double2 *psi, const double2 *b, const double2 *x, double2 *r, double *part) {
    __shared__ double sh[32];
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = sell_row<double2, double2>(K, p, x);
        double2 jx = jacobian_epilogue(acc, kd[p], psi[p], x[p]);
        double2 rr = csub(b[p], jx);
        r[p] = rr;
        a += vol[p] * (rr.x * rr.x + rr.y * rr.y);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_sumsq_vol(int64_t n, const double *vol, const double2 *b, double *part) {
    __shared__ double sh[32];
    double a = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        a += vol[p] * (b[p].x * b[p].x + b[p].y * b[p].y);
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_sum_to(const double *part, double *out) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) a += part[i];
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) *out = t;
}
// r32 = r / scale
__global__ void k_down(int64_t n, const double2 *r, double scale, float2 *r32, float2 *e32) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) {
        r32[p] = make_float2((float)(r[p].x / scale), (float)(r[p].y / scale));
        e32[p] = make_float2(0.f, 0.f);
    }
}
// x += scale * e32
__global__ void k_up(int64_t n, const float2 *e32, double scale, double2 *x) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) {
        x[p].x += scale * (double)e32[p].x;
        x[p].y += scale * (double)e32[p].y;
    }
}
__global__ void k_psi32(int64_t n, const double2 *a, float2 *b) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) b[p] = to32(a[p]);
}

struct SolveWork {
    MinresWork<double> w64;
    MinresWork<float> w32;
    DBuf<double2> r;
    DBuf<float2> r32, e32, psi32;
    DBuf<double> part, sc;
};
static SolveWork &solve_work() {
    static thread_local SolveWork w;
    return w;
}

// ------------------------------------------------------------------ batched solves
// Many independent systems J(psi_s) x_s = b_s in ONE CUDA-graph launch: each
// instance is a branch of the graph (its own buffers and preconditioner), and
// its MINRES iterations run inside a WHILE conditional node whose condition a
// kernel sets from the instance's status word, so the whole batch runs on the
// device without host round trips.  The loop is bounded by a replay count.
__global__ void k_set_cond(cudaGraphConditionalHandle h, MinresDev *S, int max_replays) {
    int go = (S->status == ST_RUN) && (S->replays < max_replays);
    S->replays += 1;
    if (!go && S->status == ST_RUN) S->status = ST_MAXIT;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

struct BatchInst {
    gl_mesh_s *m = nullptr;
    gl_prec_s *p = nullptr;
    MinresWork<double> W;
    DBuf<double2> b, x;  // solve ordering
    bool df = false;     // double-float Jacobian (FP32 V-cycle on a lattice mesh)
};

}  // namespace gl

struct gl_batch_s {
    std::vector<std::unique_ptr<gl::BatchInst>> inst;
    gl_options o{};
    bool vc32 = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> b_ptr, x_ptr;  // user pointers the graph was built for
    cudaStream_t s0 = nullptr, sb = nullptr;
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> ev;
    int64_t launches = 0;
    ~gl_batch_s() {
        cudaDeviceSynchronize();
        if (exec) cudaGraphExecDestroy(exec);
        for (auto e : ev) cudaEventDestroy(e);
        for (auto t : br) cudaStreamDestroy(t);
        if (s0) cudaStreamDestroy(s0);
        if (sb) cudaStreamDestroy(sb);
        for (auto &i : inst) delete i->p;
    }
};

namespace gl {

gl_batch_s *batch_new() { return new gl_batch_s(); }
void batch_delete(gl_batch_s *B) { delete B; }
size_t batch_size(const gl_batch_s *B) { return B->inst.size(); }

void batch_create(gl_batch_s *B, int count, gl_mesh_s *const *meshes, const double2 *const *psi, const gl_options &o,
                  cudaStream_t s) {
    B->o = o;
    B->vc32 = (o.precision != GL_FP64);
    gl_options so = o;
    so.precision = B->vc32 ? GL_MIXED_PRECOND : GL_FP64;
    for (int i = 0; i < count; ++i) {
        auto I = std::make_unique<BatchInst>();
        I->m = meshes[i];
        I->p = new gl_prec_s();
        precond_setup(I->p, I->m, psi[i], so, s);
        I->W.ensure(I->m->n);
        // as in a single mixed solve: the double-float Jacobian wherever the mesh
        // has the checked lattice stencil
        I->df = B->vc32 && I->p->lattice && I->m->lat_ok;
        if (I->df) I->W.ensure_df();
        I->b.alloc(I->m->n);
        I->x.alloc(I->m->n);
        B->inst.push_back(std::move(I));
    }
    GL_CUDA(cudaStreamCreateWithFlags(&B->s0, cudaStreamNonBlocking));
    GL_CUDA(cudaStreamCreateWithFlags(&B->sb, cudaStreamNonBlocking));
    B->br.resize(count);
    for (auto &t : B->br) GL_CUDA(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
    B->ev.resize(count + 1);
    for (auto &e : B->ev) GL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

static void batch_build(gl_batch_s *B, const double2 *const *b, double2 *const *x) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    Profiler &pr = profiler();
    bool was_active = pr.active;
    pr.active = false;  // no event nodes inside conditional bodies
    int64_t l0 = pr.launches.load();
    cudaStream_t s0 = B->s0;
    cudaGraph_t graph = nullptr;
    GL_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    try {
        GL_CUDA(cudaEventRecord(B->ev[0], s0));
        for (size_t i = 0; i < B->inst.size(); ++i) {
            BatchInst &I = *B->inst[i];
            cudaStream_t si = B->br[i];
            int64_t n = I.m->n;
            MinresDev *S = I.W.S.get();
            GL_CUDA(cudaStreamWaitEvent(si, B->ev[0], 0));
            permute_in(n, I.m->perm.get(), b[i], I.b.get(), si);
            permute_in(n, I.m->perm.get(), x[i], I.x.get(), si);
            // the double-float Jacobian's stall test, as in a single solve
            k_set_params<<<1, 1, 0, si>>>(S, B->o.tol, B->o.maxit, 1, I.df ? 1e-3 : 0.0);
            enqueue_init<double>(I.m, I.p, I.p->psi_p.get(), I.b.get(), I.x.get(), B->vc32, I.df, I.W, si);
            // the WHILE node: its handle lives in the graph being captured
            cudaStreamCaptureStatus cst;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            GL_CUDA(cudaStreamGetCaptureInfo(si, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
            cudaGraphConditionalHandle h;
            GL_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault));
            int max_replays = B->o.maxit / ITER_UNROLL + 2;
            k_set_cond<<<1, 1, 0, si>>>(h, S, max_replays);
            GL_LAUNCH_CHECK();
            GL_CUDA(cudaStreamGetCaptureInfo(si, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t wnode;
            GL_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            GL_CUDA(cudaStreamUpdateCaptureDependencies(si, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
            GL_CUDA(cudaStreamBeginCaptureToGraph(B->sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            enqueue_body<double>(I.m, I.p, I.p->psi_p.get(), I.b.get(), I.x.get(), B->vc32, I.df, I.W, B->sb);
            k_set_cond<<<1, 1, 0, B->sb>>>(h, S, max_replays);
            GL_LAUNCH_CHECK();
            GL_CUDA(cudaStreamEndCapture(B->sb, &body));
            // final FP64 true residual, back to node order
            k_true_resid<double2, double><<<RED_BLOCKS, RED_THREADS, 0, si>>>(
                n, I.m->K.view(), I.m->kdiag.get(), I.m->volp.get(), I.p->psi_p.get(), I.b.get(), I.x.get(),
                I.W.part.get(), S, 1);
            k_scal_final<<<1, 1024, 0, si>>>(S, I.W.part.get());
            GL_LAUNCH_CHECK();
            permute_out(n, I.m->perm.get(), I.x.get(), x[i], si);
            GL_CUDA(cudaEventRecord(B->ev[i + 1], si));
            GL_CUDA(cudaStreamWaitEvent(s0, B->ev[i + 1], 0));
        }
    } catch (...) {
        cudaStreamEndCapture(s0, &graph);
        if (graph) cudaGraphDestroy(graph);
        pr.active = was_active;
        throw;
    }
    GL_CUDA(cudaStreamEndCapture(s0, &graph));
    pr.active = was_active;
    B->launches = pr.launches.load() - l0;
    pr.launches.fetch_sub(B->launches);
    GL_CUDA(cudaGraphInstantiate(&B->exec, graph, 0));
    GL_CUDA(cudaGraphDestroy(graph));
    B->b_ptr.assign(b, b + B->inst.size());
    B->x_ptr.assign(x, x + B->inst.size());
}

gl_status batch_run(gl_batch_s *B, const double2 *const *b, double2 *const *x, gl_solve_info *infos, cudaStream_t s) {
    size_t k = B->inst.size();
    for (auto &I : B->inst)
        GL_REQUIRE(I->p->mesh_version == I->m->version, GL_ERR_ARG, "a batch mesh's mu changed after gl_batch_create");
    bool same = B->exec && B->b_ptr.size() == k;
    for (size_t i = 0; same && i < k; ++i) same = (B->b_ptr[i] == b[i] && B->x_ptr[i] == x[i]);
    if (!same) batch_build(B, b, x);
    auto t0 = std::chrono::steady_clock::now();
    GL_CUDA(cudaGraphLaunch(B->exec, s));
    note_launch((int)B->launches);  // captured launches; loop bodies replay on the device
    GL_CUDA(cudaStreamSynchronize(s));
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    gl_status first = GL_OK;
    for (size_t i = 0; i < k; ++i) {
        BatchInst &I = *B->inst[i];
        MinresDev h;
        GL_CUDA(cudaMemcpy(&h, I.W.S.get(), sizeof(MinresDev), cudaMemcpyDeviceToHost));
        int restarts = 0, its = h.it;
        if (h.status == ST_STALL) {
            // the double-float Jacobian's ~48-bit apply held the true residual above
            // tol: this instance continues from its x with the FP64 Jacobian, as a
            // single solve does
            const auto t1 = std::chrono::steady_clock::now();
            MinresResult r = minres<double>(I.m, I.p, I.p->psi_p.get(), I.b.get(), I.x.get(), B->o.tol,
                                            std::max(B->o.maxit - its, 1), true, B->vc32, I.W, s, false, true);
            permute_out(I.m->n, I.m->perm.get(), I.x.get(), x[i], s);
            GL_CUDA(cudaStreamSynchronize(s));
            ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
            h.status = r.status;
            h.true_rel = r.true_rel;
            h.est = r.est;
            its += r.iters;
            restarts = 1;
        }
        if (infos) {
            gl_solve_info inf{};
            inf.iters = its;
            inf.outer_iters = 1;
            inf.converged = (h.status == ST_CONV && h.true_rel <= B->o.tol);
            inf.true_relres = h.true_rel;
            inf.est_relres = h.est;
            inf.solve_ms = ms;
            inf.df_jacobian = I.df ? 1 : 0;
            inf.stall_restarts = restarts;
            infos[i] = inf;
        }
        gl_status st = (h.status == ST_CONV) ? (h.true_rel <= B->o.tol ? GL_OK : GL_ERR_NOT_CONVERGED)
                                             : status_of(h.status);
        if (st == GL_ERR_TIMEOUT) {
            sweeps_reset(B->inst[i]->p, s);
            GL_CUDA(cudaStreamSynchronize(s));
            st = GL_ERR_TIMEOUT;
            if (infos) infos[i].converged = 0;
        }
        if (st != GL_OK && first == GL_OK) first = st;
    }
    return first;
}

gl_status jacobian_solve_p(gl_mesh_s *m, gl_prec_s *p, const double2 *psi_p, const double2 *b_p, double2 *x_p,
                           const gl_options &o, gl_solve_info *info, cudaStream_t s) {
    SolveWork &W = solve_work();
    auto t0 = std::chrono::steady_clock::now();
    gl_status st;
    gl_solve_info inf{};
    GL_REQUIRE(!(p && p->rinf) || o.precision == GL_FP64, GL_ERR_ARG, "R_inf needs precision GL_FP64");
    rinf_reset(p, s);
    if (o.warmstart)
        warmstart_apply_p(o.warmstart, m, psi_p, b_p, x_p, s, (const double2 *)o.warmstart_hint);
    else if (o.warmstart_hint)
        hint_guess_p(m, psi_p, b_p, (const double2 *)o.warmstart_hint, x_p, s);
    bool mixed = (o.precision == GL_MIXED) && p;
    if (!mixed) {
        bool vc32 = (o.precision == GL_MIXED_PRECOND) && p;
        if (vc32) precond_ensure_fp32(p, s);
        // the double-float Jacobian on lattices; if its ~48-bit arithmetic stalls
        // the FP64 true residual above tol, MINRES restarts from the current x
        // with the FP64 Jacobian
        const bool df = vc32 && p->lattice && m->lat_ok;
        const bool dl = o.device_loop != 0;
        MinresResult r = minres<double>(m, p, psi_p, b_p, x_p, o.tol, o.maxit, true, vc32, W.w64, s, df, dl);
        inf.df_jacobian = df ? 1 : 0;
        if (df && r.status == ST_STALL) {
            int used = r.iters;
            r = minres<double>(m, p, psi_p, b_p, x_p, o.tol, std::max(o.maxit - used, 1), true, vc32, W.w64, s, false,
                               dl);
            r.iters += used;
            inf.stall_restarts = 1;
        }
        inf.iters = r.iters;
        inf.outer_iters = 1;
        inf.true_relres = r.true_rel;
        inf.est_relres = r.est;
        inf.converged = (r.status == ST_CONV);
        st = status_of(r.status);
    } else {
        precond_ensure_fp32(p, s);
        int64_t n = m->n;
        if (W.r.n != (size_t)n) {
            W.r.alloc(n);
            W.r32.alloc(n);
            W.e32.alloc(n);
            W.psi32.alloc(n);
        }
        W.part.alloc(RED_BLOCKS);
        W.sc.alloc(2);
        int G = grid_for(n, 256);
        k_psi32<<<G, 256, 0, s>>>(n, psi_p, W.psi32.get());
        k_sumsq_vol<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->volp.get(), b_p, W.part.get());
        k_sum_to<<<1, 1024, 0, s>>>(W.part.get(), W.sc.get());
        double bb = 0;
        GL_CUDA(cudaMemcpyAsync(&bb, W.sc.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        double bnorm = std::sqrt(bb);
        st = GL_ERR_NOT_CONVERGED;
        int max_outer = o.max_outer > 0 ? o.max_outer : 20;
        double inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-5;
        double rel = 0;
        int total = 0, outer = 0;
        double est = 0;
        if (bnorm == 0) {
            GL_CUDA(cudaMemsetAsync(x_p, 0, n * sizeof(double2), s));
            st = GL_OK;
        }
        for (; st != GL_OK && outer <= max_outer; ++outer) {
            k_resid64_scaled<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->K.view(), m->kdiag.get(), m->volp.get(), psi_p,
                                                                b_p, x_p, W.r.get(), W.part.get());
            k_sum_to<<<1, 1024, 0, s>>>(W.part.get(), W.sc.get());
            double rr = 0;
            GL_CUDA(cudaMemcpyAsync(&rr, W.sc.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
            GL_CUDA(cudaStreamSynchronize(s));
            rel = std::sqrt(rr) / bnorm;
            if (!std::isfinite(rel)) {
                st = GL_ERR_NAN;
                break;
            }
            if (rel <= o.tol) {
                st = GL_OK;
                break;
            }
            if (outer == max_outer || total >= o.maxit) break;
            double scale = std::sqrt(rr);
            k_down<<<G, 256, 0, s>>>(n, W.r.get(), scale, W.r32.get(), W.e32.get());
            GL_LAUNCH_CHECK();
            MinresResult r = minres<float>(m, p, W.psi32.get(), W.r32.get(), W.e32.get(), inner_tol,
                                           o.maxit - total, false, false, W.w32, s, false, o.device_loop != 0);
            total += r.iters;
            est = r.est;
            if (r.status == ST_BREAK || r.status == ST_NAN || r.status == ST_TIMEOUT) {
                st = status_of(r.status);
                break;
            }
            k_up<<<G, 256, 0, s>>>(n, W.e32.get(), scale, x_p);
            GL_LAUNCH_CHECK();
        }
        inf.iters = total;
        inf.outer_iters = outer;
        inf.true_relres = rel;
        inf.est_relres = est;
        inf.converged = (st == GL_OK);
    }
    GL_CUDA(cudaStreamSynchronize(s));
    auto t1 = std::chrono::steady_clock::now();
    // a coarse-sweep wait that ran out (it wrote the status word) left the
    // sweeps' counters out of step
    if (p && st == GL_ERR_TIMEOUT) {
        sweeps_reset(p, s);
        GL_CUDA(cudaStreamSynchronize(s));
        st = GL_ERR_TIMEOUT;
        inf.converged = 0;
    }
    inf.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    inf.warmstart_used = o.warmstart ? warmstart_used(o.warmstart, s) : (o.warmstart_hint ? 1 : 0);
    inf.lattice_stencil = (p && p->has32 && o.precision != GL_FP64 && p->lattice && m->lat_ok) ? 1 : 0;
    // MINRES's FP64 Jacobian (FP64 solves; mixed-preconditioner solves without the
    // double-float apply or after its stall) read the FP64 tables
    const bool fp64_j = o.precision == GL_FP64 ||
                        (o.precision == GL_MIXED_PRECOND && (!inf.df_jacobian || inf.stall_restarts));
    inf.jacobian_tables = (fp64_j && m->lat64_ok && p && p->lattice64) ? 1 : 0;
    if (p && p->rinf) {
        // measured: every application ran its own number of cycles, each followed by a residual
        const RinfDev R = rinf_read(p, s);
        const double per = p->cost_fine > 0 ? (p->cost_vcycle + p->cost_fine) / p->cost_fine : 0.0;
        inf.matvec_equiv = (double)(inf.iters + inf.outer_iters) + (double)R.cycles * per;
        inf.cycles_per_apply = R.applies ? (double)R.cycles / (double)R.applies : 0.0;
    } else {
        inf.matvec_equiv = (double)(inf.iters + inf.outer_iters) * (1.0 + (p ? precond_cost(p, p->cycles) : 0.0));
        inf.cycles_per_apply = p ? (double)p->cycles : 0.0;
    }
    if (info) {
        double setup = info->setup_ms;
        *info = inf;
        info->setup_ms = setup;
    }
    return st;
}

}  // namespace gl
