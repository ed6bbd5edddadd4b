// gl_cont.cu -- what the parameter continuation of Sec. 4 needs besides the
// Jacobian solve: the energy (Eq. discr energy), d GL / d mu, and the
// pseudo-arclength predictor-corrector driver itself (host logic over the
// library's own solves; every vector operation runs in the kernels below).
#include <chrono>

#include "gl_internal.cuh"

using namespace gl;

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename F>
gl_status guard(F &&f) {
    try {
        set_error("");
        return f();
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return GL_ERR_OOM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return GL_ERR_CUDA;
    }
}

__device__ __forceinline__ void block_sum_to(double acc, double *out) {
    __shared__ double sh[RED_THREADS];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// per row j of K-hat (node order): Re conj(psi_j) (K-hat psi)_j + |V_j| (-|psi_j|^2 + |psi_j|^4 / 2);
// summed over the rows (Re psi^H K-hat psi = sum over edges of alpha |psi_j - exp(-i theta) psi_k|^2)
__global__ void __launch_bounds__(RED_THREADS) k_energy_part(int64_t n, const int64_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci,
                                                             const double2 *__restrict__ kv,
                                                             const double *__restrict__ vol,
                                                             const double2 *__restrict__ psi, double *part) {
    double acc = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double sr = 0, si = 0;
        for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
            const double2 a = kv[q], p = psi[ci[q]];
            sr += a.x * p.x - a.y * p.y;
            si += a.x * p.y + a.y * p.x;
        }
        const double2 p = psi[j];
        const double a2 = p.x * p.x + p.y * p.y;
        acc += (p.x * sr + p.y * si) + vol[j] * (-a2 + 0.5 * a2 * a2);
    }
    block_sum_to(acc, part + blockIdx.x);
}

// out_j = |V_j|^-1 sum_{k != j} (-i theta1_jk) K-hat_jk psi_k
__global__ void k_residual_dmu(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const double2 *__restrict__ kv, const double *__restrict__ th1,
                               const double *__restrict__ vol, const double2 *__restrict__ psi, double2 *out) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sr = 0, si = 0;
    for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
        if (ci[q] == j) continue;
        const double2 a = kv[q], p = psi[ci[q]];
        const double zr = a.x * p.x - a.y * p.y, zi = a.x * p.y + a.y * p.x;
        // (-i theta) (zr + i zi) = theta (zi - i zr)
        sr += th1[q] * zi;
        si -= th1[q] * zr;
    }
    const double iv = 1.0 / vol[j];
    out[j] = make_double2(sr * iv, si * iv);
}

// <x, y>_R partial sums: sum |V_i| Re conj(x_i) y_i
__global__ void __launch_bounds__(RED_THREADS) k_dot_r_part(int64_t n, const double *__restrict__ vol,
                                                            const double2 *__restrict__ x,
                                                            const double2 *__restrict__ y, double *part) {
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = x[i], b = y[i];
        acc += vol[i] * (a.x * b.x + a.y * b.y);
    }
    block_sum_to(acc, part + blockIdx.x);
}

__global__ void __launch_bounds__(RED_THREADS) k_sum_parts(const double *__restrict__ part, double *out) {
    double acc = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) acc += part[i];
    block_sum_to(acc, out);
}

// z = x + a y
__global__ void k_axpby(int64_t n, const double2 *__restrict__ x, double a, const double2 *__restrict__ y,
                        double2 *__restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = make_double2(x[i].x + a * y[i].x, x[i].y + a * y[i].y);
}
// psi += a + d c
__global__ void k_newton_border(int64_t n, const double2 *__restrict__ a, double d, const double2 *__restrict__ c,
                                double2 *__restrict__ psi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) psi[i] = make_double2(psi[i].x + a[i].x + d * c[i].x, psi[i].y + a[i].y + d * c[i].y);
}
// t = s (x - y)
__global__ void k_scaled_diff(int64_t n, const double2 *__restrict__ x, const double2 *__restrict__ y, double sc,
                              double2 *__restrict__ t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) t[i] = make_double2(sc * (x[i].x - y[i].x), sc * (x[i].y - y[i].y));
}
// y = sc x
__global__ void k_scale(int64_t n, const double2 *__restrict__ x, double sc, double2 *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_double2(sc * x[i].x, sc * x[i].y);
}

double energy_of(gl_mesh_s *m, const double2 *psi, double *part, double *scal, cudaStream_t s) {
    k_energy_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->n, m->khat.rp.get(), m->khat.ci.get(), m->khat.v.get(),
                                                     m->vol.get(), psi, part);
    k_sum_parts<<<1, RED_THREADS, 0, s>>>(part, scal);
    GL_LAUNCH_CHECK();
    double F = 0;
    GL_CUDA(cudaMemcpyAsync(&F, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return F;
}

void residual_dmu(gl_mesh_s *m, const double2 *psi, double2 *out, cudaStream_t s) {
    k_residual_dmu<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, m->khat.rp.get(), m->khat.ci.get(), m->khat.v.get(),
                                                       m->kth1.get(), m->vol.get(), psi, out);
    GL_LAUNCH_CHECK();
}

// device state of one continuation run (node order)
struct ContWork {
    int64_t n;
    DBuf<double2> psi_s, t, r, b, a, c;
    DBuf<double> part, scal;
    explicit ContWork(int64_t n_) : n(n_), psi_s(n_), t(n_), r(n_), b(n_), a(n_), c(n_), part(RED_BLOCKS), scal(1) {}
};

struct Cont {
    gl_mesh_s *m;
    const gl_cont_options &o;
    cudaStream_t s;
    ContWork W;
    double vol_tot;
    double setup_ms = 0, solve_ms = 0;
    int iters_total = 0;

    Cont(gl_mesh_s *m_, const gl_cont_options &o_, cudaStream_t s_)
        : m(m_), o(o_), s(s_), W(m_->n), vol_tot(std::pow(m_->edge, m_->dim)) {}

    int G() const { return grid_for(m->n, 256); }
    void *sv() const { return reinterpret_cast<void *>(s); }

    // <x, y>_R / |Omega|
    double ip(const double2 *x, const double2 *y) {
        k_dot_r_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->n, m->vol.get(), x, y, W.part.get());
        k_sum_parts<<<1, RED_THREADS, 0, s>>>(W.part.get(), W.scal.get());
        GL_LAUNCH_CHECK();
        double v = 0;
        GL_CUDA(cudaMemcpyAsync(&v, W.scal.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        return v / vol_tot;
    }
    // W.r = GL(psi); returns ||GL||_R / sqrt|Omega|
    double gl_norm(const double2 *psi) {
        residual_p_node(psi, W.r.get());
        return std::sqrt(ip(W.r.get(), W.r.get()));
    }
    void residual_p_node(const double2 *psi, double2 *r) {
        gl_status st = gl_residual(m, psi, r, sv());
        if (st != GL_OK) throw Error{st, last_error()};
    }
    void set_mu(double mu) { mesh_set_mu(m, mu, s); }

    // R(psi), taking over the aggregates, colours and kernel choices of `like`
    gl_prec setup(const double2 *psi, gl_prec like) {
        if (o.solver.cycles == 0) return nullptr;
        auto t0 = std::chrono::steady_clock::now();
        gl_prec p = nullptr;
        gl_status st = gl_precond_setup_like(m, psi, &o.solver, like, sv(), &p);
        if (st != GL_OK) throw Error{st, last_error()};
        setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return p;
    }
    // x = J(psi)^-1 b from x = 0; returns the MINRES iterations, or -1 if the solve failed
    int solve(const double2 *psi, gl_prec p, const double2 *b, double2 *x) {
        GL_CUDA(cudaMemsetAsync(x, 0, m->n * sizeof(double2), s));
        gl_solve_info info{};
        gl_status st = gl_jacobian_solve(m, psi, p, b, x, &o.solver, &info, sv());
        solve_ms += info.solve_ms;
        iters_total += info.iters;
        if (st == GL_OK) return info.iters;
        if (st == GL_ERR_NOT_CONVERGED || st == GL_ERR_BREAKDOWN || st == GL_ERR_NAN) return -1;
        throw Error{st, last_error()};
    }
    void record(gl_cont_point &pt, const double2 *psi, double gnorm, double ds, int steps, int last, int retries) {
        pt.mu = m->mu;
        pt.energy = energy_of(m, psi, W.part.get(), W.scal.get(), s) / vol_tot;
        pt.gl_norm = gnorm;
        pt.ds = ds;
        pt.newton_steps = steps;
        pt.iters_last = last;
        pt.iters_total = iters_total;
        pt.retries = retries;
        pt.setup_ms = setup_ms;
        pt.solve_ms = solve_ms;
        iters_total = 0;
        setup_ms = solve_ms = 0;
    }
};

struct PrecGuard {
    gl_prec p = nullptr;
    ~PrecGuard() {
        if (p) gl_precond_destroy(p);
    }
    void reset(gl_prec q) {
        if (p) gl_precond_destroy(p);
        p = q;
    }
};

}  // namespace

gl_status gl_energy(gl_mesh m, const void *psi, double *energy, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi && energy, GL_ERR_ARG, "NULL argument");
        DBuf<double> part(RED_BLOCKS), scal(1);
        *energy = energy_of(m, static_cast<const double2 *>(psi), part.get(), scal.get(), as_stream(stream));
        return GL_OK;
    });
}

gl_status gl_residual_dmu(gl_mesh m, const void *psi, void *out, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi && out, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(psi != out, GL_ERR_ARG, "psi and out must not alias");
        residual_dmu(m, static_cast<const double2 *>(psi), static_cast<double2 *>(out), as_stream(stream));
        GL_CUDA(cudaStreamSynchronize(as_stream(stream)));
        return GL_OK;
    });
}

gl_status gl_cont_options_default(gl_cont_options *o) {
    if (!o) return GL_ERR_ARG;
    *o = gl_cont_options{};
    o->ds = 0.05;
    o->ds_min = 1e-4;
    o->ds_max = 0.2;
    o->mu_max = 1.0;
    o->max_steps = 100;
    o->newton_tol = 1e-9;
    o->newton_maxit = 8;
    gl_options_default(&o->solver);
    o->solver.tol = 1e-8;
    return GL_OK;
}

gl_status gl_continuation(gl_mesh m, void *psi_v, const gl_cont_options *o, gl_cont_point *pts, int max_points,
                          int *npoints, void *const *states, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi_v && o && pts && npoints, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(max_points >= 1, GL_ERR_ARG, "max_points must be >= 1");
        GL_REQUIRE(o->ds > 0 && o->ds_min > 0 && o->ds_max >= o->ds_min, GL_ERR_ARG, "bad step sizes");
        GL_REQUIRE(o->newton_maxit >= 1 && o->newton_tol > 0, GL_ERR_ARG, "bad Newton settings");
        *npoints = 0;
        cudaStream_t s = as_stream(stream);
        const int64_t n = m->n;
        double2 *psi = static_cast<double2 *>(psi_v);
        Cont C(m, *o, s);
        ContWork &W = C.W;
        PrecGuard P;
        auto save_state = [&](int k) {
            if (states && states[k])
                GL_CUDA(cudaMemcpyAsync(states[k], psi, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        };

        // Newton at the start's mu
        int steps = 0, last = 0;
        double g = 0;
        bool ok = false;
        for (int it = 0; it <= o->newton_maxit; ++it) {
            g = C.gl_norm(psi);
            if (g <= o->newton_tol) {
                ok = true;
                break;
            }
            if (it == o->newton_maxit) break;
            P.reset(C.setup(psi, P.p));
            k_scale<<<C.G(), 256, 0, s>>>(n, W.r.get(), -1.0, W.b.get());
            GL_LAUNCH_CHECK();
            int k = C.solve(psi, P.p, W.b.get(), W.a.get());
            if (k < 0) break;
            k_axpby<<<C.G(), 256, 0, s>>>(n, psi, 1.0, W.a.get(), psi);
            GL_LAUNCH_CHECK();
            ++steps;
            last = k;
        }
        GL_REQUIRE(ok, GL_ERR_NOT_CONVERGED, "Newton did not converge at the start of the continuation");
        C.record(pts[0], psi, g, 0.0, steps, last, 0);
        save_state(0);
        int np = 1;

        // first tangent: J c = -dGL/dmu, t = (c, 1) / norm
        P.reset(C.setup(psi, P.p));
        residual_dmu(m, psi, W.r.get(), s);
        k_scale<<<C.G(), 256, 0, s>>>(n, W.r.get(), -1.0, W.b.get());
        GL_LAUNCH_CHECK();
        GL_REQUIRE(C.solve(psi, P.p, W.b.get(), W.c.get()) >= 0, GL_ERR_NOT_CONVERGED, "tangent solve failed");
        double nrm = std::sqrt(C.ip(W.c.get(), W.c.get()) + 1.0);
        k_scale<<<C.G(), 256, 0, s>>>(n, W.c.get(), 1.0 / nrm, W.t.get());
        GL_LAUNCH_CHECK();
        double t_mu = 1.0 / nrm;
        double ds = o->ds;
        C.iters_total = 0;  // the tangent solve belongs to no point
        C.setup_ms = C.solve_ms = 0;

        for (int step = 0; step < o->max_steps && np < max_points; ++step) {
            if (m->mu >= o->mu_max) break;
            const double mu_s = m->mu;
            GL_CUDA(cudaMemcpyAsync(W.psi_s.get(), psi, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
            const double t_psi_s = C.ip(W.t.get(), W.psi_s.get());
            int retries = 0;
            double mu_n = mu_s;
            for (;;) {
                k_axpby<<<C.G(), 256, 0, s>>>(n, W.psi_s.get(), ds, W.t.get(), psi);
                GL_LAUNCH_CHECK();
                mu_n = mu_s + ds * t_mu;
                C.set_mu(mu_n);
                steps = last = 0;
                ok = false;
                for (int it = 0; it <= o->newton_maxit; ++it) {
                    g = C.gl_norm(psi);  // W.r = GL(psi)
                    if (g <= o->newton_tol) {
                        ok = true;
                        break;
                    }
                    if (it == o->newton_maxit || !std::isfinite(g)) break;
                    const double ncond = C.ip(W.t.get(), psi) - t_psi_s + t_mu * (mu_n - mu_s) - ds;
                    P.reset(C.setup(psi, P.p));
                    k_scale<<<C.G(), 256, 0, s>>>(n, W.r.get(), -1.0, W.b.get());
                    GL_LAUNCH_CHECK();
                    const int ka = C.solve(psi, P.p, W.b.get(), W.a.get());
                    if (ka < 0) break;
                    residual_dmu(m, psi, W.r.get(), s);
                    k_scale<<<C.G(), 256, 0, s>>>(n, W.r.get(), -1.0, W.b.get());
                    GL_LAUNCH_CHECK();
                    if (C.solve(psi, P.p, W.b.get(), W.c.get()) < 0) break;
                    const double dmu = (-ncond - C.ip(W.t.get(), W.a.get())) / (t_mu + C.ip(W.t.get(), W.c.get()));
                    if (!std::isfinite(dmu)) break;
                    k_newton_border<<<C.G(), 256, 0, s>>>(n, W.a.get(), dmu, W.c.get(), psi);
                    GL_LAUNCH_CHECK();
                    mu_n += dmu;
                    C.set_mu(mu_n);
                    ++steps;
                    last = ka;
                }
                if (ok) break;
                ds *= 0.5;
                ++retries;
                if (ds < o->ds_min) {
                    // give back the last accepted point
                    GL_CUDA(cudaMemcpyAsync(psi, W.psi_s.get(), n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
                    C.set_mu(mu_s);
                    *npoints = np;
                    throw Error{GL_ERR_NOT_CONVERGED, "continuation step fell below ds_min"};
                }
            }
            // secant tangent
            k_scaled_diff<<<C.G(), 256, 0, s>>>(n, psi, W.psi_s.get(), 1.0, W.a.get());
            GL_LAUNCH_CHECK();
            const double dmu = mu_n - mu_s;
            nrm = std::sqrt(C.ip(W.a.get(), W.a.get()) + dmu * dmu);
            k_scale<<<C.G(), 256, 0, s>>>(n, W.a.get(), 1.0 / nrm, W.t.get());
            GL_LAUNCH_CHECK();
            t_mu = dmu / nrm;
            C.record(pts[np], psi, g, ds, steps, last, retries);
            save_state(np);
            ++np;
            *npoints = np;
            if (steps <= 2)
                ds = std::min(ds * 1.5, o->ds_max);
            else if (steps >= 5)
                ds = std::max(ds * 0.7, o->ds_min);
        }
        GL_CUDA(cudaStreamSynchronize(s));
        *npoints = np;
        return GL_OK;
    });
}
