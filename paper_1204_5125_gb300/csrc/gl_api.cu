// gl_api.cu -- the extern "C" boundary declared in include/gl.h.  Every entry
// point validates its arguments, runs the GPU work on the caller's stream, and
// turns exceptions into gl_status codes with a per-thread message.
#include <chrono>

#include "gl_internal.cuh"
#include "gl_profile.cuh"

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

void check_opts(const gl_options *o) {
    GL_REQUIRE(o, GL_ERR_ARG, "options must not be NULL");
    GL_REQUIRE(o->tol >= 0, GL_ERR_ARG, "tol must be >= 0");
    GL_REQUIRE(o->maxit >= 0, GL_ERR_ARG, "maxit must be >= 0");
    GL_REQUIRE((o->cycles >= 0 && o->cycles <= 64) || o->cycles == GL_CYCLES_INF, GL_ERR_ARG,
               "cycles must be in [0, 64] or GL_CYCLES_INF");
    GL_REQUIRE(o->cycles != GL_CYCLES_INF || o->precision == GL_FP64, GL_ERR_ARG,
               "R_inf (cycles = GL_CYCLES_INF) needs precision GL_FP64");
    GL_REQUIRE(o->precision == GL_FP64 || o->precision == GL_MIXED || o->precision == GL_MIXED_PRECOND, GL_ERR_ARG,
               "unknown precision");
    GL_REQUIRE(o->max_coarse <= MAX_COARSE_DENSE, GL_ERR_ARG, "max_coarse must be <= 4096");
    GL_REQUIRE(o->coloring == GL_COLOR_SL || o->coloring == GL_COLOR_JP || o->coloring == GL_COLOR_PSL, GL_ERR_ARG,
               "unknown coloring");
    GL_REQUIRE(o->sweep_sync >= 0 && o->sweep_sync <= 2, GL_ERR_ARG, "sweep_sync must be 0, 1 or 2");
    GL_REQUIRE(o->lattice >= 0 && o->lattice <= 2, GL_ERR_ARG, "lattice must be 0, 1 or 2");
}

void ensure_tmp(gl_mesh_s *m) {
    if (m->t0.n != (size_t)m->n) {
        m->t0.alloc(m->n);
        m->t1.alloc(m->n);
        m->t2.alloc(m->n);
    }
}

void copy_csr_to_host(const CsrDev &A, int64_t *rp, int32_t *ci, void *v) {
    GL_REQUIRE(rp && ci && v, GL_ERR_ARG, "output pointers must not be NULL");
    GL_CUDA(cudaMemcpy(rp, A.rp.get(), (A.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    GL_CUDA(cudaMemcpy(ci, A.ci.get(), A.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    GL_CUDA(cudaMemcpy(v, A.v.get(), A.nnz * sizeof(double2), cudaMemcpyDeviceToHost));
}

}  // namespace

extern "C" {

gl_status gl_options_default(gl_options *o) {
    if (!o) return GL_ERR_ARG;
    o->tol = 1e-10;
    o->maxit = 500;
    o->cycles = 1;
    o->max_coarse = 512;
    o->max_levels = 10;
    o->power_its = 20;
    o->precision = GL_FP64;
    o->inner_tol = 1e-5;
    o->max_outer = 20;
    o->check_every = 6;
    o->autotune = 1;
    o->lattice = 1;
    o->cluster_sweeps = 1;
    o->warmstart = nullptr;
    o->coloring = GL_COLOR_PSL;
    o->sweep_sync = 0;
    o->coarse_df = 1;
    o->device_loop = 1;
    return GL_OK;
}

const char *gl_last_error(void) { return last_error(); }

gl_status gl_mesh_create(int dim, int n_per_side, double mu, const double *bhat, void *stream, gl_mesh *out) {
    return gl_mesh_create_edge(dim, n_per_side, 1.0, mu, bhat, stream, out);
}

gl_status gl_mesh_set_mu(gl_mesh m, double mu, void *stream) {
    return guard([&] {
        GL_REQUIRE(m, GL_ERR_ARG, "NULL mesh");
        mesh_set_mu(m, mu, as_stream(stream));
        return GL_OK;
    });
}

gl_status gl_mesh_create_simplicial(int dim, int64_t n, const double *x_host, int64_t ns, const int32_t *simplices_host,
                                    double mu, const double *bhat, const double *dipole_x0, const double *dipole_m,
                                    void *stream, gl_mesh *out) {
    return guard([&] {
        GL_REQUIRE(out, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE((dipole_x0 == nullptr) == (dipole_m == nullptr), GL_ERR_ARG,
                   "dipole_x0 and dipole_m must both be given or both be NULL");
        *out = nullptr;
        auto *m = new gl_mesh_s();
        try {
            mesh_create_simplicial(m, dim, n, x_host, ns, simplices_host, mu, bhat, dipole_x0, dipole_m,
                                   as_stream(stream));
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return GL_OK;
    });
}

gl_status gl_mesh_create_dipole(int dim, int n_per_side, double edge, double mu, const double *x0, const double *mom,
                                void *stream, gl_mesh *out) {
    return guard([&] {
        GL_REQUIRE(out && x0 && mom, GL_ERR_ARG, "NULL argument");
        *out = nullptr;
        auto *m = new gl_mesh_s();
        try {
            mesh_create(m, dim, n_per_side, edge, mu, nullptr, as_stream(stream), x0, mom);
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return GL_OK;
    });
}

gl_status gl_mesh_create_edge(int dim, int n_per_side, double edge, double mu, const double *bhat, void *stream,
                              gl_mesh *out) {
    return guard([&] {
        GL_REQUIRE(out, GL_ERR_ARG, "out must not be NULL");
        *out = nullptr;
        auto *m = new gl_mesh_s();
        try {
            mesh_create(m, dim, n_per_side, edge, mu, bhat, as_stream(stream));
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return GL_OK;
    });
}

gl_status gl_mesh_destroy(gl_mesh m) {
    return guard([&] {
        if (m) {
            cudaDeviceSynchronize();
            delete m;
        }
        return GL_OK;
    });
}

gl_status gl_mesh_info(gl_mesh m, int64_t *n, int64_t *nnz, double *volumes_dev) {
    return guard([&] {
        GL_REQUIRE(m, GL_ERR_ARG, "mesh must not be NULL");
        if (n) *n = m->n;
        if (nnz) *nnz = m->khat.nnz;
        if (volumes_dev)
            GL_CUDA(cudaMemcpy(volumes_dev, m->vol.get(), m->n * sizeof(double), cudaMemcpyDeviceToDevice));
        return GL_OK;
    });
}

gl_status gl_mesh_nedges(gl_mesh m, int64_t *ne) {
    return guard([&] {
        GL_REQUIRE(m && ne, GL_ERR_ARG, "NULL argument");
        *ne = m->nedges;
        return GL_OK;
    });
}

gl_status gl_mesh_edges(gl_mesh m, int32_t *ej, int32_t *ek, double *alpha, double *theta) {
    return guard([&] {
        GL_REQUIRE(m && ej && ek && alpha && theta, GL_ERR_ARG, "NULL argument");
        size_t ne = (size_t)m->nedges;
        GL_CUDA(cudaMemcpy(ej, m->ej.get(), ne * sizeof(int32_t), cudaMemcpyDeviceToHost));
        GL_CUDA(cudaMemcpy(ek, m->ek.get(), ne * sizeof(int32_t), cudaMemcpyDeviceToHost));
        GL_CUDA(cudaMemcpy(alpha, m->ealpha.get(), ne * sizeof(double), cudaMemcpyDeviceToHost));
        GL_CUDA(cudaMemcpy(theta, m->etheta.get(), ne * sizeof(double), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_mesh_khat(gl_mesh m, int64_t *rp, int32_t *ci, void *v) {
    return guard([&] {
        GL_REQUIRE(m, GL_ERR_ARG, "mesh must not be NULL");
        copy_csr_to_host(m->khat, rp, ci, v);
        return GL_OK;
    });
}

gl_status gl_residual(gl_mesh m, const void *psi, void *r, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi && r, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(psi != r, GL_ERR_ARG, "psi and r must not alias");
        cudaStream_t s = as_stream(stream);
        ensure_tmp(m);
        permute_in(m->n, m->perm.get(), (const double2 *)psi, m->t0.get(), s);
        residual_p(m, m->t0.get(), m->t1.get(), s);
        permute_out(m->n, m->perm.get(), m->t1.get(), (double2 *)r, s);
        return GL_OK;
    });
}

gl_status gl_jacobian_apply(gl_mesh m, const void *psi, const void *phi, void *y, int precision, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi && phi && y, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(y != psi && y != phi, GL_ERR_ARG, "y must not alias psi or phi");
        GL_REQUIRE(precision == GL_FP64 || precision == GL_MIXED || precision == GL_MIXED_PRECOND ||
                       precision == GL_APPLY_FP64_TABLES,
                   GL_ERR_ARG, "unknown precision");
        cudaStream_t s = as_stream(stream);
        ensure_tmp(m);
        permute_in(m->n, m->perm.get(), (const double2 *)psi, m->t0.get(), s);
        permute_in(m->n, m->perm.get(), (const double2 *)phi, m->t1.get(), s);
        if (precision == GL_MIXED_PRECOND) {
            jacobian_apply_pdf(m, m->t0.get(), m->t1.get(), m->t2.get(), s);
        } else if (precision == GL_MIXED) {
            mesh_ensure_fp32(m, s);
            jacobian_apply_p32(m, m->t0.get(), m->t1.get(), m->t2.get(), s);
        } else if (precision == GL_APPLY_FP64_TABLES) {
            jacobian_apply_lat64_p(m, m->t0.get(), m->t1.get(), m->t2.get(), s);
        } else {
            jacobian_apply_p(m, m->t0.get(), m->t1.get(), m->t2.get(), s);
        }
        permute_out(m->n, m->perm.get(), m->t2.get(), (double2 *)y, s);
        return GL_OK;
    });
}

gl_status gl_precond_setup(gl_mesh m, const void *psi, const gl_options *opt, void *stream, gl_prec *out) {
    return guard([&] {
        GL_REQUIRE(m && psi && out, GL_ERR_ARG, "NULL argument");
        check_opts(opt);
        *out = nullptr;
        auto *p = new gl_prec_s();
        try {
            precond_setup(p, m, (const double2 *)psi, *opt, as_stream(stream));
        } catch (...) {
            cudaDeviceSynchronize();
            delete p;
            throw;
        }
        *out = p;
        return GL_OK;
    });
}

gl_status gl_precond_setup_like(gl_mesh m, const void *psi, const gl_options *opt, gl_prec like, void *stream,
                                gl_prec *out) {
    return guard([&] {
        GL_REQUIRE(m && psi && out, GL_ERR_ARG, "NULL argument");
        check_opts(opt);
        *out = nullptr;
        auto *p = new gl_prec_s();
        try {
            precond_setup(p, m, (const double2 *)psi, *opt, as_stream(stream), like);
        } catch (...) {
            cudaDeviceSynchronize();
            delete p;
            throw;
        }
        *out = p;
        return GL_OK;
    });
}

gl_status gl_precond_apply(gl_prec p, const void *x, void *z, void *stream) {
    return guard([&] {
        GL_REQUIRE(p && x && z, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(x != z, GL_ERR_ARG, "x and z must not alias");
        gl_mesh_s *m = p->mesh;
        GL_REQUIRE(p->mesh_version == m->version, GL_ERR_ARG, "preconditioner set up before the mesh's mu changed");
        cudaStream_t s = as_stream(stream);
        ensure_tmp(m);
        permute_in(m->n, m->perm.get(), (const double2 *)x, m->t0.get(), s);
        precond_apply_p(p, m->t0.get(), m->t1.get(), nullptr, s);
        permute_out(m->n, m->perm.get(), m->t1.get(), (double2 *)z, s);
        if (sweeps_failed(p, s)) {
            sweeps_reset(p, s);
            GL_CUDA(cudaStreamSynchronize(s));
            GL_REQUIRE(false, GL_ERR_TIMEOUT, "a coarse-level Gauss-Seidel wait ran out; z is not R x");
        }
        return GL_OK;
    });
}

gl_status gl_precond_apply_precision(gl_prec p, const void *x, void *z, int precision, void *stream) {
    return guard([&] {
        GL_REQUIRE(p && x && z, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(x != z, GL_ERR_ARG, "x and z must not alias");
        GL_REQUIRE(precision == GL_FP64 || precision == GL_MIXED || precision == GL_MIXED_PRECOND, GL_ERR_ARG,
                   "unknown precision");
        if (precision == GL_FP64) return gl_precond_apply(p, x, z, stream);
        GL_REQUIRE(!p->rinf, GL_ERR_ARG, "R_inf runs in FP64 only");
        gl_mesh_s *m = p->mesh;
        GL_REQUIRE(p->mesh_version == m->version, GL_ERR_ARG, "preconditioner set up before the mesh's mu changed");
        cudaStream_t s = as_stream(stream);
        precond_ensure_fp32(p, s);
        ensure_tmp(m);
        permute_in(m->n, m->perm.get(), (const double2 *)x, m->t0.get(), s);
        precond_apply_p64_via32(p, m->t0.get(), m->t1.get(), nullptr, s);
        permute_out(m->n, m->perm.get(), m->t1.get(), (double2 *)z, s);
        if (sweeps_failed(p, s)) {
            sweeps_reset(p, s);
            GL_CUDA(cudaStreamSynchronize(s));
            GL_REQUIRE(false, GL_ERR_TIMEOUT, "a coarse-level Gauss-Seidel wait ran out; z is not R x");
        }
        return GL_OK;
    });
}

gl_status gl_precond_debug(gl_prec p, int action) {
    return guard([&] {
        GL_REQUIRE(p, GL_ERR_ARG, "NULL argument");
        if (action == GL_DEBUG_STALL_SWEEPS) {
            const unsigned long long far = 1ull << 40;
            GL_CUDA(cudaMemcpy(p->wait_extra.get(), &far, sizeof far, cudaMemcpyHostToDevice));
        } else if (action == GL_DEBUG_NEGATE_COARSEST) {
            precond_negate_coarsest(p, nullptr);
        } else {
            GL_REQUIRE(false, GL_ERR_ARG, "unknown debug action");
        }
        return GL_OK;
    });
}

gl_status gl_precond_cost(gl_prec p, int cycles, double *matvecs) {
    return guard([&] {
        GL_REQUIRE(p && matvecs, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(cycles >= 1 && cycles <= 64, GL_ERR_ARG, "cycles must be in [1, 64]");
        *matvecs = precond_cost(p, cycles);
        return GL_OK;
    });
}

gl_status gl_precond_destroy(gl_prec p) {
    return guard([&] {
        if (p) {
            cudaDeviceSynchronize();
            delete p;
        }
        return GL_OK;
    });
}

gl_status gl_precond_levels(gl_prec p, int *nlev) {
    return guard([&] {
        GL_REQUIRE(p && nlev, GL_ERR_ARG, "NULL argument");
        *nlev = p->nlev;
        return GL_OK;
    });
}

gl_status gl_precond_level_info(gl_prec p, int l, int64_t *n, int64_t *nnz, int32_t *ncolors, int64_t *p_nnz,
                                double *omega) {
    return guard([&] {
        GL_REQUIRE(p && l >= 0 && l < p->nlev, GL_ERR_ARG, "bad level");
        const Level &L = p->L[l];
        bool last = (l == p->nlev - 1);
        if (n) *n = L.n;
        if (nnz) *nnz = L.A_can.nnz;
        if (ncolors) *ncolors = L.ncolors;
        if (p_nnz) *p_nnz = last ? 0 : L.P_can.nnz;
        if (omega) *omega = last ? 0.0 : L.omega;
        return GL_OK;
    });
}

gl_status gl_precond_level_sweep(gl_prec p, int l, int precision, int *lanes, int *sync, int *ctas) {
    return guard([&] {
        GL_REQUIRE(p && l >= 0 && l < p->nlev, GL_ERR_ARG, "bad level");
        GL_REQUIRE(precision == GL_FP64 || ((precision == GL_MIXED || precision == GL_MIXED_PRECOND) && p->has32),
                   GL_ERR_ARG, "no sweep of that precision (FP32 copies not built)");
        const Level &L = p->L[l];
        const bool f32 = precision != GL_FP64;
        const bool coarse = l > 0 && l < p->nlev - 1;
        if (lanes) *lanes = coarse ? (f32 ? L.sgs_G32 : L.sgs_G64) : 0;
        int sy = -1, nb = 0;
        if (coarse) {
            if (f32 && L.cl_size > 0 && p->cluster_sweeps) {
                sy = 3;
                nb = L.cl_size;
            } else {
                sy = f32 ? L.sync32 : L.sync64;
                nb = sy == 1 ? (f32 ? L.fl32.nb : L.fl64.nb) : 0;
            }
        }
        if (sync) *sync = sy;
        if (ctas) *ctas = nb;
        return GL_OK;
    });
}

gl_status gl_precond_level_aggregates(gl_prec p, int l, int32_t *agg) {
    return guard([&] {
        GL_REQUIRE(p && agg && l >= 0 && l < p->nlev - 1, GL_ERR_ARG, "bad level");
        GL_CUDA(cudaMemcpy(agg, p->L[l].agg.get(), p->L[l].n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_precond_level_colors(gl_prec p, int l, int32_t *col) {
    return guard([&] {
        GL_REQUIRE(p && col && l >= 0 && l < p->nlev, GL_ERR_ARG, "bad level");
        GL_CUDA(cudaMemcpy(col, p->L[l].color.get(), p->L[l].n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_precond_level_matrix(gl_prec p, int l, int64_t *rp, int32_t *ci, void *v) {
    return guard([&] {
        GL_REQUIRE(p && l >= 0 && l < p->nlev, GL_ERR_ARG, "bad level");
        copy_csr_to_host(p->L[l].A_can, rp, ci, v);
        return GL_OK;
    });
}

gl_status gl_precond_level_P(gl_prec p, int l, int64_t *rp, int32_t *ci, void *v) {
    return guard([&] {
        GL_REQUIRE(p && l >= 0 && l < p->nlev - 1, GL_ERR_ARG, "bad level");
        copy_csr_to_host(p->L[l].P_can, rp, ci, v);
        return GL_OK;
    });
}

gl_status gl_jacobian_solve(gl_mesh m, const void *psi, gl_prec prec, const void *b, void *x, const gl_options *opt,
                            gl_solve_info *info, void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi && b && x, GL_ERR_ARG, "NULL argument");
        check_opts(opt);
        GL_REQUIRE(!prec || prec->mesh == m, GL_ERR_ARG, "preconditioner belongs to another mesh");
        GL_REQUIRE(!prec || prec->mesh_version == m->version, GL_ERR_ARG,
                   "preconditioner set up before the mesh's mu changed");
        cudaStream_t s = as_stream(stream);
        gl_solve_info inf{};
        gl_prec_s *p = prec;
        gl_prec_s *own = nullptr;
        if (!p && opt->cycles != 0) {
            auto t0 = std::chrono::steady_clock::now();
            own = new gl_prec_s();
            try {
                precond_setup(own, m, (const double2 *)psi, *opt, s);
            } catch (...) {
                cudaDeviceSynchronize();
                delete own;
                throw;
            }
            p = own;
            inf.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        gl_status st;
        try {
            ensure_tmp(m);
            double2 *psi_p = p ? p->psi_p.get() : m->t0.get();
            if (!p) permute_in(m->n, m->perm.get(), (const double2 *)psi, m->t0.get(), s);
            permute_in(m->n, m->perm.get(), (const double2 *)b, m->t1.get(), s);
            permute_in(m->n, m->perm.get(), (const double2 *)x, m->t2.get(), s);
            st = jacobian_solve_p(m, p, psi_p, m->t1.get(), m->t2.get(), *opt, &inf, s);
            permute_out(m->n, m->perm.get(), m->t2.get(), (double2 *)x, s);
            GL_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            if (own) {
                cudaDeviceSynchronize();
                delete own;
            }
            throw;
        }
        if (own) delete own;
        if (info) *info = inf;
        if (st != GL_OK) {
            char buf[160];
            snprintf(buf, sizeof buf, "solve stopped after %d iterations at relative residual %.3e", inf.iters,
                     inf.true_relres);
            set_error(buf);
        }
        return st;
    });
}

gl_status gl_newton_step(gl_mesh m, void *psi, const gl_options *opt, gl_solve_info *info, double *gl_norm_out,
                         void *stream) {
    return guard([&] {
        GL_REQUIRE(m && psi, GL_ERR_ARG, "NULL argument");
        check_opts(opt);
        cudaStream_t s = as_stream(stream);
        int64_t n = m->n;
        DBuf<double2> r(n), d(n);
        DBuf<double> part(RED_BLOCKS), scal(1);
        // r = -GL(psi) and ||GL(psi)||_R, on the device
        gl_status st = gl_residual(m, psi, r.get(), stream);
        GL_REQUIRE(st == GL_OK, st, last_error());
        double g = newton_rhs(m, r.get(), part.get(), scal.get(), s);
        if (gl_norm_out) *gl_norm_out = g;
        GL_CUDA(cudaMemsetAsync(d.get(), 0, n * sizeof(double2), s));
        st = gl_jacobian_solve(m, psi, nullptr, r.get(), d.get(), opt, info, stream);
        if (st != GL_OK && st != GL_ERR_NOT_CONVERGED) return st;
        newton_update(n, d.get(), static_cast<double2 *>(psi), s);
        GL_CUDA(cudaStreamSynchronize(s));
        return st;
    });
}

gl_status gl_batch_create(int count, const gl_mesh *meshes, const void *const *psi, const gl_options *opt, void *stream,
                          gl_batch *out) {
    return guard([&] {
        GL_REQUIRE(out && count > 0 && meshes && psi, GL_ERR_ARG, "NULL argument or empty batch");
        check_opts(opt);
        for (int i = 0; i < count; ++i) GL_REQUIRE(meshes[i] && psi[i], GL_ERR_ARG, "NULL mesh or psi in batch");
        GL_REQUIRE(opt->cycles >= 1, GL_ERR_ARG, "batched solves need a preconditioner (cycles >= 1)");
        *out = nullptr;
        gl_batch_s *B = batch_new();
        try {
            batch_create(B, count, meshes, reinterpret_cast<const double2 *const *>(psi), *opt, as_stream(stream));
        } catch (...) {
            batch_delete(B);
            throw;
        }
        *out = B;
        return GL_OK;
    });
}

gl_status gl_batch_run(gl_batch B, const void *const *b, void *const *x, gl_solve_info *infos, void *stream) {
    return guard([&] {
        GL_REQUIRE(B && b && x, GL_ERR_ARG, "NULL argument");
        for (size_t i = 0; i < batch_size(B); ++i) GL_REQUIRE(b[i] && x[i], GL_ERR_ARG, "NULL b or x in batch");
        gl_status st = batch_run(B, reinterpret_cast<const double2 *const *>(b), reinterpret_cast<double2 *const *>(x),
                                 infos, as_stream(stream));
        if (st != GL_OK) set_error("at least one batched solve did not converge");
        return st;
    });
}

gl_status gl_batch_destroy(gl_batch B) {
    return guard([&] {
        if (B) batch_delete(B);
        return GL_OK;
    });
}

gl_status gl_batch_solve(int count, const gl_mesh *meshes, const void *const *psi, const void *const *b,
                         void *const *x, const gl_options *opt, gl_solve_info *infos, void *stream) {
    if (count == 0) return GL_OK;
    gl_batch B = nullptr;
    gl_status st = gl_batch_create(count, meshes, psi, opt, stream, &B);
    if (st != GL_OK) return st;
    st = gl_batch_run(B, b, x, infos, stream);
    std::string msg = last_error();
    gl_batch_destroy(B);
    if (st != GL_OK) set_error(msg);
    return st;
}

gl_status gl_profile_begin(const char *kernel_class, int max_launches) {
    return guard([&] {
        GL_REQUIRE(max_launches >= 0 && max_launches <= (1 << 20), GL_ERR_ARG, "max_launches out of range");
        Profiler &p = profiler();
        GL_CUDA(cudaDeviceSynchronize());
        for (auto e : p.ev) cudaEventDestroy(e);
        p.ev.clear();
        p.name = kernel_class ? kernel_class : "";
        int slots = p.name.empty() ? 0 : max_launches;
        p.ev.resize(2 * (size_t)slots);
        for (auto &e : p.ev) GL_CUDA(cudaEventCreate(&e));
        p.slot_bytes.assign(slots, 0.0);
        p.slot_flops.assign(slots, 0.0);
        p.free_slots.clear();
        for (int i = slots - 1; i >= 0; --i) p.free_slots.push_back(i);
        p.pending.clear();
        p.capture = nullptr;
        p.total_ms = p.total_bytes = p.total_flops = 0;
        p.timed = p.dropped = 0;
        p.launches.store(0);
        p.retarget(p.name);
        p.active = true;
        return GL_OK;
    });
}

gl_status gl_profile_flops(double *alg_flops) {
    return guard([&] {
        GL_REQUIRE(alg_flops, GL_ERR_ARG, "NULL argument");
        *alg_flops = profiler().last_flops;
        return GL_OK;
    });
}

gl_status gl_profile_end(int64_t *launches, int64_t *timed, double *total_ms, double *alg_bytes) {
    return guard([&] {
        Profiler &p = profiler();
        GL_REQUIRE(p.active, GL_ERR_ARG, "gl_profile_begin was not called");
        GL_CUDA(cudaDeviceSynchronize());
        p.harvest_direct();
        if (launches) *launches = p.launches.load();
        if (timed) *timed = p.timed;
        if (total_ms) *total_ms = p.total_ms;
        if (alg_bytes) *alg_bytes = p.total_bytes;
        p.last_flops = p.total_flops;
        for (auto e : p.ev) cudaEventDestroy(e);
        p.ev.clear();
        p.free_slots.clear();
        p.active = false;
        p.name.clear();
        p.retarget("");
        return GL_OK;
    });
}

}  // extern "C"
