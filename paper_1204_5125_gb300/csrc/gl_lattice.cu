// gl_lattice.cu -- the finest-level operator of the structured meshes without a
// stored matrix.
//
// On the uniform lattice (nodes x = (-1/2 + i h, -1/2 + j h[, -1/2 + k h]),
// h = 1/(N-1)) only the axis edges carry a coefficient (the diagonals of the
// triangles and tetrahedra get alpha = 0, Corollary "simplex"), and every cell
// is split the same way, so the coefficient of an edge along axis e does not
// depend on its position along e: alpha_ik depends on the perpendicular
// coordinates only (through the boundary faces the edge lies on).  The link
// phase theta_ik = integral of A from x_i to x_k (Eq. link variable) is, for
// A = (mu/2) bhat x x, s h (mu/2) x_i . (e x bhat) for k = i + s e: also a
// function of the perpendicular coordinates.  Hence the off-diagonal
// K-hat_{i, i+e} = -alpha exp(-i theta) (Eq. (10)) is tabulated per axis over
// the N^(d-1) perpendicular positions, K-hat_{i, i-e} is the conjugate of the
// table entry of the edge (i - e, i) (K-hat is Hermitian, same perpendicular
// position), and the row of K = D^-1 K-hat is scaled by 1 / |V_i|.  A row then
// costs its vector entries, |V_i| and table reads that stay in cache instead of
// a stored stencil.
//
// The solve ordering puts the red nodes ((i + j + k) even) first, each colour in
// natural order.  For even N every lattice row holds N/2 nodes of each colour,
// so node v sits at position v / 2 (+ n / 2 if black) and the position of a
// neighbour follows from its node number.
//
// The tables are filled from the assembled K-hat (the edge starting at
// coordinate 0 along e), and the closed form is enabled only after every stored
// entry of the assembled FP64 operator K has been found equal to the table
// value (relative difference <= 1e-12 of the largest entry) and every row to
// hold exactly its lattice neighbours; otherwise the sliced-ELL kernels stay.
// The FP64 Jacobian takes the FP64 tables under a tighter test: every entry within
// 16 ulp of the largest and every control volume h^d 2^-b to 2 ulp (its row
// scale 2^b / h^d then needs no division).
#include <cfloat>

#include "gl_internal.cuh"

namespace gl {

namespace {

struct LatDev {
    int dim, N;
    int64_t n;
};

__device__ __forceinline__ void lat_coords(const LatDev &L, int64_t v, int c[3]) {
    c[0] = (int)(v % L.N);
    c[1] = (int)((v / L.N) % L.N);
    c[2] = L.dim == 3 ? (int)(v / ((int64_t)L.N * L.N)) : 0;
}
// perpendicular index of node coordinates c for axis e (other axes in increasing order)
__device__ __forceinline__ int64_t lat_perp(const LatDev &L, int e, const int c[3]) {
    if (e == 0) return c[1] + (int64_t)L.N * c[2];
    if (e == 1) return c[0] + (int64_t)L.N * c[2];
    return c[0] + (int64_t)L.N * c[1];
}

// table entry (axis e, perpendicular index idx) = K-hat of the edge from the node
// at coordinate 0 along e to its +e neighbour (0 if K-hat has no such entry)
__global__ void k_lat_tables(LatDev L, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double2 *__restrict__ kv, double2 *tab, int64_t per_axis) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= per_axis * L.dim) return;
    int e = (int)(t / per_axis);
    int64_t idx = t % per_axis;
    int a = (int)(idx % L.N), b = (int)(idx / L.N);
    int c[3] = {0, 0, 0};
    if (e == 0) {
        c[1] = a;
        c[2] = b;
    } else if (e == 1) {
        c[0] = a;
        c[2] = b;
    } else {
        c[0] = a;
        c[1] = b;
    }
    const int64_t stride[3] = {1, L.N, (int64_t)L.N * L.N};
    int64_t v = c[0] + stride[1] * c[1] + stride[2] * c[2];
    int64_t u = v + stride[e];
    double2 val = make_double2(0.0, 0.0);
    for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
        if (ci[q] == u) val = kv[q];
    tab[t] = val;
}

// compares every stored entry of K (solve ordering, FP64) with the table value
// (bad: beyond tol); bad64 also counts entries beyond tol64 and control volumes
// other than h^d 2^-b (b the node's boundary coordinates), the scale the FP64
// stencil applies
__global__ void k_lat_check(LatDev L, SellView<double2> K, const int32_t *__restrict__ perm,
                            const double *__restrict__ vol, const double2 *__restrict__ tab, int64_t per_axis,
                            double tol, unsigned *bad, double tol64, unsigned *bad64, double hd) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= L.n) return;
    const int N = L.N;
    const int64_t v = perm[p];
    int cc[3];
    lat_coords(L, v, cc);
    {
        int b = 0;
        for (int e = 0; e < L.dim; ++e) b += (cc[e] == 0 || cc[e] == N - 1);
        if (fabs(vol[v] - hd / (double)(1 << b)) > 2.0 * DBL_EPSILON * vol[v]) atomicAdd(bad64, 1u);
    }
    const int64_t stride[3] = {1, N, (int64_t)N * N};
    int expect = 0;
    for (int e = 0; e < L.dim; ++e) {
        const double2 t = tab[e * per_axis + lat_perp(L, e, cc)];
        const bool nz = t.x != 0.0 || t.y != 0.0;
        expect += (cc[e] < N - 1 && nz) + (cc[e] > 0 && nz);
    }
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    int found = 0;
    bool ok = true;
    for (int q = 0; q < w && ok; ++q) {
        int64_t en = beg + (int64_t)q * SELL_C + lane;
        double2 val = K.val[en];
        if (val.x == 0.0 && val.y == 0.0) continue;
        int64_t d = (int64_t)perm[K.col[en]] - v;
        int e = -1, sg = 0;
        for (int a = 0; a < L.dim; ++a) {
            if (d == stride[a] && cc[a] < N - 1) e = a, sg = 1;
            if (d == -stride[a] && cc[a] > 0) e = a, sg = -1;
        }
        if (e < 0) {
            ok = false;
            break;
        }
        double2 t = tab[e * per_axis + lat_perp(L, e, cc)];
        double ex = t.x / vol[v], ey = (sg > 0 ? t.y : -t.y) / vol[v];
        if (fabs(val.x - ex) > tol || fabs(val.y - ey) > tol) ok = false;
        if (fabs(val.x - ex) > tol64 || fabs(val.y - ey) > tol64) atomicAdd(bad64, 1u);
        ++found;
    }
    if (!ok || found != expect) atomicAdd(bad, 1u);
}

__global__ void k_lat_round(int64_t m, const double2 *__restrict__ a, float2 *__restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__device__ __forceinline__ float2 split2(double x) {
    float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
// double-float magnitude a = |K-hat| / h^d and unit phase u = -K-hat / |K-hat| of
// every table entry
__global__ void k_lat_df(int64_t m, const double2 *__restrict__ t, double hd, float2 *__restrict__ a,
                         float4 *__restrict__ u) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 k = make_double2(t[i].x / hd, t[i].y / hd);
    double mag = sqrt(k.x * k.x + k.y * k.y);
    double ur = mag > 0 ? -k.x / mag : 0.0, ui = mag > 0 ? -k.y / mag : 0.0;
    a[i] = split2(mag);
    float2 re = split2(ur), im = split2(ui);
    u[i] = make_float4(re.x, re.y, im.x, im.y);
}
// K_ii - sum_k |K_ik| over the stored row (solve ordering, FP64)
__global__ void k_lat_krem(int64_t n, SellView<double2> K, const double *__restrict__ kd, double *__restrict__ rem) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    double sum = 0;
    for (int q = 0; q < w; ++q) {
        double2 v = K.val[beg + (int64_t)q * SELL_C + lane];
        sum += sqrt(v.x * v.x + v.y * v.y);
    }
    rem[p] = kd[p] - sum;
}

}  // namespace

// fills the tables from the assembled K-hat and checks them against K; with
// `reuse` the buffers of an earlier call are rewritten in place.  Returns
// whether the check passed (the tables are left unused otherwise).
static bool lattice_tables(gl_mesh_s *m, bool reuse, cudaStream_t s) {
    LatDev L{m->dim, m->N, m->n};
    const int64_t per_axis = m->dim == 3 ? (int64_t)m->N * m->N : m->N;
    DBuf<double2> tab64((size_t)per_axis * m->dim);
    k_lat_tables<<<grid_for(per_axis * m->dim, 256), 256, 0, s>>>(L, m->khat.rp.get(), m->khat.ci.get(), m->khat.v.get(),
                                                                   tab64.get(), per_axis);
    GL_LAUNCH_CHECK();
    DBuf<unsigned> bad(2);
    GL_CUDA(cudaMemsetAsync(bad.get(), 0, 2 * sizeof(unsigned), s));
    double kmax = 0;
    {
        // largest |K| entry bounds the tolerance: the row sums of |K| are the diagonal
        std::vector<double> kd(m->n);
        GL_CUDA(cudaMemcpyAsync(kd.data(), m->kdiag.get(), m->n * sizeof(double), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        for (double v : kd) kmax = std::max(kmax, std::fabs(v));
    }
    k_lat_check<<<grid_for(m->n, 256), 256, 0, s>>>(L, m->K.view(), m->perm.get(), m->vol.get(), tab64.get(),
                                                    per_axis, 1e-12 * kmax, bad.get(), 16.0 * DBL_EPSILON * kmax,
                                                    bad.get() + 1, m->dim == 2 ? m->h * m->h : m->h * m->h * m->h);
    GL_LAUNCH_CHECK();
    unsigned nbad[2] = {0, 0};
    GL_CUDA(cudaMemcpyAsync(nbad, bad.get(), 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    m->lat64_ok = false;
    if (nbad[0] != 0) return false;
    if (!reuse) {
        m->lat_tab64.alloc((size_t)per_axis * m->dim);
        m->lat_tab.alloc((size_t)per_axis * m->dim);
        m->lat_a.alloc((size_t)per_axis * m->dim);
        m->lat_u.alloc((size_t)per_axis * m->dim);
        m->lat_krem.alloc(m->n);
    }
    k_lat_round<<<grid_for(per_axis * m->dim, 256), 256, 0, s>>>(per_axis * m->dim, tab64.get(), m->lat_tab.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaMemcpyAsync(m->lat_tab64.get(), tab64.get(), (size_t)per_axis * m->dim * sizeof(double2),
                            cudaMemcpyDeviceToDevice, s));
    m->lat64_ok = nbad[1] == 0;
    // double-float tables: the control volumes are h^d 2^-b exactly (b boundary
    // coordinates), so K_ik = 2^b (K-hat_ik / h^d) with an exact power-of-2 factor
    m->lat_hd = m->dim == 2 ? m->h * m->h : m->h * m->h * m->h;
    k_lat_df<<<grid_for(per_axis * m->dim, 256), 256, 0, s>>>(per_axis * m->dim, tab64.get(), m->lat_hd,
                                                               m->lat_a.get(), m->lat_u.get());
    k_lat_krem<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, m->K.view(), m->kdiag.get(), m->lat_krem.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
    m->lat_per_axis = per_axis;
    return true;
}

void mesh_ensure_lattice(gl_mesh_s *m, cudaStream_t s) {
    if (m->lat_checked) return;
    m->lat_checked = true;
    m->lat_ok = false;
    if (m->N % 2 != 0 || m->N < 4 || m->nred * 2 != m->n) return;
    m->lat_ok = lattice_tables(m, false, s);
}

void mesh_refresh_lattice(gl_mesh_s *m, cudaStream_t s) {
    if (!m->lat_checked || !m->lat_ok) return;
    m->lat_ok = lattice_tables(m, true, s);
}

LatticeDfView lattice_df_view(const gl_mesh_s *m) {
    LatticeDfView v{};
    v.dim = m->dim;
    v.N = m->N;
    v.dN = DivU32::make((uint32_t)m->N);
    v.nred = m->nred;
    v.per_axis = m->lat_per_axis;
    v.a = m->lat_a.get();
    v.u = m->lat_u.get();
    return v;
}

LatticeView64 lattice_view64(const gl_mesh_s *m) {
    LatticeView64 v{};
    v.dim = m->dim;
    v.N = m->N;
    v.dN = DivU32::make((uint32_t)m->N);
    v.nred = m->nred;
    v.vol = m->volp.get();
    v.tx = m->lat_tab64.get();
    v.ty = v.tx + m->lat_per_axis;
    v.tz = m->dim == 3 ? v.ty + m->lat_per_axis : nullptr;
    v.ihd = 1.0 / m->lat_hd;
    return v;
}

LatticeView lattice_view(const gl_mesh_s *m) {
    LatticeView v{};
    v.dim = m->dim;
    v.N = m->N;
    v.dN = DivU32::make((uint32_t)m->N);
    v.nred = m->nred;
    v.vol = m->volp32.get();
    v.tx = m->lat_tab.get();
    v.ty = v.tx + m->lat_per_axis;
    v.tz = m->dim == 3 ? v.ty + m->lat_per_axis : nullptr;
    return v;
}

}  // namespace gl
