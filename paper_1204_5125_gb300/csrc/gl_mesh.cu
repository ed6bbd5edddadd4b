// gl_mesh.cu -- assembly of the finite-volume discretisation (Sec. 3 of
// Schloemer & Vanroose) on structured square/cube meshes, entirely on the GPU:
//   * per-simplex edge coefficients: the cotangent formula for triangles (Remark
//     after Cor. "simplex") and the SPD system M alpha = b, M_ij = <e_i,e_j>^2,
//     b_i = |S| ||e_i||^2 for tetrahedra (Cor. "simplex"),
//   * alpha_jk summed over the simplices adjacent to edge jk (Eq. fhat),
//   * control volumes |V_j| (Eq. mass lumping) and link phases
//     theta_jk = integral of A from x_j to x_k (Eq. link variable, midpoint rule,
//     exact for the affine A = (mu/2) bhat x x),
//   * K-hat (Eq. discr kin energy, Remark rmk:dk) as a CSR in node order, and
//     K = D^-1 K-hat as a sliced-ELL in the red-black solve ordering.
#include "gl_internal.cuh"

namespace gl {

// ---------------------------------------------------------------- lattice geometry
constexpr int GL_QUAD = 8;  // Gauss-Legendre points of the dipole's edge phases

struct Lattice {
    int dim, N;
    double h, mu, b[3];
    double x0;  // coordinate of the first node on every axis (-edge / 2)
    // A = mu A_d, the dipole field (moment md at xd), when dipole != 0; its edge
    // phases use the Gauss-Legendre rule (gx, gw) on [-1, 1]
    int dipole;
    double xd[3], md[3], gx[GL_QUAD], gw[GL_QUAD];
    __device__ __host__ int64_t id(int i, int j, int k) const { return (int64_t)i + (int64_t)N * ((int64_t)j + (int64_t)N * k); }
    __device__ __host__ void coords(int64_t v, int &i, int &j, int &k) const {
        i = (int)(v % N);
        int64_t r = v / N;
        j = (int)(r % N);
        k = (int)(r / N);
    }
    __device__ void pos(int i, int j, int k, double *x) const {
        x[0] = x0 + i * h;
        x[1] = x0 + j * h;
        x[2] = (dim == 3) ? x0 + k * h : 0.0;
    }
};

// local vertex offsets (0/1 per axis) of the simplices of one cell
// 2D: two triangles split along the (0,0)-(1,1) diagonal
__constant__ int c_tri[2][3][2] = {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}};
// 3D: Kuhn tetrahedra, one per axis order, walking from (0,0,0) to (1,1,1)
__constant__ int c_kuhn_order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ void simplex_local(int dim, int s, int v, int off[3]) {
    off[0] = off[1] = off[2] = 0;
    if (dim == 2) {
        off[0] = c_tri[s][v][0];
        off[1] = c_tri[s][v][1];
        return;
    }
    for (int st = 0; st < v; ++st) off[c_kuhn_order[s][st]] += 1;
}

// edge e of a simplex with d+1 vertices: (0,1),(0,2),..,(0,d),(1,2),...
__device__ void simplex_edge(int dim, int e, int &a, int &b) {
    int q = 0;
    for (int i = 0; i <= dim; ++i)
        for (int j = i + 1; j <= dim; ++j) {
            if (q == e) {
                a = i;
                b = j;
                return;
            }
            ++q;
        }
}

// Edge coefficients of one simplex (vertices p, 3 doubles each).
__device__ void simplex_alpha(int dim, const double p[4][3], double *alpha) {
    if (dim == 2) {
        // 1/2 t / sqrt(1 - t^2), t = cosine of the angle opposite the edge
        for (int e = 0; e < 3; ++e) {
            int a, b;
            simplex_edge(2, e, a, b);
            int k = 3 - a - b;
            double u0 = p[a][0] - p[k][0], u1 = p[a][1] - p[k][1];
            double v0 = p[b][0] - p[k][0], v1 = p[b][1] - p[k][1];
            double t = (u0 * v0 + u1 * v1) / sqrt((u0 * u0 + u1 * u1) * (v0 * v0 + v1 * v1));
            alpha[e] = 0.5 * t / sqrt(1.0 - t * t);
        }
        return;
    }
    double ev[6][3];
    for (int e = 0; e < 6; ++e) {
        int a, b;
        simplex_edge(3, e, a, b);
        for (int c = 0; c < 3; ++c) ev[e][c] = p[b][c] - p[a][c];
    }
    double e1[3], e2[3], e3[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = p[1][c] - p[0][c];
        e2[c] = p[2][c] - p[0][c];
        e3[c] = p[3][c] - p[0][c];
    }
    double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                 e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
    double vol = fabs(det) / 6.0;
    double M[6][6], rhs[6];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 6; ++j) {
            double d = ev[i][0] * ev[j][0] + ev[i][1] * ev[j][1] + ev[i][2] * ev[j][2];
            M[i][j] = d * d;
        }
        rhs[i] = vol * (ev[i][0] * ev[i][0] + ev[i][1] * ev[i][1] + ev[i][2] * ev[i][2]);
    }
    // Cholesky M = L L^T (in place, lower), then two triangular solves
    for (int j = 0; j < 6; ++j) {
        double s = M[j][j];
        for (int k = 0; k < j; ++k) s -= M[j][k] * M[j][k];
        double l = sqrt(s);
        M[j][j] = l;
        for (int i = j + 1; i < 6; ++i) {
            double t = M[i][j];
            for (int k = 0; k < j; ++k) t -= M[i][k] * M[j][k];
            M[i][j] = t / l;
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= M[i][k] * y[k];
        y[i] = s / M[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= M[k][i] * alpha[k];
        alpha[i] = s / M[i][i];
    }
}

// alphaT[cell][simplex][edge] for every cell of the lattice
__global__ void k_simplex_alpha(Lattice L, int64_t ncell, double *alphaT) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int M = L.N - 1;
    int i = (int)(c % M), j = (int)((c / M) % M), k = (L.dim == 3) ? (int)(c / ((int64_t)M * M)) : 0;
    int ns = (L.dim == 2) ? 2 : 6, ne = (L.dim == 2) ? 3 : 6;
    for (int s = 0; s < ns; ++s) {
        double p[4][3];
        for (int v = 0; v <= L.dim; ++v) {
            int off[3];
            simplex_local(L.dim, s, v, off);
            L.pos(i + off[0], j + off[1], k + off[2], p[v]);
        }
        double al[6];
        simplex_alpha(L.dim, p, al);
        for (int e = 0; e < ne; ++e) alphaT[(c * ns + s) * ne + e] = al[e];
    }
}

// positive directions of the candidate edges (2D: x, y, xy; 3D: x, y, z, xy, xz, yz, xyz)
__constant__ int c_dir2[3][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}};
__constant__ int c_dir3[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

__device__ void dir_vec(int dim, int d, int v[3]) {
    for (int c = 0; c < 3; ++c) v[c] = (dim == 2) ? c_dir2[d][c] : c_dir3[d][c];
}

// Eq. fhat: alpha of edge (node, node + dir) = sum over the simplices containing
// it, gathered in a fixed order (cells by local offset, simplices, edges).
__global__ void k_edge_alpha(Lattice L, int64_t n, int ndir, const double *alphaT, double *ealpha) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * ndir) return;
    int64_t v = t / ndir;
    int d = (int)(t % ndir);
    int i, j, k;
    L.coords(v, i, j, k);
    int dv[3];
    dir_vec(L.dim, d, dv);
    int x0[3] = {i, j, k};
    double acc = 0;
    bool inside = (i + dv[0] < L.N) && (j + dv[1] < L.N) && (L.dim == 2 || k + dv[2] < L.N);
    if (inside) {
        int M = L.N - 1;
        int ns = (L.dim == 2) ? 2 : 6, ne = (L.dim == 2) ? 3 : 6;
        int ncand = 1 << L.dim;
        for (int q = 0; q < ncand; ++q) {
            int va[3] = {q & 1, (q >> 1) & 1, (L.dim == 3) ? (q >> 2) & 1 : 0};
            bool ok = true;
            int cc[3];
            for (int a = 0; a < L.dim; ++a) {
                if (va[a] + dv[a] > 1) ok = false;
                cc[a] = x0[a] - va[a];
                if (cc[a] < 0 || cc[a] >= M) ok = false;
            }
            if (!ok) continue;
            int64_t cell = (int64_t)cc[0] + (int64_t)M * ((int64_t)cc[1] + (L.dim == 3 ? (int64_t)M * cc[2] : 0));
            for (int s = 0; s < ns; ++s)
                for (int e = 0; e < ne; ++e) {
                    int a, b;
                    simplex_edge(L.dim, e, a, b);
                    int oa[3], ob[3];
                    simplex_local(L.dim, s, a, oa);
                    simplex_local(L.dim, s, b, ob);
                    bool fwd = true, bwd = true;
                    for (int c = 0; c < 3; ++c) {
                        if (oa[c] != va[c] || ob[c] != va[c] + dv[c]) fwd = false;
                        if (ob[c] != va[c] || oa[c] != va[c] + dv[c]) bwd = false;
                    }
                    if (fwd || bwd) acc += alphaT[(cell * ns + s) * ne + e];
                }
        }
    }
    ealpha[t] = acc;
}

// Neighbour list of a node: up to 2 ndir candidate edges, in ascending column order.
struct Nbr {
    int64_t col;
    double alpha;
};

__device__ int node_neighbours(const Lattice &L, int64_t v, int ndir, const double *ealpha, double cut, Nbr *out) {
    int i, j, k;
    L.coords(v, i, j, k);
    int x0[3] = {i, j, k};
    int cnt = 0;
    for (int d = 0; d < ndir; ++d) {
        int dv[3];
        dir_vec(L.dim, d, dv);
        int64_t off = (int64_t)dv[0] + (int64_t)L.N * ((int64_t)dv[1] + (int64_t)L.N * dv[2]);
        // forward edge (v, v + dir)
        double a = ealpha[v * ndir + d];
        if (fabs(a) > cut) out[cnt++] = Nbr{v + off, a};
        // backward edge (v - dir, v)
        bool ok = true;
        for (int c = 0; c < L.dim; ++c)
            if (x0[c] - dv[c] < 0) ok = false;
        if (ok) {
            double b = ealpha[(v - off) * ndir + d];
            if (fabs(b) > cut) out[cnt++] = Nbr{v - off, b};
        }
    }
    for (int s = 1; s < cnt; ++s) {  // insertion sort by column
        Nbr key = out[s];
        int r = s - 1;
        while (r >= 0 && out[r].col > key.col) {
            out[r + 1] = out[r];
            --r;
        }
        out[r + 1] = key;
    }
    return cnt;
}

__global__ void k_row_len(Lattice L, int64_t n, int ndir, const double *ealpha, double cut, int64_t *len,
                          int64_t *fwd) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    Nbr nb[16];
    int c = node_neighbours(L, v, ndir, ealpha, cut, nb);
    len[v] = c + 1;
    int64_t f = 0;
    for (int s = 0; s < c; ++s) f += (nb[s].col > v);
    fwd[v] = f;
}

__device__ double edge_phase1(const Lattice &L, const double *xa, const double *xb);

// integral of A = (mu/2) bhat x x along the straight edge from xa to xb (midpoint
// rule, exact for the affine A), or of mu A_d for the dipole
__device__ double edge_phase(const Lattice &L, const double *xa, const double *xb) {
    if (L.dipole) return L.mu * edge_phase1(L, xa, xb);
    double m[3], d[3];
    for (int c = 0; c < 3; ++c) {
        m[c] = 0.5 * (xa[c] + xb[c]);
        d[c] = xb[c] - xa[c];
    }
    double A0 = 0.5 * L.mu * (L.b[1] * m[2] - L.b[2] * m[1]);
    double A1 = 0.5 * L.mu * (L.b[2] * m[0] - L.b[0] * m[2]);
    double A2 = 0.5 * L.mu * (L.b[0] * m[1] - L.b[1] * m[0]);
    return A0 * d[0] + A1 * d[1] + A2 * d[2];
}

// the same integral per unit mu (A_1 = (1/2) bhat x x): theta = mu theta1; for
// the dipole A_1 = A_d = md x (x - xd) / |x - xd|^3, which is not polynomial,
// integrated with the Gauss-Legendre rule along the edge
__device__ double edge_phase1(const Lattice &L, const double *xa, const double *xb) {
    double m[3], d[3];
    for (int c = 0; c < 3; ++c) {
        m[c] = 0.5 * (xa[c] + xb[c]);
        d[c] = xb[c] - xa[c];
    }
    if (L.dipole) {
        double sum = 0;
        for (int q = 0; q < GL_QUAD; ++q) {
            const double t = 0.5 * (1.0 + L.gx[q]);
            double r[3];
            for (int c = 0; c < 3; ++c) r[c] = xa[c] + t * d[c] - L.xd[c];
            const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            const double ir3 = 1.0 / (r2 * sqrt(r2));
            const double A0 = (L.md[1] * r[2] - L.md[2] * r[1]) * ir3;
            const double A1 = (L.md[2] * r[0] - L.md[0] * r[2]) * ir3;
            const double A2 = (L.md[0] * r[1] - L.md[1] * r[0]) * ir3;
            sum += 0.5 * L.gw[q] * (A0 * d[0] + A1 * d[1] + A2 * d[2]);
        }
        return sum;
    }
    double A0 = 0.5 * (L.b[1] * m[2] - L.b[2] * m[1]);
    double A1 = 0.5 * (L.b[2] * m[0] - L.b[0] * m[2]);
    double A2 = 0.5 * (L.b[0] * m[1] - L.b[1] * m[0]);
    return A0 * d[0] + A1 * d[1] + A2 * d[2];
}

// CSR row of K-hat: K-hat_vv = sum alpha, K-hat_vk = -alpha exp(-i theta_vk); per
// stored entry also alpha and the phase per unit mu (0 on the diagonal), per edge
// the phase per unit mu
__global__ void k_fill_khat(Lattice L, int64_t n, int ndir, const double *ealpha, double cut, const int64_t *rp,
                            int32_t *ci, double2 *val, const int64_t *erp, int32_t *ej, int32_t *ek, double *eal,
                            double *eth, double *kal, double *kth1, double *eth1) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    Nbr nb[16];
    int c = node_neighbours(L, v, ndir, ealpha, cut, nb);
    int i, j, k;
    L.coords(v, i, j, k);
    double xv[3];
    L.pos(i, j, k, xv);
    int64_t q = rp[v], e = erp[v];
    double diag = 0;
    bool diag_done = false;
    for (int s = 0; s < c; ++s) diag += nb[s].alpha;
    for (int s = 0; s < c; ++s) {
        if (!diag_done && nb[s].col > v) {
            ci[q] = (int32_t)v;
            kal[q] = 0.0;
            kth1[q] = 0.0;
            val[q++] = make_double2(diag, 0.0);
            diag_done = true;
        }
        int a, b, cc;
        L.coords(nb[s].col, a, b, cc);
        double xk[3];
        L.pos(a, b, cc, xk);
        double th = edge_phase(L, xv, xk);
        double th1 = edge_phase1(L, xv, xk);
        double sn, cs;
        sincos(th, &sn, &cs);
        ci[q] = (int32_t)nb[s].col;
        kal[q] = nb[s].alpha;
        kth1[q] = th1;
        val[q++] = make_double2(-nb[s].alpha * cs, nb[s].alpha * sn);
        if (nb[s].col > v) {
            ej[e] = (int32_t)v;
            ek[e] = (int32_t)nb[s].col;
            eal[e] = nb[s].alpha;
            eth[e] = th;
            eth1[e] = th1;
            ++e;
        }
    }
    if (!diag_done) {
        ci[q] = (int32_t)v;
        kal[q] = 0.0;
        kth1[q] = 0.0;
        val[q] = make_double2(diag, 0.0);
    }
}

// the phase-dependent values at a new mu: K-hat_vk = -alpha exp(-i mu theta1)
// (stored entries and edge list); the diagonal sums of alpha do not change
__global__ void k_khat_set_mu(int64_t n, double mu, const int64_t *rp, const int32_t *ci, const double *kal,
                              const double *kth1, double2 *val) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int64_t q = rp[v]; q < rp[v + 1]; ++q) {
        if (ci[q] == v) continue;
        double sn, cs;
        sincos(mu * kth1[q], &sn, &cs);
        val[q] = make_double2(-kal[q] * cs, kal[q] * sn);
    }
}
__global__ void k_edges_set_mu(int64_t ne, double mu, const double *eth1, double *eth) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < ne) eth[e] = mu * eth1[e];
}

__global__ void k_volumes(Lattice L, int64_t n, double *vol) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int i, j, k;
    L.coords(v, i, j, k);
    int nb = (i == 0 || i == L.N - 1) + (j == 0 || j == L.N - 1);
    if (L.dim == 3) nb += (k == 0 || k == L.N - 1);
    double hd = (L.dim == 2) ? L.h * L.h : L.h * L.h * L.h;
    vol[v] = hd / (double)(1 << nb);
}

// red-black colour of each lattice node: (i + j + k) mod 2
__global__ void k_lattice_parity(Lattice L, int64_t n, int32_t *color, int64_t *is_red) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int i, j, k;
    L.coords(v, i, j, k);
    int c = (i + j + k) & 1;
    color[v] = c;
    is_red[v] = (c == 0);
}

// solve ordering: red nodes (ascending) first, then black nodes (ascending)
__global__ void k_rb_perm(int64_t n, const int32_t *color, const int64_t *red_rank, int64_t nred, int32_t *perm,
                          int32_t *iperm) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t p = (color[v] == 0) ? red_rank[v] : nred + (v - red_rank[v]);
    perm[p] = (int32_t)v;
    iperm[v] = (int32_t)p;
}

__global__ void k_permute_real(int64_t n, const int32_t *perm, const double *in, double *out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) out[p] = in[perm[p]];
}

// ---------------------------------------------------------------- sliced ELL builder
__global__ void k_sell_rowlen(int64_t nrows, const int32_t *perm, const int64_t *rp, const int32_t *ci, bool drop_diag,
                              int32_t *len) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrows) return;
    int64_t r = perm ? perm[p] : p;
    int64_t l = rp[r + 1] - rp[r];
    if (drop_diag)
        for (int64_t q = rp[r]; q < rp[r + 1]; ++q)
            if (ci[q] == r) --l;
    len[p] = (int32_t)l;
}

__global__ void k_sell_width(int64_t nrows, int64_t nslices, const int32_t *len, int64_t *ssize) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int l = 0; l < SELL_C; ++l) {
        int64_t p = s * SELL_C + l;
        if (p < nrows) w = max(w, len[p]);
    }
    ssize[s] = (int64_t)w * SELL_C;
}

template <typename C>
__global__ void k_sell_fill(int64_t nrows, int64_t ncols, const int32_t *perm, const int32_t *icol, const int64_t *rp,
                            const int32_t *ci, const double2 *v, const double *row_scale, bool drop_diag,
                            const int64_t *sptr, int32_t *scol, C *sval, double *diag_out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrows) return;
    int64_t r = perm ? perm[p] : p;
    int64_t s = p / SELL_C;
    int lane = (int)(p % SELL_C);
    int64_t base = sptr[s] + lane;
    int w = (int)((sptr[s + 1] - sptr[s]) / SELL_C);
    double sc = row_scale ? 1.0 / row_scale[r] : 1.0;
    int k = 0;
    double dg = 0;
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        int64_t c = ci[q];
        double2 a = v[q];
        if (drop_diag && c == r) {
            dg = a.x * sc;
            continue;
        }
        scol[base + (int64_t)k * SELL_C] = icol ? icol[c] : (int32_t)c;
        C val;
        val.x = a.x * sc;
        val.y = a.y * sc;
        sval[base + (int64_t)k * SELL_C] = val;
        ++k;
    }
    int32_t pad = (int32_t)(p < ncols ? p : ncols - 1);
    for (; k < w; ++k) {
        scol[base + (int64_t)k * SELL_C] = pad;
        C z;
        z.x = 0;
        z.y = 0;
        sval[base + (int64_t)k * SELL_C] = z;
    }
    if (diag_out) diag_out[p] = dg;
}

template <typename C>
void build_sell(int64_t nrows, int64_t ncols, const int32_t *perm, const int32_t *icol, const CsrDev &A,
                const double *row_scale, bool drop_diag, Sell<C> &out, double *diag_out, cudaStream_t s) {
    out.nrows = nrows;
    out.nslices = (nrows + SELL_C - 1) / SELL_C;
    DBuf<int32_t> len(nrows > 0 ? nrows : 1);
    out.sptr.alloc(out.nslices + 1);
    k_sell_rowlen<<<grid_for(nrows, 256), 256, 0, s>>>(nrows, perm, A.rp.get(), A.ci.get(), drop_diag, len.get());
    GL_LAUNCH_CHECK();
    k_sell_width<<<grid_for(out.nslices, 256), 256, 0, s>>>(nrows, out.nslices, len.get(), out.sptr.get());
    GL_LAUNCH_CHECK();
    scan_exclusive(out.sptr.get(), out.sptr.get(), out.nslices, true, s);
    int64_t total = 0;
    GL_CUDA(cudaMemcpyAsync(&total, out.sptr.get() + out.nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    out.nnz_stored = total;
    out.nnz_real = A.nnz - (drop_diag ? nrows : 0);
    out.col.alloc(total > 0 ? total : 1);
    out.val.alloc(total > 0 ? total : 1);
    k_sell_fill<C><<<grid_for(nrows, 256), 256, 0, s>>>(nrows, ncols, perm, icol, A.rp.get(), A.ci.get(), A.v.get(),
                                                        row_scale, drop_diag, out.sptr.get(), out.col.get(),
                                                        out.val.get(), diag_out);
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
}

template void build_sell<double2>(int64_t, int64_t, const int32_t *, const int32_t *, const CsrDev &, const double *,
                                  bool, Sell<double2> &, double *, cudaStream_t);
template void build_sell<float2>(int64_t, int64_t, const int32_t *, const int32_t *, const CsrDev &, const double *,
                                 bool, Sell<float2> &, double *, cudaStream_t);

// ---------------------------------------------------------------- grouped CSR builder
__global__ void k_csrg_len(int64_t nrows, const int32_t *perm, const int32_t *icol, const int64_t *rp,
                           const int32_t *ci, bool drop_diag, int64_t col_lo, int64_t *len) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrows) return;
    int64_t r = perm ? perm[p] : p;
    int64_t l = 0;
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        const int64_t c = ci[q];
        if (drop_diag && c == r) continue;
        if ((icol ? icol[c] : c) < col_lo) continue;
        ++l;
    }
    len[p] = l;
}

template <typename C>
__global__ void k_csrg_fill(int64_t nrows, const int32_t *perm, const int32_t *icol, const int64_t *rp,
                            const int32_t *ci, const double2 *v, bool drop_diag, int64_t col_lo, const int64_t *orp,
                            int32_t *ocol, C *oval, double *diag_out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrows) return;
    int64_t r = perm ? perm[p] : p;
    int64_t o = orp[p];
    double dg = 0;
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        int64_t c = ci[q];
        if (drop_diag && c == r) {
            dg = v[q].x;
            continue;
        }
        const int32_t oc = icol ? icol[c] : (int32_t)c;
        if (oc < col_lo) continue;
        ocol[o] = oc;
        C val;
        val.x = v[q].x;
        val.y = v[q].y;
        oval[o] = val;
        ++o;
    }
    if (diag_out) diag_out[p] = dg;
}

template <typename C>
void build_csrg(int64_t nrows, const int32_t *perm, const int32_t *icol, const CsrDev &A, bool drop_diag,
                CsrG<C> &out, double *diag_out, cudaStream_t s, int64_t col_lo) {
    out.nrows = nrows;
    DBuf<int64_t> len(nrows + 1);
    k_csrg_len<<<grid_for(nrows, 256), 256, 0, s>>>(nrows, perm, icol, A.rp.get(), A.ci.get(), drop_diag, col_lo,
                                                     len.get());
    GL_LAUNCH_CHECK();
    out.rp.alloc(nrows + 1);
    scan_exclusive(len.get(), out.rp.get(), nrows, true, s);
    GL_CUDA(cudaMemcpyAsync(&out.nnz, out.rp.get() + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    out.col.alloc(out.nnz > 0 ? out.nnz : 1);
    out.val.alloc(out.nnz > 0 ? out.nnz : 1);
    k_csrg_fill<C><<<grid_for(nrows, 256), 256, 0, s>>>(nrows, perm, icol, A.rp.get(), A.ci.get(), A.v.get(),
                                                        drop_diag, col_lo, out.rp.get(), out.col.get(),
                                                        out.val.get(), diag_out);
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
    // lanes per row: the power of two nearest a quarter of the mean row length
    double avg = nrows > 0 ? (double)out.nnz / nrows : 0;
    int G = 1;
    while (G < 32 && 2 * G * 4 <= avg * 1.5) G *= 2;
    out.G = G;
}

template void build_csrg<double2>(int64_t, const int32_t *, const int32_t *, const CsrDev &, bool, CsrG<double2> &,
                                  double *, cudaStream_t, int64_t);
template void build_csrg<float2>(int64_t, const int32_t *, const int32_t *, const CsrDev &, bool, CsrG<float2> &,
                                 double *, cudaStream_t, int64_t);

__global__ void k_d2f(int64_t n, const double *in, float *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}
void to_float(const double *in, float *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_d2f<<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
    GL_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- mesh creation
// nodes and weights of the q-point Gauss-Legendre rule on [-1, 1]: the roots of
// the Legendre polynomial P_q by Newton's method (three-term recurrence for P_q,
// P_q' from P_q and P_{q-1}), weights 2 / ((1 - x^2) P_q'(x)^2)
static void legendre_rule(int q, double *x, double *w) {
    const double pi = std::acos(-1.0);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5)), der = 0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1, pc = z;
            for (int k = 2; k <= q; ++k) {
                const double pn = ((2.0 * k - 1) * z * pc - (k - 1.0) * pm) / k;
                pm = pc;
                pc = pn;
            }
            der = q * (z * pc - pm) / (z * z - 1.0);
            const double step = pc / der;
            z -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * der * der);
    }
}

void mesh_create(gl_mesh_s *m, int dim, int N, double edge, double mu, const double *bhat, cudaStream_t s,
                 const double *dip_x0, const double *dip_m) {
    GL_REQUIRE(dim == 2 || dim == 3, GL_ERR_ARG, "dim must be 2 or 3");
    GL_REQUIRE(N >= 2, GL_ERR_ARG, "n_per_side must be >= 2");
    GL_REQUIRE(edge > 0 && std::isfinite(edge), GL_ERR_ARG, "edge length must be positive");
    double nd = (dim == 2) ? (double)N * N : (double)N * N * N;
    GL_REQUIRE(nd < 2147483647.0, GL_ERR_ARG, "too many nodes for int32 indices");
    Lattice L;
    L.dim = dim;
    L.N = N;
    L.h = edge / (N - 1);
    L.x0 = -0.5 * edge;
    L.mu = mu;
    L.dipole = (dip_x0 && dip_m) ? 1 : 0;
    for (int c = 0; c < 3; ++c) {
        L.xd[c] = L.dipole ? dip_x0[c] : 0.0;
        L.md[c] = L.dipole ? dip_m[c] : 0.0;
    }
    legendre_rule(GL_QUAD, L.gx, L.gw);
    if (L.dipole) {
        // the dipole must lie outside the closed domain
        bool inside = true;
        for (int c = 0; c < dim; ++c) inside = inside && std::fabs(dip_x0[c]) <= 0.5 * edge;
        if (dim == 2) inside = inside && dip_x0[2] == 0.0;
        GL_REQUIRE(!inside, GL_ERR_ARG, "the dipole must lie outside the domain");
    }
    m->dipole = L.dipole;
    double b[3] = {0, 0, 1};
    if (bhat) {
        double nb = std::sqrt(bhat[0] * bhat[0] + bhat[1] * bhat[1] + bhat[2] * bhat[2]);
        GL_REQUIRE(nb > 0, GL_ERR_ARG, "bhat must be nonzero");
        for (int c = 0; c < 3; ++c) b[c] = bhat[c] / nb;
    }
    for (int c = 0; c < 3; ++c) L.b[c] = m->bhat[c] = b[c];
    m->dim = dim;
    m->N = N;
    m->h = L.h;
    m->edge = edge;
    m->mu = mu;
    int64_t n = (int64_t)nd;
    m->n = n;
    int ndir = (dim == 2) ? 3 : 7;

    // per-simplex coefficients, then per-edge sums
    int64_t ncell = (dim == 2) ? (int64_t)(N - 1) * (N - 1) : (int64_t)(N - 1) * (N - 1) * (N - 1);
    int ns = (dim == 2) ? 2 : 6, ne = (dim == 2) ? 3 : 6;
    DBuf<double> ealpha(n * ndir);
    {
        DBuf<double> alphaT(ncell * ns * ne > 0 ? ncell * ns * ne : 1);
        if (ncell > 0) {
            k_simplex_alpha<<<grid_for(ncell, 128), 128, 0, s>>>(L, ncell, alphaT.get());
            GL_LAUNCH_CHECK();
        }
        k_edge_alpha<<<grid_for(n * ndir, 256), 256, 0, s>>>(L, n, ndir, alphaT.get(), ealpha.get());
        GL_LAUNCH_CHECK();
        GL_CUDA(cudaStreamSynchronize(s));
    }
    double amax = reduce_max_abs(ealpha.get(), n * ndir, s);
    double cut = 1e-12 * amax;

    // K-hat CSR in node order, plus the edge list
    DBuf<int64_t> len(n + 1), fwd(n + 1);
    k_row_len<<<grid_for(n, 128), 128, 0, s>>>(L, n, ndir, ealpha.get(), cut, len.get(), fwd.get());
    GL_LAUNCH_CHECK();
    CsrDev &K = m->khat;
    K.n = K.m = n;
    K.rp.alloc(n + 1);
    scan_exclusive(len.get(), K.rp.get(), n, true, s);
    GL_CUDA(cudaMemcpyAsync(&K.nnz, K.rp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DBuf<int64_t> erp(n + 1);
    scan_exclusive(fwd.get(), erp.get(), n, true, s);
    GL_CUDA(cudaMemcpyAsync(&m->nedges, erp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    K.ci.alloc(K.nnz);
    K.v.alloc(K.nnz);
    m->kal.alloc(K.nnz);
    m->kth1.alloc(K.nnz);
    int64_t nem = m->nedges > 0 ? m->nedges : 1;
    m->ej.alloc(nem);
    m->ek.alloc(nem);
    m->ealpha.alloc(nem);
    m->etheta.alloc(nem);
    m->etheta1.alloc(nem);
    k_fill_khat<<<grid_for(n, 128), 128, 0, s>>>(L, n, ndir, ealpha.get(), cut, K.rp.get(), K.ci.get(), K.v.get(),
                                                  erp.get(), m->ej.get(), m->ek.get(), m->ealpha.get(),
                                                  m->etheta.get(), m->kal.get(), m->kth1.get(), m->etheta1.get());
    GL_LAUNCH_CHECK();
    m->vol.alloc(n);
    k_volumes<<<grid_for(n, 256), 256, 0, s>>>(L, n, m->vol.get());
    GL_LAUNCH_CHECK();

    // red-black solve ordering
    m->color0.alloc(n);
    DBuf<int64_t> isred(n + 1);
    k_lattice_parity<<<grid_for(n, 256), 256, 0, s>>>(L, n, m->color0.get(), isred.get());
    GL_LAUNCH_CHECK();
    scan_exclusive(isred.get(), isred.get(), n, true, s);
    GL_CUDA(cudaMemcpyAsync(&m->nred, isred.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    m->perm.alloc(n);
    m->iperm.alloc(n);
    k_rb_perm<<<grid_for(n, 256), 256, 0, s>>>(n, m->color0.get(), isred.get(), m->nred, m->perm.get(),
                                               m->iperm.get());
    GL_LAUNCH_CHECK();
    m->ncolors0 = n > 1 ? 2 : 1;
    m->cstart0 = n > 1 ? std::vector<int64_t>{0, m->nred, n} : std::vector<int64_t>{0, n};

    // K = D^-1 K-hat, off-diagonals as sliced ELL in the solve ordering
    m->kdiag.alloc(n);
    build_sell<double2>(n, n, m->perm.get(), m->iperm.get(), K, m->vol.get(), true, m->K, m->kdiag.get(), s);
    m->volp.alloc(n);
    k_permute_real<<<grid_for(n, 256), 256, 0, s>>>(n, m->perm.get(), m->vol.get(), m->volp.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
    // the matrix-free lattice stencil, checked against K (even N)
    mesh_ensure_lattice(m, s);
}

// rewrites the values of a sliced ELL built by build_sell from a CSR of the same
// sparsity (same slices, widths and columns; buffers kept, so captured graphs
// that read them stay valid)
template <typename C>
static void refill_sell(int64_t nrows, int64_t ncols, const int32_t *perm, const int32_t *icol, const CsrDev &A,
                        const double *row_scale, bool drop_diag, Sell<C> &out, double *diag_out, cudaStream_t s) {
    k_sell_fill<C><<<grid_for(nrows, 256), 256, 0, s>>>(nrows, ncols, perm, icol, A.rp.get(), A.ci.get(), A.v.get(),
                                                        row_scale, drop_diag, out.sptr.get(), out.col.get(),
                                                        out.val.get(), diag_out);
    GL_LAUNCH_CHECK();
}

void mesh_set_mu(gl_mesh_s *m, double mu, cudaStream_t s) {
    GL_REQUIRE(std::isfinite(mu), GL_ERR_ARG, "mu must be finite");
    const int64_t n = m->n;
    k_khat_set_mu<<<grid_for(n, 256), 256, 0, s>>>(n, mu, m->khat.rp.get(), m->khat.ci.get(), m->kal.get(),
                                                   m->kth1.get(), m->khat.v.get());
    if (m->nedges > 0)
        k_edges_set_mu<<<grid_for(m->nedges, 256), 256, 0, s>>>(m->nedges, mu, m->etheta1.get(), m->etheta.get());
    GL_LAUNCH_CHECK();
    refill_sell<double2>(n, n, m->perm.get(), m->iperm.get(), m->khat, m->vol.get(), true, m->K, m->kdiag.get(), s);
    if (m->has32)
        refill_sell<float2>(n, n, m->perm.get(), m->iperm.get(), m->khat, m->vol.get(), true, m->K32, nullptr, s);
    mesh_refresh_lattice(m, s);
    GL_CUDA(cudaStreamSynchronize(s));
    m->mu = mu;
    m->version += 1;
}

// FP32 copies of the fine operator for the mixed-precision path (built on demand)
void mesh_ensure_fp32(gl_mesh_s *m, cudaStream_t s) {
    if (m->has32) return;
    build_sell<float2>(m->n, m->n, m->perm.get(), m->iperm.get(), m->khat, m->vol.get(), true, m->K32, nullptr, s);
    m->kdiag32.alloc(m->n);
    m->volp32.alloc(m->n);
    to_float(m->kdiag.get(), m->kdiag32.get(), m->n, s);
    to_float(m->volp.get(), m->volp32.get(), m->n, s);
    GL_CUDA(cudaStreamSynchronize(s));
    mesh_ensure_lattice(m, s);
    m->has32 = true;
}


// ---------------------------------------------------------------- general simplicial meshes
// Any conforming simplicial mesh (the paper's Delaunay meshes of its test domains,
// Sec. 4): the coefficient of every edge of every simplex (the cotangent formula
// in 2D, its dihedral form in 3D), summed
// per edge over the simplices at the edge's first node in ascending simplex order
// (Eq. fhat; a deterministic order), the edges with |alpha| <= 1e-12 max |alpha|
// dropped (O2), the link phases of the uniform field or the dipole (Eq. link
// variable), K-hat in node order (Eq. discr kin energy with Remark rmk:dk), and the
// control volumes from the same coefficients (Eq. mass lumping, read as the dual of
// the coefficients): |V_j| = sum_k alpha_jk |x_j - x_k|^2 / (2 d), the Voronoi
// region of x_j for well-centred Delaunay simplices.  The finest level has no
// lattice colouring: the nodes are coloured like a coarse level (round-based
// smallest-last) and put in colour-major order.
constexpr int GEN_MAXDEG = 64;  // neighbours of one node

__global__ void k_gen_check(int64_t q, const int32_t *simp, int64_t n, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < q && (simp[i] < 0 || simp[i] >= n)) atomicExch(bad, 1);
}
// Tetrahedron coefficients in closed form: alpha_ij = |e_kl| cot(theta_kl) / 6,
// e_kl the opposite edge, theta_kl the dihedral angle there (the unique solution
// of simplex_alpha's system, since these weights satisfy sum_e alpha_e e e^T =
// |S| I, without its 6 x 6 system, badly conditioned for flat tetrahedra);
// cot theta = (a . b) / |a x b| with a, b the parts of x_i - x_k, x_j - x_k
// perpendicular to e_kl.
__device__ void simplex_alpha_dihedral(const double p[4][3], double *alpha) {
    for (int s = 0; s < 6; ++s) {
        int i, j;
        simplex_edge(3, s, i, j);
        int k = -1, l = -1;
        for (int t = 0; t < 4; ++t)
            if (t != i && t != j) {
                if (k < 0)
                    k = t;
                else
                    l = t;
            }
        double e[3], a[3], b[3];
        for (int c = 0; c < 3; ++c) {
            e[c] = p[l][c] - p[k][c];
            a[c] = p[i][c] - p[k][c];
            b[c] = p[j][c] - p[k][c];
        }
        const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2], L = sqrt(ee);
        const double ae = (a[0] * e[0] + a[1] * e[1] + a[2] * e[2]) / ee;
        const double be = (b[0] * e[0] + b[1] * e[1] + b[2] * e[2]) / ee;
        for (int c = 0; c < 3; ++c) {
            a[c] -= ae * e[c];
            b[c] -= be * e[c];
        }
        const double x0 = a[1] * b[2] - a[2] * b[1], x1 = a[2] * b[0] - a[0] * b[2], x2 = a[0] * b[1] - a[1] * b[0];
        const double sn = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
        alpha[s] = L * (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (6.0 * sn);
    }
}
// alphaT[s * ne + e]: coefficient of local edge e of simplex s
__global__ void k_gen_alpha(int dim, int64_t ns, const double *xyz, const int32_t *simp, double *alphaT, int *bad) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    double p[4][3];
    for (int v = 0; v <= dim; ++v) {
        const int64_t id = simp[s * (dim + 1) + v];
        for (int c = 0; c < 3; ++c) p[v][c] = xyz[3 * id + c];
    }
    double al[6];
    if (dim == 2)
        simplex_alpha(2, p, al);
    else
        simplex_alpha_dihedral(p, al);
    const int ne = dim == 2 ? 3 : 6;
    for (int e = 0; e < ne; ++e) {
        if (!isfinite(al[e])) atomicExch(bad, 1);
        alphaT[s * ne + e] = al[e];
    }
}
// simplices at each node: counts, then the lists (sorted afterwards)
__global__ void k_gen_inc_count(int dim, int64_t ns, const int32_t *simp, unsigned long long *cnt) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    for (int v = 0; v <= dim; ++v) atomicAdd(cnt + simp[s * (dim + 1) + v], 1ull);
}
__global__ void k_gen_inc_fill(int dim, int64_t ns, const int32_t *simp, const int64_t *irp, unsigned long long *fill,
                               int32_t *inc) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ns) return;
    for (int v = 0; v <= dim; ++v) {
        const int32_t a = simp[s * (dim + 1) + v];
        const unsigned long long k = atomicAdd(fill + a, 1ull);
        inc[irp[a] + (int64_t)k] = (int32_t)s;
    }
}
// node a: its neighbours b > a with the coefficients summed over a's simplices in
// ascending order, sorted by b, into slots [a GEN_MAXDEG, (a + 1) GEN_MAXDEG)
__global__ void k_gen_node_edges(int dim, int64_t n, const int32_t *simp, const int64_t *irp, const int32_t *inc,
                                 const double *alphaT, int32_t *nb_out, double *al_out, int32_t *cnt_out, int *bad) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int32_t nb[GEN_MAXDEG];
    double al[GEN_MAXDEG];
    int c = 0;
    const int ne = dim == 2 ? 3 : 6;
    for (int64_t q = irp[a]; q < irp[a + 1]; ++q) {
        const int64_t s = inc[q];
        for (int e = 0; e < ne; ++e) {
            int u, w;
            simplex_edge(dim, e, u, w);
            int32_t gu = simp[s * (dim + 1) + u], gw = simp[s * (dim + 1) + w];
            if (gu > gw) {
                const int32_t t = gu;
                gu = gw;
                gw = t;
            }
            if (gu != (int32_t)a) continue;
            int k = 0;
            while (k < c && nb[k] != gw) ++k;
            if (k == c) {
                if (c == GEN_MAXDEG) {
                    atomicExch(bad, 2);
                    continue;
                }
                nb[c] = gw;
                al[c] = 0.0;
                ++c;
            }
            al[k] += alphaT[s * ne + e];
        }
    }
    for (int i = 1; i < c; ++i) {
        const int32_t kb = nb[i];
        const double ka = al[i];
        int r = i - 1;
        while (r >= 0 && nb[r] > kb) {
            nb[r + 1] = nb[r];
            al[r + 1] = al[r];
            --r;
        }
        nb[r + 1] = kb;
        al[r + 1] = ka;
    }
    for (int i = 0; i < GEN_MAXDEG; ++i) {
        nb_out[a * GEN_MAXDEG + i] = i < c ? nb[i] : -1;
        al_out[a * GEN_MAXDEG + i] = i < c ? al[i] : 0.0;
    }
    cnt_out[a] = c;
}
// kept edges of each node (forward) and of the nodes they reach (backward)
__global__ void k_gen_keep_count(int64_t n, const int32_t *nb, const double *al, const int32_t *cnt, double cut,
                                 int64_t *fwd, unsigned long long *back) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int64_t f = 0;
    for (int i = 0; i < cnt[a]; ++i)
        if (fabs(al[a * GEN_MAXDEG + i]) > cut) {
            ++f;
            atomicAdd(back + nb[a * GEN_MAXDEG + i], 1ull);
        }
    fwd[a] = f;
}
// the edge list (j < k, lexicographic) with coefficients and phases
__global__ void k_gen_edges(int64_t n, const int32_t *nb, const double *al, const int32_t *cnt, double cut,
                            const int64_t *erp, const double *xyz, Lattice L, int32_t *ej, int32_t *ek, double *eal,
                            double *eth, double *eth1) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int64_t e = erp[a];
    const double *xa = xyz + 3 * a;
    for (int i = 0; i < cnt[a]; ++i) {
        const double alpha = al[a * GEN_MAXDEG + i];
        if (!(fabs(alpha) > cut)) continue;
        const int32_t b = nb[a * GEN_MAXDEG + i];
        const double *xb = xyz + 3 * (int64_t)b;
        ej[e] = (int32_t)a;
        ek[e] = b;
        eal[e] = alpha;
        eth1[e] = edge_phase1(L, xa, xb);
        eth[e] = edge_phase(L, xa, xb);
        ++e;
    }
}
// the edges ending at each node (by edge id; sorted afterwards)
__global__ void k_gen_back_fill(int64_t ne, const int32_t *ek, const int64_t *brp, unsigned long long *fill, int32_t *bl) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int32_t b = ek[e];
    const unsigned long long k = atomicAdd(fill + b, 1ull);
    bl[brp[b] + (int64_t)k] = (int32_t)e;
}
__global__ void k_gen_row_max(int64_t n, const int64_t *rp, int *mx) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < n) atomicMax(mx, (int)(rp[a + 1] - rp[a]));
}
// the longest row of a row-pointer array (synchronises s)
static int64_t longest_row(int64_t n, const int64_t *rp, cudaStream_t s) {
    DBuf<int> mx(1);
    GL_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
    k_gen_row_max<<<grid_for(n, 256), 256, 0, s>>>(n, rp, mx.get());
    GL_LAUNCH_CHECK();
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, mx.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return h;
}
__global__ void k_gen_row_len(int64_t n, const int64_t *erp, const int64_t *brp, int64_t *len) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < n) len[a] = (erp[a + 1] - erp[a]) + (brp[a + 1] - brp[a]) + 1;
}
// row a of K-hat: the edges ending at a (neighbours below a), the diagonal, the
// edges starting at a (neighbours above a): columns ascending
__global__ void k_gen_khat(int64_t n, const int64_t *krp, const int64_t *brp, const int32_t *bl, const int64_t *erp,
                           const int32_t *ej, const int32_t *ek, const double *eal, const double *eth,
                           const double *eth1, int32_t *ci, double2 *v, double *kal, double *kth1) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    double diag = 0;
    for (int64_t q = brp[a]; q < brp[a + 1]; ++q) diag += eal[bl[q]];
    for (int64_t e = erp[a]; e < erp[a + 1]; ++e) diag += eal[e];
    int64_t q = krp[a];
    for (int64_t r = brp[a]; r < brp[a + 1]; ++r) {
        const int32_t e = bl[r];
        // K-hat_{a c} = -alpha exp(-i theta_{a c}), theta_{a c} = -theta_{c a}
        double sn, cs;
        sincos(eth[e], &sn, &cs);
        ci[q] = ej[e];
        kal[q] = eal[e];
        kth1[q] = -eth1[e];
        v[q++] = make_double2(-eal[e] * cs, -eal[e] * sn);
    }
    ci[q] = (int32_t)a;
    kal[q] = 0.0;
    kth1[q] = 0.0;
    v[q++] = make_double2(diag, 0.0);
    for (int64_t e = erp[a]; e < erp[a + 1]; ++e) {
        double sn, cs;
        sincos(eth[e], &sn, &cs);
        ci[q] = ek[e];
        kal[q] = eal[e];
        kth1[q] = eth1[e];
        v[q++] = make_double2(-eal[e] * cs, eal[e] * sn);
    }
}
__global__ void k_gen_volumes(int64_t n, int dim, const int64_t *krp, const int32_t *ci, const double *kal,
                              const double *xyz, double *vol) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    double s = 0;
    for (int64_t q = krp[a]; q < krp[a + 1]; ++q) {
        const int64_t c = ci[q];
        if (c == a) continue;
        const double d0 = xyz[3 * c] - xyz[3 * a], d1 = xyz[3 * c + 1] - xyz[3 * a + 1],
                     d2 = xyz[3 * c + 2] - xyz[3 * a + 2];
        s += kal[q] * (d0 * d0 + d1 * d1 + d2 * d2) / (2.0 * dim);
    }
    vol[a] = s;
}
// colour-major order: the nodes of colour c at [base, base + count), in node order
__global__ void k_gen_flag_colour(int64_t n, const int32_t *color, int c, int64_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = color[i] == c ? 1 : 0;
}
__global__ void k_gen_place(int64_t n, const int32_t *color, int c, const int64_t *rank, int64_t base, int32_t *perm,
                            int32_t *iperm) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || color[i] != c) return;
    const int64_t p = base + rank[i];
    perm[p] = (int32_t)i;
    iperm[i] = (int32_t)p;
}

void mesh_create_simplicial(gl_mesh_s *m, int dim, int64_t n, const double *xyz_host, int64_t ns,
                            const int32_t *simp_host, double mu, const double *bhat, const double *dip_x0,
                            const double *dip_m, cudaStream_t s) {
    GL_REQUIRE(dim == 2 || dim == 3, GL_ERR_ARG, "dim must be 2 or 3");
    GL_REQUIRE(n >= 2 && n < 2147483647, GL_ERR_ARG, "node count out of range");
    GL_REQUIRE(ns >= 1 && ns * (dim + 1) < 2147483647, GL_ERR_ARG, "simplex count out of range");
    GL_REQUIRE(xyz_host && simp_host, GL_ERR_ARG, "NULL mesh arrays");
    GL_REQUIRE(std::isfinite(mu), GL_ERR_ARG, "mu must be finite");
    Lattice L{};
    L.dim = dim;
    L.N = 0;
    L.h = 0;
    L.mu = mu;
    L.dipole = (dip_x0 && dip_m) ? 1 : 0;
    for (int c = 0; c < 3; ++c) {
        L.xd[c] = L.dipole ? dip_x0[c] : 0.0;
        L.md[c] = L.dipole ? dip_m[c] : 0.0;
    }
    legendre_rule(GL_QUAD, L.gx, L.gw);
    double b[3] = {0, 0, 1};
    if (bhat) {
        double nb = std::sqrt(bhat[0] * bhat[0] + bhat[1] * bhat[1] + bhat[2] * bhat[2]);
        GL_REQUIRE(nb > 0, GL_ERR_ARG, "bhat must be nonzero");
        for (int c = 0; c < 3; ++c) b[c] = bhat[c] / nb;
    }
    for (int c = 0; c < 3; ++c) L.b[c] = m->bhat[c] = b[c];
    m->dim = dim;
    m->N = 0;
    m->h = 0;
    m->edge = 0;
    m->mu = mu;
    m->dipole = L.dipole;
    m->n = n;
    const int ne = dim == 2 ? 3 : 6;
    DBuf<double> xyz(3 * n);
    DBuf<int32_t> simp(ns * (dim + 1));
    GL_CUDA(cudaMemcpyAsync(xyz.get(), xyz_host, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    GL_CUDA(cudaMemcpyAsync(simp.get(), simp_host, ns * (dim + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DBuf<int> bad(1);
    GL_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_gen_check<<<grid_for(ns * (dim + 1), 256), 256, 0, s>>>(ns * (dim + 1), simp.get(), n, bad.get());
    GL_LAUNCH_CHECK();
    int hb = 0;
    GL_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(hb == 0, GL_ERR_ARG, "simplex node id out of range");
    if (dim == 2) {
        // z = 0 in 2D
        std::vector<double> xh(xyz_host, xyz_host + 3 * n);
        for (int64_t j = 0; j < n; ++j) xh[3 * j + 2] = 0.0;
        GL_CUDA(cudaMemcpyAsync(xyz.get(), xh.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        GL_CUDA(cudaStreamSynchronize(s));
    }
    // coefficients per simplex edge, then per edge summed at its first node
    DBuf<double> alphaT(ns * ne);
    k_gen_alpha<<<grid_for(ns, 128), 128, 0, s>>>(dim, ns, xyz.get(), simp.get(), alphaT.get(), bad.get());
    GL_LAUNCH_CHECK();
    DBuf<int64_t> irp(n + 1);
    {
        DBuf<unsigned long long> cnt(n);
        GL_CUDA(cudaMemsetAsync(cnt.get(), 0, n * sizeof(unsigned long long), s));
        k_gen_inc_count<<<grid_for(ns, 256), 256, 0, s>>>(dim, ns, simp.get(), cnt.get());
        GL_LAUNCH_CHECK();
        scan_exclusive(reinterpret_cast<const int64_t *>(cnt.get()), irp.get(), n, true, s);
    }
    const int64_t ninc = ns * (dim + 1);
    DBuf<int32_t> inc(ninc);
    {
        DBuf<unsigned long long> fill(n);
        GL_CUDA(cudaMemsetAsync(fill.get(), 0, n * sizeof(unsigned long long), s));
        k_gen_inc_fill<<<grid_for(ns, 256), 256, 0, s>>>(dim, ns, simp.get(), irp.get(), fill.get(), inc.get());
        GL_LAUNCH_CHECK();
        DBuf<double2> dummy(ninc);
        sort_rows_by_col(n, irp.get(), inc.get(), dummy.get(), longest_row(n, irp.get(), s), s);
    }
    DBuf<int32_t> nbs(n * GEN_MAXDEG), cnts(n);
    DBuf<double> als(n * GEN_MAXDEG);
    k_gen_node_edges<<<grid_for(n, 128), 128, 0, s>>>(dim, n, simp.get(), irp.get(), inc.get(), alphaT.get(),
                                                       nbs.get(), als.get(), cnts.get(), bad.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaMemcpyAsync(&hb, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(hb != 1, GL_ERR_ARG, "a degenerate simplex (its coefficients are not finite)");
    GL_REQUIRE(hb != 2, GL_ERR_CAPACITY, "a node has more than 64 neighbours");
    const double amax = reduce_max_abs(als.get(), n * GEN_MAXDEG, s);
    const double cut = 1e-12 * amax;
    DBuf<int64_t> fwd(n + 1), erp(n + 1), brp(n + 1);
    DBuf<unsigned long long> back(n);
    GL_CUDA(cudaMemsetAsync(back.get(), 0, n * sizeof(unsigned long long), s));
    k_gen_keep_count<<<grid_for(n, 256), 256, 0, s>>>(n, nbs.get(), als.get(), cnts.get(), cut, fwd.get(), back.get());
    GL_LAUNCH_CHECK();
    scan_exclusive(fwd.get(), erp.get(), n, true, s);
    scan_exclusive(reinterpret_cast<const int64_t *>(back.get()), brp.get(), n, true, s);
    GL_CUDA(cudaMemcpyAsync(&m->nedges, erp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    const int64_t nem = m->nedges > 0 ? m->nedges : 1;
    m->ej.alloc(nem);
    m->ek.alloc(nem);
    m->ealpha.alloc(nem);
    m->etheta.alloc(nem);
    m->etheta1.alloc(nem);
    k_gen_edges<<<grid_for(n, 128), 128, 0, s>>>(n, nbs.get(), als.get(), cnts.get(), cut, erp.get(), xyz.get(), L,
                                                  m->ej.get(), m->ek.get(), m->ealpha.get(), m->etheta.get(),
                                                  m->etheta1.get());
    GL_LAUNCH_CHECK();
    DBuf<int32_t> bl(nem);
    {
        DBuf<unsigned long long> fill(n);
        GL_CUDA(cudaMemsetAsync(fill.get(), 0, n * sizeof(unsigned long long), s));
        k_gen_back_fill<<<grid_for(nem, 256), 256, 0, s>>>(m->nedges, m->ek.get(), brp.get(), fill.get(), bl.get());
        GL_LAUNCH_CHECK();
        DBuf<double2> dummy(nem);
        sort_rows_by_col(n, brp.get(), bl.get(), dummy.get(), longest_row(n, brp.get(), s), s);
    }
    // K-hat: row a holds its backward and forward edges and the diagonal
    CsrDev &K = m->khat;
    K.n = K.m = n;
    K.rp.alloc(n + 1);
    {
        DBuf<int64_t> len(n + 1);
        k_gen_row_len<<<grid_for(n, 256), 256, 0, s>>>(n, erp.get(), brp.get(), len.get());
        GL_LAUNCH_CHECK();
        scan_exclusive(len.get(), K.rp.get(), n, true, s);
    }
    GL_CUDA(cudaMemcpyAsync(&K.nnz, K.rp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    K.ci.alloc(K.nnz);
    K.v.alloc(K.nnz);
    m->kal.alloc(K.nnz);
    m->kth1.alloc(K.nnz);
    k_gen_khat<<<grid_for(n, 128), 128, 0, s>>>(n, K.rp.get(), brp.get(), bl.get(), erp.get(), m->ej.get(),
                                                 m->ek.get(), m->ealpha.get(), m->etheta.get(), m->etheta1.get(),
                                                 K.ci.get(), K.v.get(), m->kal.get(), m->kth1.get());
    GL_LAUNCH_CHECK();
    m->vol.alloc(n);
    k_gen_volumes<<<grid_for(n, 256), 256, 0, s>>>(n, dim, K.rp.get(), K.ci.get(), m->kal.get(), xyz.get(),
                                                    m->vol.get());
    GL_LAUNCH_CHECK();
    // finest-level colours and the colour-major solve ordering
    m->color0.alloc(n);
    const int nc = colour_graph_psl(K, m->color0.get(), s);
    m->perm.alloc(n);
    m->iperm.alloc(n);
    m->cstart0.assign(1, 0);
    {
        DBuf<int64_t> flag(n + 1), rank(n + 1);
        int64_t base = 0;
        for (int c = 0; c < nc; ++c) {
            k_gen_flag_colour<<<grid_for(n, 256), 256, 0, s>>>(n, m->color0.get(), c, flag.get());
            GL_LAUNCH_CHECK();
            scan_exclusive(flag.get(), rank.get(), n, true, s);
            int64_t cnt = 0;
            GL_CUDA(cudaMemcpyAsync(&cnt, rank.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GL_CUDA(cudaStreamSynchronize(s));
            k_gen_place<<<grid_for(n, 256), 256, 0, s>>>(n, m->color0.get(), c, rank.get(), base, m->perm.get(),
                                                          m->iperm.get());
            GL_LAUNCH_CHECK();
            base += cnt;
            m->cstart0.push_back(base);
        }
    }
    m->ncolors0 = nc;
    m->nred = m->cstart0.size() > 1 ? m->cstart0[1] : n;
    // K = D^-1 K-hat, off-diagonals as sliced ELL in the solve ordering
    m->kdiag.alloc(n);
    build_sell<double2>(n, n, m->perm.get(), m->iperm.get(), K, m->vol.get(), true, m->K, m->kdiag.get(), s);
    m->volp.alloc(n);
    k_permute_real<<<grid_for(n, 256), 256, 0, s>>>(n, m->perm.get(), m->vol.get(), m->volp.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
    m->lat_checked = true;  // no lattice stencil
    m->lat_ok = false;
}
}  // namespace gl
