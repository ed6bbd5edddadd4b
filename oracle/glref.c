/*
 * glref.c -- the CPU oracle for the Jacobian solve of the extreme type-II
 * Ginzburg-Landau problem (Schloemer & Vanroose, arXiv:1204.5125).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow FP64 restatement of
 * the paper's method, written to be checked against the paper by eye.  It runs
 * on one host thread unless glref_set_threads asks for more; then only loops
 * whose iterations write disjoint rows are shared out (OpenMP), while every sum
 * across rows stays serial in index order, so the results are bit-identical for
 * any thread count.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or helper with the
 * CUDA library, and the CUDA library never calls it.
 *
 * Complex numbers are C99 `double complex`; an array of them has the same
 * interleaved (re, im) layout as numpy's complex128.
 *
 * Contents, in the paper's order:
 *   1. structured square/cube node sets and their Delaunay simplices (Sec. 3)
 *   2. per-simplex edge coefficients: cotangent formula for triangles (Remark
 *      after Cor. "simplex") and M alpha = b for tetrahedra (Cor. "simplex")
 *   3. edge coefficients summed over simplices (Eq. fhat), control volumes
 *      |V_j| (Eq. mass lumping), link phases (Eq. link variable)
 *   4. K-hat (Eq. discr kin energy, Remark rmk:dk), GL residual (Eq. discr
 *      ginla), Jacobian (Sec. 3, discrete J), energy (Eq. discr energy)
 *   5. smoothed-aggregation AMG for P-hat = K-hat + 2 D |psi|^2 (Eq. prec2,
 *      Sec. 4.1) with symmetric Gauss-Seidel smoothing (Sec. 4)
 *   6. preconditioned MINRES in Re<.,.>_D (Sec. 4, Eq. disc inner2)
 *   7. a dense direct solve of the realified system (Remark rmk:isometry)
 *
 * Parity status: every function here is pinned by a test in tests/ against a
 * closed form, an invariant from the paper, brute force, or a dense solve.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#ifdef _OPENMP
#include <omp.h>
#endif

/* host threads for the row loops (1 unless glref_set_threads says otherwise) */
static int glref_threads = 1;
void glref_set_threads(int n) { glref_threads = n > 0 ? n : 1; }
int glref_get_threads(void) { return glref_threads; }
int glref_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
/* a loop over rows whose iterations each write only their own row */
#define ROWS_PARALLEL _Pragma("omp parallel for schedule(static) num_threads(glref_threads)")

#define GLREF_MAXDEG 16
#define GLREF_MAXLEV 16

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz);
    if (!p) {
        fprintf(stderr, "glref: out of memory (%zu x %zu)\n", n, sz);
        abort();
    }
    return p;
}

typedef struct {
    int64_t n, m;   /* rows, columns */
    int64_t *rp;    /* n + 1 */
    int32_t *ci;    /* nnz, sorted ascending within each row */
    cplx *v;        /* nnz */
} csr;

static int64_t csr_nnz(const csr *a) { return a->rp[a->n]; }

static void csr_free(csr *a) {
    free(a->rp);
    free(a->ci);
    free(a->v);
    memset(a, 0, sizeof *a);
}

/* y = A x */
static void csr_matvec(const csr *a, const cplx *x, cplx *y) {
    ROWS_PARALLEL
    for (int64_t i = 0; i < a->n; ++i) {
        cplx s = 0;
        for (int64_t p = a->rp[i]; p < a->rp[i + 1]; ++p) s += a->v[p] * x[a->ci[p]];
        y[i] = s;
    }
}

static cplx csr_get(const csr *a, int64_t i, int64_t j) {
    for (int64_t p = a->rp[i]; p < a->rp[i + 1]; ++p)
        if (a->ci[p] == j) return a->v[p];
    return 0;
}

/* conjugate transpose, columns sorted (counting sort by column keeps rows ascending) */
static void csr_adjoint(const csr *a, csr *t) {
    int64_t nnz = csr_nnz(a);
    t->n = a->m;
    t->m = a->n;
    t->rp = xcalloc((size_t)t->n + 1, sizeof(int64_t));
    t->ci = xcalloc((size_t)nnz, sizeof(int32_t));
    t->v = xcalloc((size_t)nnz, sizeof(cplx));
    for (int64_t p = 0; p < nnz; ++p) t->rp[a->ci[p] + 1]++;
    for (int64_t i = 0; i < t->n; ++i) t->rp[i + 1] += t->rp[i];
    int64_t *fill = xcalloc((size_t)t->n, sizeof(int64_t));
    for (int64_t i = 0; i < a->n; ++i)
        for (int64_t p = a->rp[i]; p < a->rp[i + 1]; ++p) {
            int64_t j = a->ci[p];
            int64_t q = t->rp[j] + fill[j]++;
            t->ci[q] = (int32_t)i;
            t->v[q] = conj(a->v[p]);
        }
    free(fill);
}

/* C = A B by Gustavson's row-by-row method; the pattern of C is the full
 * structural union of products (no value-based dropping). */
static void csr_matmul(const csr *a, const csr *b, csr *c) {
    int64_t n = a->n, m = b->m;
    int64_t *mark = xcalloc((size_t)m, sizeof(int64_t));
    cplx *acc = xcalloc((size_t)m, sizeof(cplx));
    int32_t *cols = xcalloc((size_t)m, sizeof(int32_t));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
    /* symbolic pass */
    c->n = n;
    c->m = m;
    c->rp = xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        for (int64_t p = a->rp[i]; p < a->rp[i + 1]; ++p) {
            int64_t k = a->ci[p];
            for (int64_t q = b->rp[k]; q < b->rp[k + 1]; ++q) {
                int64_t j = b->ci[q];
                if (mark[j] != i) {
                    mark[j] = i;
                    cnt++;
                }
            }
        }
        c->rp[i + 1] = c->rp[i] + cnt;
    }
    c->ci = xcalloc((size_t)c->rp[n], sizeof(int32_t));
    c->v = xcalloc((size_t)c->rp[n], sizeof(cplx));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
    /* numeric pass */
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        for (int64_t p = a->rp[i]; p < a->rp[i + 1]; ++p) {
            int64_t k = a->ci[p];
            for (int64_t q = b->rp[k]; q < b->rp[k + 1]; ++q) {
                int64_t j = b->ci[q];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0;
                    cols[cnt++] = (int32_t)j;
                }
                acc[j] += a->v[p] * b->v[q];
            }
        }
        /* insertion sort of the (short) column list */
        for (int64_t s = 1; s < cnt; ++s) {
            int32_t key = cols[s];
            int64_t t = s - 1;
            while (t >= 0 && cols[t] > key) {
                cols[t + 1] = cols[t];
                --t;
            }
            cols[t + 1] = key;
        }
        for (int64_t s = 0; s < cnt; ++s) {
            c->ci[c->rp[i] + s] = cols[s];
            c->v[c->rp[i] + s] = acc[cols[s]];
        }
    }
    free(mark);
    free(acc);
    free(cols);
}

/* ------------------------------------------------------------------ */
/* 1-2. simplices and per-simplex edge coefficients                    */
/* ------------------------------------------------------------------ */

/* Edge order inside a simplex with vertices 0..d: (0,1),(0,2),...,(0,d),(1,2),... */
static int simplex_edges(int dim, int ea[6], int eb[6]) {
    int ne = 0;
    for (int a = 0; a <= dim; ++a)
        for (int b = a + 1; b <= dim; ++b) {
            ea[ne] = a;
            eb[ne] = b;
            ++ne;
        }
    return ne;
}

static double dot3(const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

/* |S| of a simplex given its vertices (3 doubles each, z = 0 in 2D) */
static double simplex_volume(int dim, const double *p) {
    double e[3][3];
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < 3; ++c) e[r][c] = p[3 * (r + 1) + c] - p[c];
    if (dim == 2) return 0.5 * fabs(e[0][0] * e[1][1] - e[0][1] * e[1][0]);
    double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                 e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                 e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    return fabs(det) / 6.0;
}

/* Solve the SPD system M x = b (n <= 6) by Cholesky; returns 0 on success. */
static int spd_solve(int n, double M[6][6], const double *b, double *x) {
    double L[6][6] = {{0}};
    for (int j = 0; j < n; ++j) {
        double s = M[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0)) return -1;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = M[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    double y[6];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return 0;
}

/* Edge coefficients of one simplex by the linear system M alpha = b with
 * M_ij = <e_i, e_j>^2 and b_i = |S| ||e_i||^2 (Cor. "simplex" and the paragraph
 * after it).  Works for triangles (3 x 3) and tetrahedra (6 x 6). */
int glref_simplex_alpha_linsys(int dim, const double *p, double *alpha) {
    int ea[6], eb[6];
    int ne = simplex_edges(dim, ea, eb);
    double e[6][3];
    for (int i = 0; i < ne; ++i)
        for (int c = 0; c < 3; ++c) e[i][c] = p[3 * eb[i] + c] - p[3 * ea[i] + c];
    double vol = simplex_volume(dim, p);
    double M[6][6], b[6];
    for (int i = 0; i < ne; ++i) {
        for (int j = 0; j < ne; ++j) {
            double d = dot3(e[i], e[j]);
            M[i][j] = d * d;
        }
        b[i] = vol * dot3(e[i], e[i]);
    }
    return spd_solve(ne, M, b, alpha);
}

/* Triangle edge coefficients from the cotangent formula of the Remark after
 * Cor. "simplex": alpha_ij = 1/2 t / sqrt(1 - t^2), t = cosine of the angle at
 * the vertex opposite edge (i, j). */
/* Tetrahedron: the closed form of the same coefficients, alpha_ij = |e_kl|
 * cot(theta_kl) / 6, with e_kl the edge opposite ij and theta_kl the dihedral
 * angle there (between the faces kli and klj): these weights satisfy
 * sum_e alpha_e e e^T = |S| I, the corollary's identity, so they are its
 * system's unique solution, without forming the (for flat tetrahedra badly
 * conditioned) 6 x 6 system.  cot theta = (a . b) / |a x b| with a, b the parts of
 * x_i - x_k and x_j - x_k perpendicular to e_kl. */
int glref_simplex_alpha_dihedral(const double *p, double *alpha) {
    int ea[6], eb[6];
    simplex_edges(3, ea, eb);
    for (int s = 0; s < 6; ++s) {
        int i = ea[s], j = eb[s], k = -1, l = -1;
        for (int t = 0; t < 4; ++t)
            if (t != i && t != j) {
                if (k < 0)
                    k = t;
                else
                    l = t;
            }
        double e[3], a[3], b[3];
        for (int c = 0; c < 3; ++c) {
            e[c] = p[3 * l + c] - p[3 * k + c];
            a[c] = p[3 * i + c] - p[3 * k + c];
            b[c] = p[3 * j + c] - p[3 * k + c];
        }
        const double ee = dot3(e, e), L = sqrt(ee);
        if (!(ee > 0)) return -1;
        const double ae = dot3(a, e) / ee, be = dot3(b, e) / ee;
        for (int c = 0; c < 3; ++c) {
            a[c] -= ae * e[c];
            b[c] -= be * e[c];
        }
        double x[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        const double sn = sqrt(dot3(x, x));
        if (!(sn > 0)) return -1;
        alpha[s] = L * dot3(a, b) / (6.0 * sn);
    }
    return 0;
}

int glref_simplex_alpha_cot(const double *p, double *alpha) {
    int ea[6], eb[6];
    simplex_edges(2, ea, eb);
    for (int s = 0; s < 3; ++s) {
        int i = ea[s], j = eb[s], k = 3 - i - j;
        double u[3], v[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = p[3 * i + c] - p[3 * k + c];
            v[c] = p[3 * j + c] - p[3 * k + c];
        }
        double t = dot3(u, v) / sqrt(dot3(u, u) * dot3(v, v));
        if (!(t * t < 1.0)) return -1;
        alpha[s] = 0.5 * t / sqrt(1.0 - t * t);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 3. the mesh: nodes, edges, alpha, |V|, link phases, K-hat            */
/* ------------------------------------------------------------------ */

typedef struct glref_mesh {
    int dim, N;                 /* N = 0: a general simplicial mesh (glref_mesh_create_simplicial) */
    int64_t n;
    double h, mu, bhat[3], a0[3], edge;
    int dipole;                 /* 0: A = (mu/2) bhat x x + a0; 1: A = mu A_d (dipole at xd, moment md) */
    double xd[3], md[3];
    double *x;     /* n x 3 node coordinates (z = 0 in 2D) */
    double *vol;   /* |V_j| */
    int64_t ne;    /* kept edges, (j < k) lexicographic */
    int32_t *ej, *ek;
    double *alpha, *theta; /* theta = integral of A along the edge from x_j to x_k */
    csr K;         /* K-hat */
} glref_mesh;

static int64_t node_id(const glref_mesh *m, int i, int j, int k) {
    return (int64_t)i + (int64_t)m->N * ((int64_t)j + (int64_t)m->N * k);
}

/* The vector potential A(x) = (mu/2) bhat x x + a0 (Eq. mvp0 scaled by mu and
 * rotated to the field direction bhat; a0 is a constant gauge offset). */
static void vector_potential(const glref_mesh *m, const double *x, double *A) {
    const double *b = m->bhat;
    A[0] = 0.5 * m->mu * (b[1] * x[2] - b[2] * x[1]) + m->a0[0];
    A[1] = 0.5 * m->mu * (b[2] * x[0] - b[0] * x[2]) + m->a0[1];
    A[2] = 0.5 * m->mu * (b[0] * x[1] - b[1] * x[0]) + m->a0[2];
}

/* Gauss-Legendre rule of GLREF_GL_POINTS points on [-1, 1]: the nodes are the
 * roots of the Legendre polynomial P_Q, found by Newton's method from the
 * Chebyshev-like start cos(pi (i + 3/4) / (Q + 1/2)), and the weights are
 * 2 / ((1 - x^2) P_Q'(x)^2). */
#define GLREF_GL_POINTS 8
static void gauss_legendre(int q, double *x, double *w) {
    for (int i = 0; i < q; ++i) {
        double z = cos(acos(-1.0) * (i + 0.75) / (q + 0.5)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;  /* P_0, P_1, then the three-term recurrence up to P_q */
            for (int k = 2; k <= q; ++k) {
                double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* the dipole potential A_d(x) = m x (x - x0) / |x - x0|^3 (Sec. 4), per unit mu */
static void dipole_potential(const glref_mesh *m, const double *x, double *A) {
    double r[3] = {x[0] - m->xd[0], x[1] - m->xd[1], x[2] - m->xd[2]};
    double r2 = dot3(r, r), ir3 = 1.0 / (r2 * sqrt(r2));
    A[0] = (m->md[1] * r[2] - m->md[2] * r[1]) * ir3;
    A[1] = (m->md[2] * r[0] - m->md[0] * r[2]) * ir3;
    A[2] = (m->md[0] * r[1] - m->md[1] * r[0]) * ir3;
}

/* integral of A . dl along the straight edge from xa to xb per unit mu of the
 * mu-dependent part (the link phase is mu times this plus the a0 part) */
static double edge_integral1(const glref_mesh *m, const double *xa, const double *xb) {
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = xb[c] - xa[c];
    if (!m->dipole) {
        /* affine A: the midpoint rule is exact (the quadrature remark after Eq. link variable) */
        double mid[3], A[3];
        const double *b = m->bhat;
        for (int c = 0; c < 3; ++c) mid[c] = 0.5 * (xa[c] + xb[c]);
        A[0] = 0.5 * (b[1] * mid[2] - b[2] * mid[1]);
        A[1] = 0.5 * (b[2] * mid[0] - b[0] * mid[2]);
        A[2] = 0.5 * (b[0] * mid[1] - b[1] * mid[0]);
        return dot3(A, d);
    }
    /* A_d is not polynomial: Gauss-Legendre along the edge (the quadrature
     * remark after Eq. link variable) */
    double gx[GLREF_GL_POINTS], gw[GLREF_GL_POINTS], s = 0;
    gauss_legendre(GLREF_GL_POINTS, gx, gw);
    for (int i = 0; i < GLREF_GL_POINTS; ++i) {
        double t = 0.5 * (1.0 + gx[i]), x[3], A[3];
        for (int c = 0; c < 3; ++c) x[c] = xa[c] + t * d[c];
        dipole_potential(m, x, A);
        s += 0.5 * gw[i] * dot3(A, d);
    }
    return s;
}

/* integral of A . dl along the straight edge from xa to xb */
static double edge_integral(const glref_mesh *m, const double *xa, const double *xb) {
    if (m->dipole) return m->mu * edge_integral1(m, xa, xb);
    double mid[3], d[3], A[3];
    for (int c = 0; c < 3; ++c) {
        mid[c] = 0.5 * (xa[c] + xb[c]);
        d[c] = xb[c] - xa[c];
    }
    vector_potential(m, mid, A);
    return dot3(A, d);
}

/* exposed for the tests: the per-unit-mu edge integral on this mesh's potential */
double glref_edge_integral1(const glref_mesh *m, const double *xa, const double *xb) {
    return edge_integral1(m, xa, xb);
}

/* per-node neighbour table used while summing simplex contributions */
typedef struct {
    int64_t n;
    int cap;        /* neighbours per node */
    int32_t *cnt;
    int32_t *nb;    /* n x cap */
    double *al;     /* n x cap */
} edge_table;

static void table_add(edge_table *t, int64_t a, int64_t b, double alpha) {
    if (a > b) {
        int64_t s = a;
        a = b;
        b = s;
    }
    int32_t *nb = t->nb + a * t->cap;
    double *al = t->al + a * t->cap;
    for (int s = 0; s < t->cnt[a]; ++s)
        if (nb[s] == b) {
            al[s] += alpha;
            return;
        }
    if (t->cnt[a] >= t->cap) {
        fprintf(stderr, "glref: node degree above %d\n", t->cap);
        abort();
    }
    nb[t->cnt[a]] = (int32_t)b;
    al[t->cnt[a]] = alpha;
    t->cnt[a]++;
}

/* Vertices of the simplices of one lattice cell with lower corner (i,j,k).
 * 2D: the cell is split by its diagonal (i,j)-(i+1,j+1).
 * 3D: the Kuhn (Freudenthal) split into 6 tetrahedra along the main diagonal.
 * Returns the number of simplices; vid[s][v] holds node ids. */
static int cell_simplices(const glref_mesh *m, int i, int j, int k, int64_t vid[6][4]) {
    if (m->dim == 2) {
        vid[0][0] = node_id(m, i, j, 0);
        vid[0][1] = node_id(m, i + 1, j, 0);
        vid[0][2] = node_id(m, i + 1, j + 1, 0);
        vid[1][0] = node_id(m, i, j, 0);
        vid[1][1] = node_id(m, i + 1, j + 1, 0);
        vid[1][2] = node_id(m, i, j + 1, 0);
        return 2;
    }
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int s = 0; s < 6; ++s) {
        int c[3] = {i, j, k};
        vid[s][0] = node_id(m, c[0], c[1], c[2]);
        for (int step = 0; step < 3; ++step) {
            c[perm[s][step]]++;
            vid[s][step + 1] = node_id(m, c[0], c[1], c[2]);
        }
    }
    return 6;
}

/* The square/cube of side `edge` centred at the origin (the paper's domains have
 * edge lengths of order 10; the unit domain is glref_mesh_create). */
static glref_mesh *mesh_assemble(glref_mesh *m);

glref_mesh *glref_mesh_create_edge(int dim, int N, double edge, double mu, const double *bhat, const double *a0) {
    if ((dim != 2 && dim != 3) || N < 2 || !(edge > 0)) return NULL;
    glref_mesh *m = xcalloc(1, sizeof *m);
    m->dim = dim;
    m->N = N;
    m->edge = edge;
    m->mu = mu;
    for (int c = 0; c < 3; ++c) {
        m->bhat[c] = bhat ? bhat[c] : (c == 2 ? 1.0 : 0.0);
        m->a0[c] = a0 ? a0[c] : 0.0;
    }
    return mesh_assemble(m);
}

/* The same domain in mu A_d, the field of a magnetic dipole of moment md at xd
 * (Sec. 4: xd = (0,0,1) for the 2D domains, (0,0,6) for the 3D ones, md = e_z). */
glref_mesh *glref_mesh_create_dipole(int dim, int N, double edge, double mu, const double *xd, const double *md) {
    if ((dim != 2 && dim != 3) || N < 2 || !(edge > 0) || !xd || !md) return NULL;
    glref_mesh *m = xcalloc(1, sizeof *m);
    m->dim = dim;
    m->N = N;
    m->edge = edge;
    m->mu = mu;
    m->dipole = 1;
    for (int c = 0; c < 3; ++c) {
        m->bhat[c] = c == 2 ? 1.0 : 0.0;
        m->xd[c] = xd[c];
        m->md[c] = md[c];
    }
    return mesh_assemble(m);
}

/* From the per-node table of summed edge coefficients: the kept edges (those
 * with |alpha| > 1e-12 max |alpha|; O2), their link phases (Eq. link variable)
 * and K-hat (Eq. discr kin energy with Remark rmk:dk).  Frees the table. */
static void mesh_edges_khat(glref_mesh *m, edge_table *tp) {
    edge_table t = *tp;
    const int64_t n = m->n;
    /* edges whose coefficient vanishes (|alpha| <= 1e-12 max |alpha|) are dropped */
    double amax = 0;
    for (int64_t a = 0; a < n; ++a)
        for (int s = 0; s < t.cnt[a]; ++s) amax = fmax(amax, fabs(t.al[a * t.cap + s]));
    double cut = 1e-12 * amax;
    int64_t ne = 0;
    for (int64_t a = 0; a < n; ++a)
        for (int s = 0; s < t.cnt[a]; ++s)
            if (fabs(t.al[a * t.cap + s]) > cut) ++ne;
    m->ne = ne;
    m->ej = xcalloc((size_t)ne, sizeof(int32_t));
    m->ek = xcalloc((size_t)ne, sizeof(int32_t));
    m->alpha = xcalloc((size_t)ne, sizeof(double));
    m->theta = xcalloc((size_t)ne, sizeof(double));
    int64_t q = 0;
    for (int64_t a = 0; a < n; ++a) {
        /* neighbours of a in ascending order */
        int32_t *nb = t.nb + a * t.cap;
        double *al = t.al + a * t.cap;
        int c = t.cnt[a];
        for (int s = 1; s < c; ++s) {
            int32_t kb = nb[s];
            double ka = al[s];
            int r = s - 1;
            while (r >= 0 && nb[r] > kb) {
                nb[r + 1] = nb[r];
                al[r + 1] = al[r];
                --r;
            }
            nb[r + 1] = kb;
            al[r + 1] = ka;
        }
        for (int s = 0; s < c; ++s) {
            if (!(fabs(al[s]) > cut)) continue;
            m->ej[q] = (int32_t)a;
            m->ek[q] = nb[s];
            m->alpha[q] = al[s];
            /* Eq. link variable: the phase of the link from x_a to x_b */
            m->theta[q] = edge_integral(m, m->x + 3 * a, m->x + 3 * (int64_t)nb[s]);
            ++q;
        }
    }
    free(t.cnt);
    free(t.nb);
    free(t.al);

    /* K-hat (Eq. discr kin energy with Remark rmk:dk), read as the derivative of
     * F_1 = sum_edges alpha |U psi_j - psi_k|^2:
     *   (K-hat psi)_j = sum_k alpha_jk (psi_j - exp(-i theta_jk) psi_k),
     * theta_jk = integral of A from x_j to x_k, so theta_kj = -theta_jk. */
    int64_t *deg = xcalloc((size_t)n, sizeof(int64_t));
    for (int64_t e = 0; e < ne; ++e) {
        deg[m->ej[e]]++;
        deg[m->ek[e]]++;
    }
    csr *K = &m->K;
    K->n = K->m = n;
    K->rp = xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) K->rp[i + 1] = K->rp[i] + deg[i] + 1;
    K->ci = xcalloc((size_t)K->rp[n], sizeof(int32_t));
    K->v = xcalloc((size_t)K->rp[n], sizeof(cplx));
    /* row entries: gather (column, value) then sort by column */
    int64_t *fill = xcalloc((size_t)n, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        K->ci[K->rp[i]] = (int32_t)i;
        K->v[K->rp[i]] = 0;
        fill[i] = 1;
    }
    for (int64_t e = 0; e < ne; ++e) {
        int64_t a = m->ej[e], b = m->ek[e];
        double al = m->alpha[e], th = m->theta[e];
        K->v[K->rp[a]] += al;
        K->v[K->rp[b]] += al;
        int64_t pa = K->rp[a] + fill[a]++;
        K->ci[pa] = (int32_t)b;
        K->v[pa] = -al * cexp(-I * th);
        int64_t pb = K->rp[b] + fill[b]++;
        K->ci[pb] = (int32_t)a;
        K->v[pb] = -al * cexp(I * th);
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo = K->rp[i], hi = K->rp[i + 1];
        for (int64_t s = lo + 1; s < hi; ++s) {
            int32_t kc = K->ci[s];
            cplx kv = K->v[s];
            int64_t r = s - 1;
            while (r >= lo && K->ci[r] > kc) {
                K->ci[r + 1] = K->ci[r];
                K->v[r + 1] = K->v[r];
                --r;
            }
            K->ci[r + 1] = kc;
            K->v[r + 1] = kv;
        }
    }
    free(fill);
    free(deg);
}

static glref_mesh *mesh_assemble(glref_mesh *m) {
    const int dim = m->dim, N = m->N;
    const double edge = m->edge;
    m->n = (dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    m->h = edge / (N - 1);
    int64_t n = m->n;
    int nz = (dim == 2) ? 1 : N;

    /* nodes of the square/cube centred at the origin */
    const double x0 = -0.5 * edge;
    m->x = xcalloc((size_t)n * 3, sizeof(double));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                int64_t id = node_id(m, i, j, k);
                m->x[3 * id + 0] = x0 + i * m->h;
                m->x[3 * id + 1] = x0 + j * m->h;
                m->x[3 * id + 2] = (dim == 3) ? x0 + k * m->h : 0.0;
            }

    /* control volumes: the Voronoi cell of a lattice node is the cube of side h
     * around it, clipped to the domain: h^d 2^(-number of boundary coordinates) */
    m->vol = xcalloc((size_t)n, sizeof(double));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                int nb = (i == 0 || i == N - 1) + (j == 0 || j == N - 1);
                if (dim == 3) nb += (k == 0 || k == N - 1);
                m->vol[node_id(m, i, j, k)] = pow(m->h, dim) / (double)(1 << nb);
            }

    /* Eq. fhat: alpha_jk = sum over the simplices adjacent to edge jk of the
     * simplex coefficients */
    edge_table t;
    t.n = n;
    t.cap = GLREF_MAXDEG;
    t.cnt = xcalloc((size_t)n, sizeof(int32_t));
    t.nb = xcalloc((size_t)n * GLREF_MAXDEG, sizeof(int32_t));
    t.al = xcalloc((size_t)n * GLREF_MAXDEG, sizeof(double));
    int ncell_z = (dim == 2) ? 1 : N - 1;
    int ea[6], eb[6];
    int nse = simplex_edges(dim, ea, eb);
    for (int k = 0; k < ncell_z; ++k)
        for (int j = 0; j < N - 1; ++j)
            for (int i = 0; i < N - 1; ++i) {
                int64_t vid[6][4];
                int ns = cell_simplices(m, i, j, k, vid);
                for (int s = 0; s < ns; ++s) {
                    double p[12];
                    for (int v = 0; v <= dim; ++v)
                        for (int c = 0; c < 3; ++c) p[3 * v + c] = m->x[3 * vid[s][v] + c];
                    double al[6];
                    int rc = (dim == 2) ? glref_simplex_alpha_cot(p, al) : glref_simplex_alpha_linsys(3, p, al);
                    if (rc) {
                        fprintf(stderr, "glref: degenerate simplex\n");
                        abort();
                    }
                    for (int e = 0; e < nse; ++e) table_add(&t, vid[s][ea[e]], vid[s][eb[e]], al[e]);
                }
            }

    mesh_edges_khat(m, &t);
    return m;
}

/* A mesh given by its nodes and simplices (the paper's Delaunay meshes of its
 * test domains, Sec. 4; any conforming simplicial mesh).  x: n x 3 coordinates
 * (z = 0 in 2D); simp: ns x (dim + 1) node ids.  The coefficient of each edge of
 * each simplex (the cotangent formula in 2D, its dihedral form in 3D) is summed
 * per edge in simplex order (Eq. fhat).  The control volumes
 * come from the same coefficients: by the corollary's identity taken over an
 * orthonormal basis, a simplex's volume is sum_e alpha_e |e|^2 / d, and the part
 * alpha_e |e|^2 / d of edge e lies half at each end, so |V_j| = sum_k alpha_jk
 * |x_j - x_k|^2 / (2 d) over the kept edges of j (the Voronoi region of x_j
 * within the mesh, for well-centred simplices; Eq. mass lumping).  Link phases
 * of A = (mu / 2) bhat x x, or of mu A_d when xd and md are given.  Returns NULL
 * on invalid input. */
void glref_mesh_destroy(glref_mesh *m);
glref_mesh *glref_mesh_create_simplicial(int dim, int64_t n, const double *x, int64_t ns, const int32_t *simp,
                                         double mu, const double *bhat, const double *xd, const double *md) {
    if ((dim != 2 && dim != 3) || n < 2 || ns < 1 || !x || !simp) return NULL;
    for (int64_t q = 0; q < ns * (dim + 1); ++q)
        if (simp[q] < 0 || simp[q] >= n) return NULL;
    glref_mesh *m = xcalloc(1, sizeof *m);
    m->dim = dim;
    m->N = 0;
    m->n = n;
    m->mu = mu;
    double b[3] = {0, 0, 1}, nb = 1;
    if (bhat) {
        nb = sqrt(dot3(bhat, bhat));
        for (int c = 0; c < 3; ++c) b[c] = bhat[c] / nb;
    }
    for (int c = 0; c < 3; ++c) m->bhat[c] = b[c];
    if (xd && md) {
        m->dipole = 1;
        for (int c = 0; c < 3; ++c) {
            m->xd[c] = xd[c];
            m->md[c] = md[c];
        }
    }
    m->x = xcalloc((size_t)n * 3, sizeof(double));
    memcpy(m->x, x, sizeof(double) * 3 * (size_t)n);
    if (dim == 2)
        for (int64_t j = 0; j < n; ++j) m->x[3 * j + 2] = 0.0;
    edge_table t;
    t.n = n;
    t.cap = 64;
    t.cnt = xcalloc((size_t)n, sizeof(int32_t));
    t.nb = xcalloc((size_t)n * t.cap, sizeof(int32_t));
    t.al = xcalloc((size_t)n * t.cap, sizeof(double));
    int ea[6], eb[6];
    const int nse = simplex_edges(dim, ea, eb);
    for (int64_t q = 0; q < ns; ++q) {
        const int32_t *v = simp + q * (dim + 1);
        double p[12], al[6];
        for (int k = 0; k <= dim; ++k)
            for (int c = 0; c < 3; ++c) p[3 * k + c] = m->x[3 * (int64_t)v[k] + c];
        int rc = (dim == 2) ? glref_simplex_alpha_cot(p, al) : glref_simplex_alpha_dihedral(p, al);
        if (rc) {
            free(t.cnt);
            free(t.nb);
            free(t.al);
            glref_mesh_destroy(m);
            return NULL;
        }
        for (int e = 0; e < nse; ++e) table_add(&t, v[ea[e]], v[eb[e]], al[e]);
    }
    mesh_edges_khat(m, &t);
    /* control volumes: the kept edges in lexicographic order reach each node in
     * the order of its neighbours' ids (those below it first) */
    m->vol = xcalloc((size_t)n, sizeof(double));
    for (int64_t e = 0; e < m->ne; ++e) {
        const int64_t a = m->ej[e], b = m->ek[e];
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = m->x[3 * b + c] - m->x[3 * a + c];
        const double part = m->alpha[e] * dot3(d, d) / (2.0 * dim);
        m->vol[a] += part;
        m->vol[b] += part;
    }
    return m;
}

glref_mesh *glref_mesh_create(int dim, int N, double mu, const double *bhat, const double *a0) {
    return glref_mesh_create_edge(dim, N, 1.0, mu, bhat, a0);
}

void glref_mesh_destroy(glref_mesh *m) {
    if (!m) return;
    free(m->x);
    free(m->vol);
    free(m->ej);
    free(m->ek);
    free(m->alpha);
    free(m->theta);
    csr_free(&m->K);
    free(m);
}

int64_t glref_mesh_n(const glref_mesh *m) { return m->n; }
int64_t glref_mesh_nedges(const glref_mesh *m) { return m->ne; }
int64_t glref_mesh_nnz(const glref_mesh *m) { return csr_nnz(&m->K); }

void glref_mesh_nodes(const glref_mesh *m, double *x) { memcpy(x, m->x, sizeof(double) * 3 * m->n); }
void glref_mesh_volumes(const glref_mesh *m, double *v) { memcpy(v, m->vol, sizeof(double) * m->n); }
void glref_mesh_edges(const glref_mesh *m, int32_t *ej, int32_t *ek, double *alpha, double *theta) {
    memcpy(ej, m->ej, sizeof(int32_t) * m->ne);
    memcpy(ek, m->ek, sizeof(int32_t) * m->ne);
    memcpy(alpha, m->alpha, sizeof(double) * m->ne);
    memcpy(theta, m->theta, sizeof(double) * m->ne);
}
void glref_mesh_khat(const glref_mesh *m, int64_t *rp, int32_t *ci, cplx *v) {
    memcpy(rp, m->K.rp, sizeof(int64_t) * (m->n + 1));
    memcpy(ci, m->K.ci, sizeof(int32_t) * csr_nnz(&m->K));
    memcpy(v, m->K.v, sizeof(cplx) * csr_nnz(&m->K));
}

/* ------------------------------------------------------------------ */
/* 4. operators                                                        */
/* ------------------------------------------------------------------ */

/* (K psi)_i = (K-hat psi)_i / |V_i|  (Remark rmk:dk: K = D^-1 K-hat) */
void glref_kinetic_apply(const glref_mesh *m, const cplx *psi, cplx *y) {
    csr_matvec(&m->K, psi, y);
    ROWS_PARALLEL
    for (int64_t i = 0; i < m->n; ++i) y[i] /= m->vol[i];
}

/* Eq. discr ginla: GL(psi)_i = (K psi)_i - psi_i (1 - |psi_i|^2) */
void glref_residual(const glref_mesh *m, const cplx *psi, cplx *r) {
    glref_kinetic_apply(m, psi, r);
    ROWS_PARALLEL
    for (int64_t i = 0; i < m->n; ++i) {
        double a2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        r[i] -= psi[i] * (1.0 - a2);
    }
}

/* Discrete Jacobian (Sec. 3): (J phi)_i = (K phi)_i + (-1 + 2|psi_i|^2) phi_i + psi_i^2 conj(phi_i) */
void glref_jacobian_apply(const glref_mesh *m, const cplx *psi, const cplx *phi, cplx *y) {
    glref_kinetic_apply(m, phi, y);
    ROWS_PARALLEL
    for (int64_t i = 0; i < m->n; ++i) {
        double a2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        y[i] += (-1.0 + 2.0 * a2) * phi[i] + psi[i] * psi[i] * conj(phi[i]);
    }
}

/* Eq. discr energy: F = F_1 + F_2 with F_1 = sum_edges alpha |U_jk psi_j - psi_k|^2
 * (|U psi_j - psi_k| = |psi_j - exp(-i theta_jk) psi_k|) and F_2 by Eq. mass lumping. */
double glref_energy(const glref_mesh *m, const cplx *psi) {
    double f1 = 0, f2 = 0;
    for (int64_t e = 0; e < m->ne; ++e) {
        cplx d = psi[m->ej[e]] - cexp(-I * m->theta[e]) * psi[m->ek[e]];
        f1 += m->alpha[e] * (creal(d) * creal(d) + cimag(d) * cimag(d));
    }
    for (int64_t i = 0; i < m->n; ++i) {
        double a2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        f2 += m->vol[i] * (-a2 + 0.5 * a2 * a2);
    }
    return f1 + f2;
}

/* d GL / d mu at fixed psi for A = mu A_1 + a0 (A_1 = (1/2) bhat x x): only the
 * link phases depend on mu, theta_jk = mu theta1_jk + (a0 part), so
 * d K-hat_jk / d mu = i theta1_jk alpha_jk exp(-i theta_jk) on the stored edge
 * j < k and its conjugate on (k, j); the diagonal sum of alpha does not move.
 * out = D^-1 (d K-hat / d mu) psi.  (The tangent of the continuation curve in
 * Sec. 4's parameter continuation needs this derivative.) */
void glref_residual_dmu(const glref_mesh *m, const cplx *psi, cplx *out) {
    for (int64_t i = 0; i < m->n; ++i) out[i] = 0;
    for (int64_t e = 0; e < m->ne; ++e) {
        const int64_t j = m->ej[e], k = m->ek[e];
        const double th1 = edge_integral1(m, m->x + 3 * j, m->x + 3 * k);
        const cplx djk = I * th1 * m->alpha[e] * cexp(-I * m->theta[e]);
        out[j] += djk * psi[k];
        out[k] += conj(djk) * psi[j];
    }
    for (int64_t i = 0; i < m->n; ++i) out[i] /= m->vol[i];
}

/* Eq. disc inner2: <x, y>_R = Re sum_i |V_i| conj(x_i) y_i */
double glref_inner_r(const glref_mesh *m, const cplx *x, const cplx *y) {
    double s = 0;
    for (int64_t i = 0; i < m->n; ++i) s += m->vol[i] * creal(conj(x[i]) * y[i]);
    return s;
}

/* ------------------------------------------------------------------ */
/* 5. smoothed-aggregation AMG for P-hat = K-hat + 2 D |psi|^2          */
/* ------------------------------------------------------------------ */

#define GLREF_CYCLES_INF (-1)
#define GLREF_RINF_TOL 1e-12
#define GLREF_RINF_MAXCYC 200

typedef struct {
    double tol;        /* relative residual target */
    int maxit;         /* MINRES iteration cap */
    int cycles;        /* k in R_k (Eq. prec2); 0 = no preconditioner;
                          GLREF_CYCLES_INF = R_inf, cycled to high accuracy (Eq. prec1) */
    int max_coarse;    /* stop coarsening at or below this size */
    int max_levels;
    int power_its;     /* power iterations for the spectral radius of D^-1 A */
    int coloring;      /* coarse-level colouring: GLREF_COLOR_PSL (default), GLREF_COLOR_SL or GLREF_COLOR_JP */
} glref_options;

#define GLREF_COLOR_SL 0
#define GLREF_COLOR_JP 1
#define GLREF_COLOR_PSL 2
/* degree slack of one removal round of the round-based smallest-last order */
#define GLREF_PSL_SLACK 4

typedef struct {
    csr A;            /* level operator (Hermitian) */
    int32_t *agg;     /* aggregate of each node (to the next level); NULL on the coarsest */
    double *B;        /* near-null candidate on this level */
    int32_t ncolors;
    int32_t *color;
    double rho, omega;
    csr P, PH;        /* prolongator from the next level, and its adjoint */
    cplx *chol;       /* coarsest level: lower Cholesky factor, row-major n x n */
} level_t;

typedef struct glref_prec {
    int nlev;
    int cycles;
    level_t L[GLREF_MAXLEV];
    const glref_mesh *mesh;
    cplx *work[GLREF_MAXLEV][3];
} glref_prec;

/* The fixed integer hash used for every priority (aggregation and colouring):
 * the "lowbias32" mixer (C. Wellons), applied to the node id. */
uint32_t glref_hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

/* priority key: (hash, id), unique per node; 0 is reserved for "no key" */
static uint64_t prio_key(int64_t i) { return (((uint64_t)glref_hash32((uint32_t)i)) << 32 | (uint64_t)(uint32_t)i) + 1; }

/* Aggregation by a distance-2 maximal independent set computed in synchronous
 * Luby rounds (Bell, Dalton & Olson 2012): in each round an undecided node
 * becomes a root if its key is the largest key of any undecided node within
 * graph distance 2; undecided nodes within distance 2 of a new root are then
 * excluded.  Roots get aggregate ids in ascending node-id order; neighbours of
 * a root join it; the remaining nodes join the neighbouring aggregate with the
 * smallest id.  Every off-diagonal is a strong connection (threshold 0).
 * Returns the number of aggregates. */
int64_t glref_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *agg) {
    enum { UNDECIDED = 0, ROOT = 1, OUT = 2 };
    uint8_t *state = xcalloc((size_t)n, 1);
    uint64_t *key = xcalloc((size_t)n, sizeof(uint64_t));
    uint64_t *m1 = xcalloc((size_t)n, sizeof(uint64_t));
    uint8_t *newroot = xcalloc((size_t)n, 1);
    uint8_t *d1 = xcalloc((size_t)n, 1);
    int64_t undecided = n;
    while (undecided > 0) {
        for (int64_t i = 0; i < n; ++i) key[i] = (state[i] == UNDECIDED) ? prio_key(i) : 0;
        for (int64_t i = 0; i < n; ++i) {       /* max over the closed 1-neighbourhood */
            uint64_t k = key[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) k = key[ci[p]] > k ? key[ci[p]] : k;
            m1[i] = k;
        }
        for (int64_t i = 0; i < n; ++i) {       /* max over the closed 2-neighbourhood */
            uint64_t k = m1[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) k = m1[ci[p]] > k ? m1[ci[p]] : k;
            newroot[i] = (state[i] == UNDECIDED && key[i] == k);
        }
        for (int64_t i = 0; i < n; ++i)
            if (newroot[i]) state[i] = ROOT;
        for (int64_t i = 0; i < n; ++i) {       /* within distance 1 of a new root */
            uint8_t f = newroot[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) f |= newroot[ci[p]];
            d1[i] = f;
        }
        for (int64_t i = 0; i < n; ++i) {       /* within distance 2 of a new root */
            if (state[i] != UNDECIDED) continue;
            uint8_t f = d1[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) f |= d1[ci[p]];
            if (f) state[i] = OUT;
        }
        undecided = 0;
        for (int64_t i = 0; i < n; ++i) undecided += (state[i] == UNDECIDED);
    }
    int64_t nagg = 0;
    for (int64_t i = 0; i < n; ++i) agg[i] = (state[i] == ROOT) ? (int32_t)(nagg++) : -1;
    /* neighbours of roots (roots are at least 3 apart, so the root is unique) */
    int32_t *first = xcalloc((size_t)n, sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) {
        first[i] = agg[i];
        if (agg[i] >= 0) continue;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (state[ci[p]] == ROOT) first[i] = agg[ci[p]];
    }
    /* the rest join the neighbouring aggregate with the smallest id */
    for (int64_t i = 0; i < n; ++i) {
        int32_t a = first[i];
        if (a < 0) {
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int32_t b = first[ci[p]];
                if (b >= 0 && (a < 0 || b < a)) a = b;
            }
        }
        agg[i] = a;
    }
    free(first);
    free(state);
    free(key);
    free(m1);
    free(newroot);
    free(d1);
    return nagg;
}

/* Jones-Plassmann colouring in synchronous rounds: an uncoloured node whose key
 * exceeds the keys of all its uncoloured neighbours takes the smallest colour
 * not used by its already coloured neighbours.  Returns the number of colours. */
int32_t glref_color_jp(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *color) {
    for (int64_t i = 0; i < n; ++i) color[i] = -1;
    uint8_t *pick = xcalloc((size_t)n, 1);
    int64_t left = n;
    int32_t ncol = 0;
    while (left > 0) {
        for (int64_t i = 0; i < n; ++i) {
            pick[i] = 0;
            if (color[i] >= 0) continue;
            uint64_t k = prio_key(i);
            int ok = 1;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int64_t j = ci[p];
                if (j != i && color[j] < 0 && prio_key(j) > k) ok = 0;
            }
            pick[i] = (uint8_t)ok;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (!pick[i]) continue;
            int32_t c = 0;
            for (;;) {
                int used = 0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                    if (ci[p] != i && color[ci[p]] == c) used = 1;
                if (!used) break;
                ++c;
            }
            color[i] = c;
            if (c + 1 > ncol) ncol = c + 1;
            --left;
        }
    }
    free(pick);
    return ncol;
}

/* Smallest-last colouring in rounds: Matula & Beck's smallest-last order with
 * whole sets removed at once, so that a parallel machine needs few rounds:
 *   degree d(v) = off-diagonal entries of row v among the vertices not yet
 *   removed (the graph is symmetric);
 *   round r = 0, 1, ...: with d_min the smallest degree of the remaining
 *   vertices, every remaining vertex with d(v) <= d_min + GLREF_PSL_SLACK (degrees
 *   as at the start of the round) is removed and gets level r;
 *   then the vertices are coloured greedily in decreasing (level, prio_key)
 *   order, each with the smallest colour that none of its already coloured
 *   neighbours has (a vertex removed later, i.e. in a denser remainder, first).
 * This is the greedy colouring of a total order, so a Jones-Plassmann colouring
 * with the key (level, prio_key) gives the same colours.  level (nullable): the
 * removal round of each vertex.  Returns the number of colours. */
static const int32_t *psl_level;
static int psl_cmp(const void *a, const void *b) {
    const int64_t u = *(const int64_t *)a, v = *(const int64_t *)b;
    if (psl_level[u] != psl_level[v]) return psl_level[u] > psl_level[v] ? -1 : 1;
    const uint64_t ku = prio_key(u), kv = prio_key(v);
    return ku > kv ? -1 : (ku < kv ? 1 : 0);
}
int32_t glref_color_psl(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *color, int32_t *level_out) {
    int64_t *deg = xcalloc((size_t)n, sizeof(int64_t));
    int32_t *level = xcalloc((size_t)n, sizeof(int32_t));
    uint8_t *sel = xcalloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        for (int64_t q = rp[v]; q < rp[v + 1]; ++q) deg[v] += (ci[q] != v);
    }
    int64_t remaining = n;
    for (int32_t r = 0; remaining > 0; ++r) {
        int64_t dmin = INT64_MAX;
        for (int64_t v = 0; v < n; ++v)
            if (level[v] < 0 && deg[v] < dmin) dmin = deg[v];
        for (int64_t v = 0; v < n; ++v) sel[v] = (level[v] < 0 && deg[v] <= dmin + GLREF_PSL_SLACK);
        for (int64_t v = 0; v < n; ++v)
            if (sel[v]) {
                level[v] = r;
                --remaining;
            }
        for (int64_t v = 0; v < n; ++v) {
            if (!sel[v]) continue;
            for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
                if (ci[q] != v && level[ci[q]] < 0) --deg[ci[q]];
        }
    }
    int64_t *order = xcalloc((size_t)n, sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) order[v] = v;
    psl_level = level;
    qsort(order, (size_t)n, sizeof(int64_t), psl_cmp);
    for (int64_t v = 0; v < n; ++v) color[v] = -1;
    int32_t ncol = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t v = order[k];
        int32_t c = 0;
        for (;;) {
            int used = 0;
            for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
                if (ci[q] != v && color[ci[q]] == c) used = 1;
            if (!used) break;
            ++c;
        }
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    if (level_out) memcpy(level_out, level, sizeof(int32_t) * (size_t)n);
    free(order);
    free(deg);
    free(level);
    free(sel);
    return ncol;
}

/* Smallest-last greedy colouring (Matula & Beck's smallest-last ordering, then
 * the greedy colouring in reverse removal order), made deterministic:
 *   degree d(v) = off-diagonal entries of row v (the graph is symmetric);
 *   vertices sit in degree buckets, each a list; they enter in ascending id,
 *   each at the head of its bucket;
 *   n times: take the head of the lowest non-empty bucket, remove it, and move
 *   each of its remaining neighbours (ascending column order) to the head of
 *   the bucket one degree lower;
 *   then colour the vertices from the last removed to the first, each with the
 *   smallest colour none of its coloured neighbours has.
 * Every vertex is removed with at most the graph's degeneracy k remaining
 * neighbours, all coloured after it, so at most k + 1 colours are used.
 * Returns the number of colours. */
int32_t glref_color_sl(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *color, int32_t *order) {
    int64_t *deg = xcalloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t maxd = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t p = rp[v]; p < rp[v + 1]; ++p)
            if (ci[p] != v) ++deg[v];
        if (deg[v] > maxd) maxd = deg[v];
    }
    int64_t *head = xcalloc((size_t)maxd + 1, sizeof(int64_t));
    int64_t *next = xcalloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t *prev = xcalloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    uint8_t *gone = xcalloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t d = 0; d <= maxd; ++d) head[d] = -1;
    /* list operations: unlink v from bucket deg[v]; push v at the head of bucket deg[v] */
#define SL_UNLINK(v)                                        \
    do {                                                    \
        if (prev[v] >= 0) next[prev[v]] = next[v];          \
        else head[deg[v]] = next[v];                        \
        if (next[v] >= 0) prev[next[v]] = prev[v];          \
    } while (0)
#define SL_PUSH(v)                                          \
    do {                                                    \
        prev[v] = -1;                                       \
        next[v] = head[deg[v]];                             \
        if (head[deg[v]] >= 0) prev[head[deg[v]]] = v;      \
        head[deg[v]] = v;                                   \
    } while (0)
    for (int64_t v = 0; v < n; ++v) SL_PUSH(v);
    int64_t lo = 0;
    for (int64_t step = 0; step < n; ++step) {
        while (head[lo] < 0) ++lo;
        int64_t v = head[lo];
        SL_UNLINK(v);
        gone[v] = 1;
        order[n - 1 - step] = (int32_t)v;
        for (int64_t p = rp[v]; p < rp[v + 1]; ++p) {
            int64_t u = ci[p];
            if (u == v || gone[u]) continue;
            SL_UNLINK(u);
            --deg[u];
            SL_PUSH(u);
        }
        lo = lo > 0 ? lo - 1 : 0;
    }
#undef SL_UNLINK
#undef SL_PUSH
    /* greedy in that order; stamp[c] = the vertex that last saw colour c taken */
    int64_t *stamp = xcalloc((size_t)maxd + 2, sizeof(int64_t));
    for (int64_t c = 0; c <= maxd + 1; ++c) stamp[c] = -1;
    for (int64_t v = 0; v < n; ++v) color[v] = -1;
    int32_t ncol = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = order[k];
        for (int64_t p = rp[v]; p < rp[v + 1]; ++p) {
            int64_t u = ci[p];
            if (u != v && color[u] >= 0) stamp[color[u]] = v;
        }
        int32_t c = 0;
        while (stamp[c] == v) ++c;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(deg);
    free(head);
    free(next);
    free(prev);
    free(gone);
    free(stamp);
    return ncol;
}

/* spectral radius estimate of D^-1 A: `its` power iterations from the fixed
 * start x_i = 1 + (i mod 7)/7, then the Rayleigh quotient in the D inner
 * product, Re(x^H A x) / (x^H D x). */
double glref_spectral_radius(const csr *A, int its) {
    int64_t n = A->n;
    cplx *x = xcalloc((size_t)n, sizeof(cplx)), *y = xcalloc((size_t)n, sizeof(cplx));
    double *d = xcalloc((size_t)n, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        x[i] = 1.0 + (double)(i % 7) / 7.0;
        d[i] = creal(csr_get(A, i, i));
    }
    for (int it = 0; it < its; ++it) {
        csr_matvec(A, x, y);
        double nrm = 0;
        for (int64_t i = 0; i < n; ++i) {
            y[i] /= d[i];
            nrm += creal(y[i]) * creal(y[i]) + cimag(y[i]) * cimag(y[i]);
        }
        nrm = sqrt(nrm);
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    csr_matvec(A, x, y);
    double num = 0, den = 0;
    for (int64_t i = 0; i < n; ++i) {
        num += creal(conj(x[i]) * y[i]);
        den += d[i] * (creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]));
    }
    free(x);
    free(y);
    free(d);
    return num / den;
}

/* dense Hermitian Cholesky A = L L^H, row-major; returns 0 on success */
static int dense_cholesky(int64_t n, const csr *A, cplx *L) {
    memset(L, 0, sizeof(cplx) * n * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) L[i * n + A->ci[p]] = A->v[p];
    for (int64_t j = 0; j < n; ++j) {
        double s = creal(L[j * n + j]);
        for (int64_t k = 0; k < j; ++k) s -= creal(L[j * n + k] * conj(L[j * n + k]));
        if (!(s > 0)) return -1;
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            cplx t = L[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= L[i * n + k] * conj(L[j * n + k]);
            L[i * n + j] = t / ljj;
        }
        for (int64_t k = j + 1; k < n; ++k) L[j * n + k] = 0;
    }
    return 0;
}

static void dense_cholesky_solve(int64_t n, const cplx *L, const cplx *b, cplx *x) {
    for (int64_t i = 0; i < n; ++i) {
        cplx s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / creal(L[i * n + i]);
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        cplx s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s -= conj(L[k * n + i]) * x[k];
        x[i] = s / creal(L[i * n + i]);
    }
}

void glref_precond_destroy(glref_prec *p) {
    if (!p) return;
    for (int l = 0; l < p->nlev; ++l) {
        level_t *L = &p->L[l];
        csr_free(&L->A);
        csr_free(&L->P);
        csr_free(&L->PH);
        free(L->agg);
        free(L->B);
        free(L->color);
        free(L->chol);
        for (int w = 0; w < 3; ++w) free(p->work[l][w]);
    }
    free(p);
}

/* Setup of R_k (Eq. prec2) for P-hat = K-hat + 2 D |psi|^2 (Sec. 4.1).  The
 * paper names smoothed aggregation with symmetric Gauss-Seidel (PyAMG); the
 * remaining choices are this implementation's reading:
 *   candidate B = 1 on the finest level, B_c = aggregate norms of B below;
 *   tentative P_tent[i, agg(i)] = B_i / ||B restricted to agg(i)||;
 *   P = (I - omega D^-1 A) P_tent with omega = 4 / (3 rho(D^-1 A));
 *   Galerkin A_c = P^H A P, made exactly Hermitian as (A_c + A_c^H)/2;
 *   colours: red-black (i+j+k mod 2) on the finest lattice level, the
 *   options' colouring below and on the finest level of a general simplicial
 *   mesh; coarsest level factored by dense Cholesky. */
glref_prec *glref_precond_setup(const glref_mesh *m, const cplx *psi, const glref_options *o) {
    glref_prec *p = xcalloc(1, sizeof *p);
    p->mesh = m;
    p->cycles = o->cycles == GLREF_CYCLES_INF ? GLREF_CYCLES_INF : (o->cycles > 0 ? o->cycles : 1);
    int maxlev = o->max_levels > 0 ? o->max_levels : 10;
    if (maxlev > GLREF_MAXLEV) maxlev = GLREF_MAXLEV;
    int64_t max_coarse = o->max_coarse > 0 ? o->max_coarse : 512;
    int power_its = o->power_its > 0 ? o->power_its : 20;

    /* level 0: P-hat = K-hat + 2 D |psi|^2 (a diagonal update of K-hat) */
    level_t *L0 = &p->L[0];
    int64_t n = m->n, nnz = csr_nnz(&m->K);
    L0->A.n = L0->A.m = n;
    L0->A.rp = xcalloc((size_t)n + 1, sizeof(int64_t));
    L0->A.ci = xcalloc((size_t)nnz, sizeof(int32_t));
    L0->A.v = xcalloc((size_t)nnz, sizeof(cplx));
    memcpy(L0->A.rp, m->K.rp, sizeof(int64_t) * (n + 1));
    memcpy(L0->A.ci, m->K.ci, sizeof(int32_t) * nnz);
    memcpy(L0->A.v, m->K.v, sizeof(cplx) * nnz);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = m->K.rp[i]; q < m->K.rp[i + 1]; ++q)
            if (m->K.ci[q] == i) {
                double a2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
                L0->A.v[q] += 2.0 * m->vol[i] * a2;
            }
    L0->B = xcalloc((size_t)n, sizeof(double));
    for (int64_t i = 0; i < n; ++i) L0->B[i] = 1.0;

    int l = 0;
    for (;;) {
        level_t *L = &p->L[l];
        int64_t nl = L->A.n;
        /* colours */
        L->color = xcalloc((size_t)nl, sizeof(int32_t));
        if (l == 0 && m->N > 0) {
            int nz = (m->dim == 2) ? 1 : m->N;
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < m->N; ++j)
                    for (int i = 0; i < m->N; ++i) L->color[node_id(m, i, j, k)] = (i + j + k) & 1;
            L->ncolors = (nl > 1) ? 2 : 1;
        } else if (o->coloring == GLREF_COLOR_JP) {
            L->ncolors = glref_color_jp(nl, L->A.rp, L->A.ci, L->color);
        } else if (o->coloring == GLREF_COLOR_PSL) {
            L->ncolors = glref_color_psl(nl, L->A.rp, L->A.ci, L->color, NULL);
        } else {
            int32_t *order = xcalloc((size_t)nl, sizeof(int32_t));
            L->ncolors = glref_color_sl(nl, L->A.rp, L->A.ci, L->color, order);
            free(order);
        }
        for (int w = 0; w < 3; ++w) p->work[l][w] = xcalloc((size_t)nl, sizeof(cplx));
        if (nl <= max_coarse || l + 1 >= maxlev) break;
        /* aggregation */
        L->agg = xcalloc((size_t)nl, sizeof(int32_t));
        int64_t nc = glref_aggregate(nl, L->A.rp, L->A.ci, L->agg);
        if (nc >= nl || nc == 0) {
            free(L->agg);
            L->agg = NULL;
            break;
        }
        /* tentative prolongator */
        double *bn = xcalloc((size_t)nc, sizeof(double));
        for (int64_t i = 0; i < nl; ++i) bn[L->agg[i]] += L->B[i] * L->B[i];
        for (int64_t c = 0; c < nc; ++c) bn[c] = sqrt(bn[c]);
        csr Pt;
        Pt.n = nl;
        Pt.m = nc;
        Pt.rp = xcalloc((size_t)nl + 1, sizeof(int64_t));
        Pt.ci = xcalloc((size_t)nl, sizeof(int32_t));
        Pt.v = xcalloc((size_t)nl, sizeof(cplx));
        for (int64_t i = 0; i < nl; ++i) {
            Pt.rp[i + 1] = i + 1;
            Pt.ci[i] = L->agg[i];
            Pt.v[i] = L->B[i] / bn[L->agg[i]];
        }
        /* prolongator smoothing */
        L->rho = glref_spectral_radius(&L->A, power_its);
        L->omega = 4.0 / (3.0 * L->rho);
        csr AP;
        csr_matmul(&L->A, &Pt, &AP);
        for (int64_t i = 0; i < nl; ++i) {
            double dii = creal(csr_get(&L->A, i, i));
            for (int64_t q = AP.rp[i]; q < AP.rp[i + 1]; ++q) {
                cplx pt = (AP.ci[q] == L->agg[i]) ? Pt.v[i] : 0;
                AP.v[q] = pt - L->omega / dii * AP.v[q];
            }
        }
        L->P = AP; /* AP now holds P (same pattern as A P_tent) */
        csr_free(&Pt);
        csr_adjoint(&L->P, &L->PH);
        /* Galerkin coarse operator */
        csr T, Ac;
        csr_matmul(&L->A, &L->P, &T);
        csr_matmul(&L->PH, &T, &Ac);
        csr_free(&T);
        for (int64_t i = 0; i < nc; ++i)
            for (int64_t q = Ac.rp[i]; q < Ac.rp[i + 1]; ++q) {
                int64_t j = Ac.ci[q];
                if (j < i) continue;
                cplx aij = Ac.v[q], aji = csr_get(&Ac, j, i);
                cplx s = 0.5 * (aij + conj(aji));
                Ac.v[q] = s;
                for (int64_t r = Ac.rp[j]; r < Ac.rp[j + 1]; ++r)
                    if (Ac.ci[r] == i) Ac.v[r] = conj(s);
            }
        level_t *Lc = &p->L[l + 1];
        Lc->A = Ac;
        Lc->B = bn;
        ++l;
    }
    p->nlev = l + 1;
    /* coarsest level: dense Cholesky */
    level_t *Lc = &p->L[l];
    int64_t nc = Lc->A.n;
    if (nc > 8192) {
        glref_precond_destroy(p);
        return NULL;
    }
    Lc->chol = xcalloc((size_t)(nc * nc), sizeof(cplx));
    if (dense_cholesky(nc, &Lc->A, Lc->chol)) {
        glref_precond_destroy(p);
        return NULL;
    }
    return p;
}

int glref_prec_nlevels(const glref_prec *p) { return p->nlev; }

void glref_prec_level_info(const glref_prec *p, int l, int64_t *n, int64_t *nnz, int32_t *ncolors, int64_t *p_nnz,
                           double *omega) {
    const level_t *L = &p->L[l];
    *n = L->A.n;
    *nnz = csr_nnz(&L->A);
    *ncolors = L->ncolors;
    *p_nnz = (l + 1 < p->nlev) ? csr_nnz(&L->P) : 0;
    *omega = (l + 1 < p->nlev) ? L->omega : 0.0;
}

void glref_prec_level_matrix(const glref_prec *p, int l, int64_t *rp, int32_t *ci, cplx *v) {
    const csr *A = &p->L[l].A;
    memcpy(rp, A->rp, sizeof(int64_t) * (A->n + 1));
    memcpy(ci, A->ci, sizeof(int32_t) * csr_nnz(A));
    memcpy(v, A->v, sizeof(cplx) * csr_nnz(A));
}

void glref_prec_level_P(const glref_prec *p, int l, int64_t *rp, int32_t *ci, cplx *v) {
    const csr *A = &p->L[l].P;
    memcpy(rp, A->rp, sizeof(int64_t) * (A->n + 1));
    memcpy(ci, A->ci, sizeof(int32_t) * csr_nnz(A));
    memcpy(v, A->v, sizeof(cplx) * csr_nnz(A));
}

void glref_prec_level_aggregates(const glref_prec *p, int l, int32_t *agg) {
    memcpy(agg, p->L[l].agg, sizeof(int32_t) * p->L[l].A.n);
}

void glref_prec_level_colors(const glref_prec *p, int l, int32_t *color) {
    memcpy(color, p->L[l].color, sizeof(int32_t) * p->L[l].A.n);
}

/* one Gauss-Seidel sweep over the rows of colour c:
 * x_i <- (b_i - sum_{j != i} A_ij x_j) / A_ii */
static void gs_color(const level_t *L, int32_t c, const cplx *b, cplx *x) {
    const csr *A = &L->A;
    /* rows of one colour are not coupled: any order gives the same values */
    ROWS_PARALLEL
    for (int64_t i = 0; i < A->n; ++i) {
        if (L->color[i] != c) continue;
        cplx s = b[i];
        double d = 0;
        for (int64_t q = A->rp[i]; q < A->rp[i + 1]; ++q) {
            if (A->ci[q] == i)
                d = creal(A->v[q]);
            else
                s -= A->v[q] * x[A->ci[q]];
        }
        x[i] = s / d;
    }
}

/* symmetric Gauss-Seidel: a forward sweep (colours ascending) then a backward
 * sweep (colours descending) */
static void sgs(const level_t *L, const cplx *b, cplx *x) {
    for (int32_t c = 0; c < L->ncolors; ++c) gs_color(L, c, b, x);
    for (int32_t c = L->ncolors - 1; c >= 0; --c) gs_color(L, c, b, x);
}

/* one V-cycle for A_l x = b from x = 0 (Sec. 4: one pre- and one post-smoothing
 * step of symmetric Gauss-Seidel) */
static void vcycle(const glref_prec *p, int l, const cplx *b, cplx *x) {
    const level_t *L = &p->L[l];
    int64_t n = L->A.n;
    if (l == p->nlev - 1) {
        dense_cholesky_solve(n, L->chol, b, x);
        return;
    }
    cplx *r = p->work[l][0];
    cplx *bc = p->work[l + 1][1], *xc = p->work[l + 1][2];
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) x[i] = 0;
    sgs(L, b, x);
    csr_matvec(&L->A, x, r);
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    csr_matvec(&L->PH, r, bc);
    vcycle(p, l + 1, bc, xc);
    csr_matvec(&L->P, xc, r);
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) x[i] += r[i];
    sgs(L, b, x);
}

/* z = R_k v = AMG_k(P-hat, D v) (Eq. prec2): k V-cycles for P-hat z = D v from
 * z = 0.  R_inf (Eq. prec1, P^-1 D v) is the same iteration cycled until the
 * scaled residual D^-1 (D v - P-hat z) is at most GLREF_RINF_TOL of v in the
 * norm ||x||_D^2 = sum_i |V_i| |x_i|^2, checked after every cycle, with at most
 * GLREF_RINF_MAXCYC cycles.  Returns the number of V-cycles applied. */
int glref_precond_apply_count(const glref_prec *p, const cplx *v, cplx *z) {
    const glref_mesh *m = p->mesh;
    int64_t n = m->n;
    cplx *b = xcalloc((size_t)n, sizeof(cplx)), *e = xcalloc((size_t)n, sizeof(cplx));
    cplx *r = xcalloc((size_t)n, sizeof(cplx));
    double v2 = 0;
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) {
        b[i] = m->vol[i] * v[i];
        z[i] = 0;
    }
    for (int64_t i = 0; i < n; ++i) v2 += m->vol[i] * (creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]));
    const int inf = p->cycles == GLREF_CYCLES_INF;
    const int kmax = inf ? GLREF_RINF_MAXCYC : p->cycles;
    int k = 0;
    for (;;) {
        csr_matvec(&p->L[0].A, z, r);
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        if (inf && k > 0) {
            /* ||D^-1 r||_D^2 = sum |r_i|^2 / |V_i| */
            double r2 = 0;
            for (int64_t i = 0; i < n; ++i) r2 += (creal(r[i]) * creal(r[i]) + cimag(r[i]) * cimag(r[i])) / m->vol[i];
            if (!(r2 > GLREF_RINF_TOL * GLREF_RINF_TOL * v2)) break;
        }
        if (k == kmax) break;
        vcycle(p, 0, r, e);
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) z[i] += e[i];
        ++k;
    }
    free(b);
    free(e);
    free(r);
    return k;
}

void glref_precond_apply(const glref_prec *p, const cplx *v, cplx *z) { (void)glref_precond_apply_count(p, v, z); }

/* one V-cycle on level l for A_l x = b (exposed for the tests) */
void glref_vcycle(const glref_prec *p, int l, const cplx *b, cplx *x) { vcycle(p, l, b, x); }

/* ------------------------------------------------------------------ */
/* 6. preconditioned MINRES in <.,.>_R                                  */
/* ------------------------------------------------------------------ */

typedef struct {
    int iters;
    int converged;
    double true_relres;  /* ||b - J x||_D / ||b||_D */
    double est_relres;   /* MINRES recurrence estimate, preconditioned norm */
} glref_info;

static double norm_r(const glref_mesh *m, const cplx *x) { return sqrt(glref_inner_r(m, x, x)); }

static double true_relres(const glref_mesh *m, const cplx *psi, const cplx *b, const cplx *x, double bnorm,
                          cplx *tmp) {
    glref_jacobian_apply(m, psi, x, tmp);
    ROWS_PARALLEL
    for (int64_t i = 0; i < m->n; ++i) tmp[i] = b[i] - tmp[i];
    return norm_r(m, tmp) / bnorm;
}

/* z = R v, or z = v when no preconditioner is given (k = 0 in Fig. 1) */
static void apply_prec(const glref_prec *p, int64_t n, const cplx *v, cplx *z) {
    if (p)
        glref_precond_apply(p, v, z);
    else
        memcpy(z, v, sizeof(cplx) * n);
}

/* Preconditioned MINRES (Paige & Saunders 1975) for J(psi) x = b, J self-adjoint
 * in <.,.>_R (Sec. 3), preconditioner R_k (Eq. prec2), self-adjoint positive
 * definite in the same inner product.  x holds the initial guess on entry.
 * Stopping: the tolerance is relative to b (Sec. 4: the relative residual in the
 * norm of Eq. disc inner2).  The recurrence's estimate |eta| / eta_0 is relative
 * to the initial residual r_0 = b - J x_0, so it is scaled by
 * rho_0 = ||r_0||_D / ||b||_D (1 from x_0 = 0); once rho_0 |eta| / eta_0 <= tol the
 * true residual ||b - J x||_D / ||b||_D is computed, and the iteration stops when
 * that is <= tol as well.  Returns 0 when converged, 1 at maxit, 2 on breakdown. */
int glref_minres(const glref_mesh *m, const cplx *psi, const glref_prec *prec, const cplx *b, cplx *x,
                 const glref_options *o, glref_info *info) {
    int64_t n = m->n;
    cplx *v_old = xcalloc((size_t)n, sizeof(cplx)), *v = xcalloc((size_t)n, sizeof(cplx));
    cplx *v_new = xcalloc((size_t)n, sizeof(cplx)), *z = xcalloc((size_t)n, sizeof(cplx));
    cplx *z_new = xcalloc((size_t)n, sizeof(cplx)), *q = xcalloc((size_t)n, sizeof(cplx));
    cplx *w_old = xcalloc((size_t)n, sizeof(cplx)), *w = xcalloc((size_t)n, sizeof(cplx));
    cplx *w_new = xcalloc((size_t)n, sizeof(cplx)), *tmp = xcalloc((size_t)n, sizeof(cplx));
    int status = 1;
    double bnorm = norm_r(m, b);
    info->iters = 0;
    info->converged = 0;
    info->true_relres = 0;
    info->est_relres = 0;
    if (bnorm == 0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0;
        info->converged = 1;
        status = 0;
        goto done;
    }
    /* v_1 = b - J x_0, z_1 = R v_1, gamma_1 = sqrt(<v_1, z_1>_R) */
    glref_jacobian_apply(m, psi, x, q);
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) v[i] = b[i] - q[i];
    apply_prec(prec, n, v, z);
    double gamma = glref_inner_r(m, v, z);
    if (gamma < 0) {
        status = 2;
        goto done;
    }
    gamma = sqrt(gamma);
    double gamma_old = 1.0;
    double eta = gamma, eta0 = gamma;
    double c_old = 1, c = 1, s_old = 0, s = 0;
    info->true_relres = true_relres(m, psi, b, x, bnorm, tmp);
    const double rho0 = info->true_relres;  /* ||r_0||_D / ||b||_D */
    if (gamma == 0 || info->true_relres <= o->tol) {
        info->converged = 1;
        status = 0;
        goto done;
    }
    for (int it = 1; it <= o->maxit; ++it) {
        /* Lanczos step: z <- z / gamma, delta = <J z, z>_R */
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) z[i] /= gamma;
        glref_jacobian_apply(m, psi, z, q);
        double delta = glref_inner_r(m, q, z);
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) v_new[i] = q[i] - (delta / gamma) * v[i] - (gamma / gamma_old) * v_old[i];
        apply_prec(prec, n, v_new, z_new);
        double gamma_new = glref_inner_r(m, v_new, z_new);
        if (gamma_new < 0) {
            status = 2;
            info->iters = it;
            goto done;
        }
        gamma_new = sqrt(gamma_new);
        /* Givens rotations on the tridiagonal */
        double a0 = c * delta - c_old * s * gamma;
        double a1 = sqrt(a0 * a0 + gamma_new * gamma_new);
        double a2 = s * delta + c_old * c * gamma;
        double a3 = s_old * gamma;
        double c_new = a0 / a1, s_new = gamma_new / a1;
        /* search direction and update */
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) w_new[i] = (z[i] - a3 * w_old[i] - a2 * w[i]) / a1;
        ROWS_PARALLEL
        for (int64_t i = 0; i < n; ++i) x[i] += c_new * eta * w_new[i];
        eta = -s_new * eta;
        /* shift */
        cplx *t;
        t = v_old; v_old = v; v = v_new; v_new = t;
        t = z; z = z_new; z_new = t;
        t = w_old; w_old = w; w = w_new; w_new = t;
        gamma_old = gamma;
        gamma = gamma_new;
        c_old = c;
        c = c_new;
        s_old = s;
        s = s_new;
        info->iters = it;
        info->est_relres = rho0 * fabs(eta) / eta0;
        if (info->est_relres <= o->tol) {
            info->true_relres = true_relres(m, psi, b, x, bnorm, tmp);
            if (info->true_relres <= o->tol) {
                info->converged = 1;
                status = 0;
                goto done;
            }
        }
        if (gamma == 0) break;
    }
    info->true_relres = true_relres(m, psi, b, x, bnorm, tmp);
    info->converged = info->true_relres <= o->tol;
    status = info->converged ? 0 : 1;
done:
    free(v_old); free(v); free(v_new); free(z); free(z_new);
    free(q); free(w_old); free(w); free(w_new); free(tmp);
    return status;
}

/* setup + solve in one call */
int glref_jacobian_solve(const glref_mesh *m, const cplx *psi, const cplx *b, cplx *x, const glref_options *o,
                         glref_info *info) {
    glref_prec *p = NULL;
    if (o->cycles != 0) {
        p = glref_precond_setup(m, psi, o);
        if (!p) return 3;
    }
    int rc = glref_minres(m, psi, p, b, x, o, info);
    glref_precond_destroy(p);
    return rc;
}

/* Newton step on Eq. Newton system: solve J(psi) d = -GL(psi), psi <- psi + d.
 * Returns ||GL(psi)||_R of the state on entry in *gl_norm. */
int glref_newton_step(const glref_mesh *m, cplx *psi, const glref_options *o, glref_info *info, double *gl_norm) {
    int64_t n = m->n;
    cplx *r = xcalloc((size_t)n, sizeof(cplx)), *d = xcalloc((size_t)n, sizeof(cplx));
    glref_residual(m, psi, r);
    *gl_norm = norm_r(m, r);
    for (int64_t i = 0; i < n; ++i) r[i] = -r[i];
    int rc = glref_jacobian_solve(m, psi, r, d, o, info);
    for (int64_t i = 0; i < n; ++i) psi[i] += d[i];
    free(r);
    free(d);
    return rc;
}

/* ------------------------------------------------------------------ */
/* 7. dense pin: the realified 2n x 2n system (Remark rmk:isometry)     */
/* ------------------------------------------------------------------ */

/* Builds the real 2n x 2n matrix of phi -> J(psi) phi on [Re phi; Im phi]
 * column by column (row-major output). */
void glref_jacobian_dense_real(const glref_mesh *m, const cplx *psi, double *Jr) {
    int64_t n = m->n, n2 = 2 * n;
    cplx *e = xcalloc((size_t)n, sizeof(cplx)), *y = xcalloc((size_t)n, sizeof(cplx));
    for (int64_t col = 0; col < n2; ++col) {
        for (int64_t i = 0; i < n; ++i) e[i] = 0;
        e[col % n] = (col < n) ? 1.0 : I;
        glref_jacobian_apply(m, psi, e, y);
        for (int64_t i = 0; i < n; ++i) {
            Jr[i * n2 + col] = creal(y[i]);
            Jr[(n + i) * n2 + col] = cimag(y[i]);
        }
    }
    free(e);
    free(y);
}

/* LU with partial pivoting; solves A x = b in place (A row-major n x n,
 * destroyed).  Returns 0 on success, -1 if singular. */
int glref_lu_solve(int64_t n, double *A, double *b) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (A[piv * n + k] == 0) return -1;
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            if (f == 0) continue;
            for (int64_t j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    return 0;
}

/* dense direct solve of J(psi) x = b through the realified system */
int glref_dense_solve(const glref_mesh *m, const cplx *psi, const cplx *b, cplx *x) {
    int64_t n = m->n, n2 = 2 * n;
    double *A = xcalloc((size_t)(n2 * n2), sizeof(double)), *rhs = xcalloc((size_t)n2, sizeof(double));
    glref_jacobian_dense_real(m, psi, A);
    for (int64_t i = 0; i < n; ++i) {
        rhs[i] = creal(b[i]);
        rhs[n + i] = cimag(b[i]);
    }
    int rc = glref_lu_solve(n2, A, rhs);
    for (int64_t i = 0; i < n; ++i) x[i] = rhs[i] + I * rhs[n + i];
    free(A);
    free(rhs);
    return rc;
}
