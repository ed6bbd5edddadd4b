/*
 * gl.h -- C ABI of the GB300 library for the Jacobian solve of the extreme
 * type-II Ginzburg-Landau problem (Schloemer & Vanroose, "An optimal linear
 * solver for the Jacobian system of the extreme type-II Ginzburg-Landau
 * problem", arXiv:1204.5125).
 *
 * Conventions shared by every call below.
 *   - Complex vectors are arrays of n interleaved (re, im) FP64 pairs
 *     (C99 double complex / numpy complex128 layout), n = number of mesh nodes.
 *     Node j = i + N*(j_y + N*k) for lattice coordinates (i, j_y, k), x fastest.
 *   - Every pointer named *_dev is a device pointer of the current CUDA device;
 *     the caller allocates and owns it.  Pointers named *_host are host memory,
 *     also owned by the caller.  No call retains a caller pointer after it
 *     returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that only launch work return as soon as it is queued; the
 *     caller synchronises the stream before reading results.  Calls that return
 *     host values (setup, solve, info) synchronise the stream themselves.
 *   - The library owns gl_mesh and gl_prec handles (all their device memory)
 *     until the matching *_destroy call.
 *   - Every call returns a gl_status.  On failure gl_last_error() returns a
 *     message (per host thread) and outputs are unspecified unless stated.
 *   - Only structured meshes are supported: the unit square (dim 2) or cube
 *     (dim 3) centred at the origin with N nodes per side, spacing h = 1/(N-1),
 *     split into right triangles along the (i,j)-(i+1,j+1) diagonal in 2D and
 *     into Kuhn (Freudenthal) tetrahedra along the main diagonal in 3D.
 */
#ifndef GL_GB300_H
#define GL_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define GL_API __attribute__((visibility("default")))
#else
#define GL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gl_mesh_s *gl_mesh;
typedef struct gl_prec_s *gl_prec;
typedef struct gl_batch_s *gl_batch;
typedef struct gl_warmstart_s *gl_warmstart;

/* Size of the warm-start network's flat parameter vector: four 64 x 128 layer
 * matrices W^0..W^3 (row-major, outputs x inputs), then the 2 x 64 head U. */
#define GL_WS_NPARAM (4 * 64 * 128 + 2 * 64)

typedef enum {
    GL_OK = 0,
    GL_ERR_ARG = 1,           /* invalid argument (null handle, bad size, ...) */
    GL_ERR_CUDA = 2,          /* a CUDA runtime call or kernel failed */
    GL_ERR_OOM = 3,           /* device allocation failed */
    GL_ERR_NOT_CONVERGED = 4, /* solve stopped at maxit, or (FP64) its true residual stayed above tol while
                                 the MINRES estimate fell nine decades below it (the attainable accuracy
                                 of the iterate); x holds the last iterate */
    GL_ERR_BREAKDOWN = 5,     /* preconditioner not positive definite (<v, R v>_R < 0) */
    GL_ERR_NAN = 6,           /* a non-finite residual or scalar appeared */
    GL_ERR_TIMEOUT = 7,       /* a bounded device-side wait ran out */
    GL_ERR_CAPACITY = 8       /* an internal per-row or per-level limit was exceeded */
} gl_status;

typedef enum {
    GL_FP64 = 0,          /* everything in FP64 complex */
    GL_MIXED = 1,         /* FP64 defect correction around inner MINRES solves whose vectors,
                             Jacobian applies and V-cycles are FP32 complex */
    GL_MIXED_PRECOND = 2, /* FP64 MINRES and Jacobian applies; the V-cycle of R_k runs in FP32 */
    GL_APPLY_FP64_TABLES = 3 /* gl_jacobian_apply only: the FP64 apply from the lattice stencil's FP64 tables */
} gl_precision;

/* options.cycles value selecting R_inf = P^-1 D (Eq. prec1), realised as the
 * V-cycle repeated until ||D^-1 (D x - P-hat z)||_D <= 1e-12 ||x||_D (checked
 * after every cycle on the device, at most 200 cycles).  FP64 only: a setup or
 * solve with another precision returns GL_ERR_ARG, and so does gl_batch_create. */
#define GL_CYCLES_INF (-1)

/* Solver options.  Fill with gl_options_default() and override fields. */
typedef struct {
    double tol;          /* target ||b - J x||_D / ||b||_D (default 1e-10) */
    int maxit;           /* MINRES iteration cap (inner cap in GL_MIXED) (default 500) */
    int cycles;          /* k in R_k = AMG_k(...) (Eq. prec2); 0 = no preconditioner; GL_CYCLES_INF = R_inf
                            (Eq. prec1), see gl_precond_apply (default 1) */
    int max_coarse;      /* stop coarsening at or below this many nodes (default 512, max 4096) */
    int max_levels;      /* hierarchy depth cap (default 10, max 16) */
    int power_its;       /* power iterations for rho(D^-1 A) in prolongator smoothing (default 20) */
    int precision;       /* gl_precision (default GL_FP64); the coarsest solve keeps FP64 accuracy in
                            every mode (see coarse_df) */
    double inner_tol;    /* GL_MIXED: relative reduction asked of each FP32 inner solve (default 1e-5) */
    int max_outer;       /* GL_MIXED: cap on FP64 refinement steps (default 20) */
    int check_every;     /* host polls the device convergence flag every this many iterations (default 6) */
    int autotune;        /* 1: at setup, time the SpMV variants of every coarse operator on this GPU and keep
                            the fastest lanes-per-row width (default 1) */
    int lattice;         /* 1: on a mesh with an even number of nodes per side, the FP32 finest-level
                            sweeps and residuals of the V-cycle use the closed-form lattice stencil (checked
                            entry by entry against the assembled K at setup) instead of the stored one;
                            2: as 1, and MINRES's FP64 Jacobian also runs matrix-free from the stencil's
                            FP64 tables where they match the stored K to 16 ulp of its largest entry (it
                            reads a quarter of the bytes but is bound by this GPU's FP64 rate, and took
                            longer than the stored form when measured); 0: always the stored stencil
                            (default 1) */
    int cluster_sweeps;  /* 1: FP32 coarse-level Gauss-Seidel steps whose level vector fits the shared memory
                            of one thread-block cluster may run in that cluster (hardware barrier between
                            colours) instead of a cooperative grid: with autotune, where the setup timing
                            finds it faster; without, wherever it fits; 0: always the grid (default 1) */
    gl_warmstart warmstart; /* learned initial guess: when set, gl_jacobian_solve and gl_newton_step ignore the
                            x passed in, start from the network's x0 (with warmstart_hint, below), and fall
                            back to x0 = 0 when ||b - J x0||_D >= ||b||_D (default NULL: start from x as
                            given) */
    int coloring;        /* colouring of the coarse levels for the multicolour Gauss-Seidel steps:
                            GL_COLOR_PSL (smallest-last in removal rounds, on the device: each round
                            removes every vertex within 4 of the smallest remaining degree, then the
                            greedy colouring in decreasing (round, hashed id) order by Jones-Plassmann
                            rounds; default), GL_COLOR_SL (smallest-last one vertex at a time, on the
                            host) or GL_COLOR_JP (Jones-Plassmann with hashed priorities, on the
                            device).  Each colour is one dependent phase of a sweep.  The finest lattice
                            level is always red-black. */
    int sweep_sync;      /* synchronisation between the colours of a coarse-level Gauss-Seidel step:
                            0 = chosen per level (timed at setup with autotune; else the neighbour flags
                            where their partition fits), 1 = a grid-wide barrier, 2 = neighbour flags
                            (each CTA waits only for the CTAs whose rows its rows read; the grid barrier
                            where no partition fits).  The result is the same; only the time differs.
                            Every wait is bounded (1 s); one that runs out ends the call with
                            GL_ERR_TIMEOUT (default 0) */
    int coarse_df;       /* the dense coarsest product of the FP32 V-cycle (GL_MIXED, GL_MIXED_PRECOND):
                            1 = double-FP32 arithmetic (the FP64 inverse as FP32 hi + lo pairs, error-free
                            products and compensated sums, about 48 significant bits: the FP64 product's
                            value before its FP32 rounding, at the FP32 rate); 0 = FP64 arithmetic.  The
                            FP64 V-cycle always uses FP64 (default 1) */
    int device_loop;     /* 1: a solve runs as one CUDA graph whose MINRES iterations loop on the device
                            (conditional WHILE / IF nodes; no kernel after convergence, one host wait);
                            0: the same six-iteration body graph replayed by the host, which polls the
                            status word between replays (for profilers that cannot see inside
                            conditional graphs).  Solves that time a kernel class with gl_profile_begin,
                            and R_inf, always use 0 (default 1) */
    const void *warmstart_hint; /* a device vector (n complex FP64, node order) the solution is expected to
                            resemble, e.g. the same Newton step's correction at the previous mu of a
                            continuation.  With warmstart: the guess is the hint's minimal-residual
                            multiple plus the network's correction (see gl_warmstart_predict).
                            Without (warmstart NULL): gl_jacobian_solve ignores the x passed in and
                            starts from the multiple alone, alpha a with alpha = <J a, b>_R /
                            <J a, J a>_R (one FP64 Jacobian apply and three inner products; never a
                            worse guess than zero); warmstart_used reports 1 (default NULL) */
} gl_options;

#define GL_COLOR_SL 0
#define GL_COLOR_JP 1
#define GL_COLOR_PSL 2

/* Per-solve report. */
typedef struct {
    int iters;           /* MINRES iterations (summed over inner solves in GL_MIXED) */
    int outer_iters;     /* FP64 refinement steps (GL_MIXED), 1 in GL_FP64 */
    int converged;       /* 1 if true_relres <= tol */
    double true_relres;  /* ||b - J x||_D / ||b||_D computed in FP64 at the end */
    double est_relres;   /* last MINRES recurrence estimate (preconditioned norm) */
    double setup_ms;     /* preconditioner setup time inside this call (0 if a gl_prec was given) */
    double solve_ms;     /* wall time of the Krylov part */
    int warmstart_used;  /* 1 if the solve started from the learned guess, 0 if from x as given or after
                            the zero-guess fallback */
    int lattice_stencil; /* 1 if the FP32 finest-level V-cycle kernels used the closed-form stencil */
    int df_jacobian;     /* 1 if MINRES applied the Jacobian in double-FP32 arithmetic (GL_MIXED_PRECOND on
                            an even-N lattice with options.lattice = 1) */
    int stall_restarts;  /* 1 if that run stalled above tol and MINRES finished with the FP64 Jacobian */
    double matvec_equiv; /* cost in matrix-vector-product equivalents (Fig. 1): (iters + outer_iters) x
                            (1 + cost of R_k from gl_precond_cost); with R_inf, iters + outer_iters plus
                            (cycles applied) x (one V-cycle + one finest residual) */
    double cycles_per_apply; /* V-cycles per preconditioner application: k for R_k, the average for R_inf,
                            0 without a preconditioner */
    int jacobian_tables; /* 1 if MINRES's FP64 Jacobian applies ran from the lattice stencil's FP64 tables
                            (gl_options.lattice = 2 on an even-N lattice whose stored K matches them to 16
                            ulp of its largest entry) instead of the stored K */
} gl_solve_info;

/* Default options (values listed in gl_options).  Returns GL_ERR_ARG on NULL. */
GL_API gl_status gl_options_default(gl_options *opt);

/* Builds the finite-volume discretisation of Sec. 3 on the structured mesh:
 * edge coefficients alpha_jk summed over simplices (Eq. fhat; cotangent formula
 * for triangles, M alpha = b of Cor. "simplex" for tetrahedra), control volumes
 * |V_j| (Eq. mass lumping), link phases theta_jk = integral of A from x_j to x_k
 * (Eq. link variable) for A(x) = (mu/2) bhat x x (Eq. mvp0 scaled by mu, field
 * along the unit vector bhat), and K-hat with (K-hat psi)_j = sum_k alpha_jk
 * (psi_j - exp(-i theta_jk) psi_k) (Eq. discr kin energy, Remark rmk:dk).
 * Edges with |alpha| <= 1e-12 max|alpha| are dropped.
 * dim: 2 or 3.  n_per_side: N >= 2 (n = N^dim < 2^31).  bhat: 3 doubles (host),
 * normalised internally; NULL means (0,0,1).  Runs on `stream` and
 * synchronises it.  *out receives a new handle. */
GL_API gl_status gl_mesh_create(int dim, int n_per_side, double mu, const double *bhat_host, void *stream,
                         gl_mesh *out);
/* The same on the square / cube of side `edge` > 0 centred at the origin (nodes
 * -edge/2 + i h, h = edge / (N - 1)); gl_mesh_create is edge = 1.  The paper's
 * domains have edges of order 10 (Sec. 4; the continuation of Fig. 4 uses a
 * square of edge 10). */
GL_API gl_status gl_mesh_create_edge(int dim, int n_per_side, double edge, double mu, const double *bhat_host,
                                     void *stream, gl_mesh *out);
/* A general simplicial mesh (Sec. 3: any conforming Delaunay triangulation; the
 * paper's test domains of Sec. 4 are meshed this way).  x_host: n x 3 node
 * coordinates (the third ignored in 2D); simplices_host: ns x (dim + 1) node ids
 * (int32).  Per simplex the edge coefficients (the cotangent formula in 2D, the
 * linear system of the corollary in 3D) are summed per edge (Eq. fhat); edges
 * with |alpha| <= 1e-12 max |alpha| are dropped; the link phases are those of
 * A = (mu/2) bhat x x (bhat NULL: e_z; normalised) or, with dipole_x0 and
 * dipole_m, of mu A_d (8-point Gauss-Legendre along each edge); the control
 * volumes are the dual of the coefficients, |V_j| = sum_k alpha_jk
 * |x_j - x_k|^2 / (2 dim) (the Voronoi region of x_j for well-centred Delaunay
 * simplices; Eq. mass lumping).  The finest level is coloured like a coarse level
 * (round-based smallest-last) instead of red-black, and the lattice stencil is
 * off.  GL_ERR_ARG on bad ids or a degenerate simplex, GL_ERR_CAPACITY on a node
 * with more than 64 neighbours.  Synchronises `stream`. */
GL_API gl_status gl_mesh_create_simplicial(int dim, int64_t n, const double *x_host, int64_t ns,
                                           const int32_t *simplices_host, double mu, const double *bhat,
                                           const double *dipole_x0, const double *dipole_m, void *stream,
                                           gl_mesh *out);

/* The same domain in mu A_d, the field of a magnetic dipole (Sec. 4):
 * A_d(x) = m x (x - x0) / |x - x0|^3, m = mom_host, x0 = x0_host (3 doubles
 * each; the paper takes m = e_z and x0 = (0,0,1) in 2D, (0,0,6) in 3D).  The
 * link phases are integrals of A_d along each edge by an 8-point
 * Gauss-Legendre rule (A_d is not polynomial; the quadrature remark after Eq.
 * link variable); they vary along every axis, so the lattice-table stencil is
 * not used on such meshes.  x0 must lie outside the closed domain.
 * gl_mesh_set_mu scales A_d by the new mu. */
GL_API gl_status gl_mesh_create_dipole(int dim, int n_per_side, double edge, double mu, const double *x0_host,
                                       const double *mom_host, void *stream, gl_mesh *out);
GL_API gl_status gl_mesh_destroy(gl_mesh mesh);

/* Changes the field strength of A = (mu/2) bhat x x in place: only the link
 * phases depend on mu (theta_jk = mu theta1_jk, Eq. link variable), so every
 * stored K-hat entry becomes -alpha_jk exp(-i mu theta1_jk), and K, its FP32
 * copy and the lattice tables are rewritten into the same buffers.  The sparsity,
 * ordering, volumes and the diagonal stay.  A preconditioner set up before the
 * call no longer matches the operator: using it afterwards returns GL_ERR_ARG.
 * (Entries may differ from a mesh created at that mu in the last bit: the phase
 * is formed as mu * theta1.)  Synchronises `stream`. */
GL_API gl_status gl_mesh_set_mu(gl_mesh mesh, double mu, void *stream);

/* n = number of nodes; nnz = stored entries of K-hat (diagonal included);
 * volumes_dev (nullable): receives |V_j| as n doubles.  Synchronises `stream`
 * only when volumes_dev is given (copy on the legacy stream). */
GL_API gl_status gl_mesh_info(gl_mesh mesh, int64_t *n, int64_t *nnz, double *volumes_dev);

/* Discrete GL residual (Eq. discr ginla): r_i = (K psi)_i - psi_i (1 - |psi_i|^2),
 * K = D^-1 K-hat.  psi_dev, r_dev: n complex (FP64); may not alias. */
GL_API gl_status gl_residual(gl_mesh mesh, const void *psi_dev, void *r_dev, void *stream);

/* d GL / d mu at fixed psi (the parameter derivative that pseudo-arclength
 * continuation in mu needs, Sec. 4): only K depends on mu, through the phases,
 * so out = D^-1 (d K-hat / d mu) psi with (d K-hat / d mu)_jk =
 * -i theta1_jk K-hat_jk off the diagonal and 0 on it.  psi_dev, out_dev: n
 * complex FP64, may not alias. */
GL_API gl_status gl_residual_dmu(gl_mesh mesh, const void *psi_dev, void *out_dev, void *stream);

/* Discrete energy (Eq. discr energy): F = F_1 + F_2 with
 * F_1 = sum_edges alpha_jk |psi_j - exp(-i theta_jk) psi_k|^2 = Re psi^H K-hat psi
 * and F_2 = sum_i |V_i| (-|psi_i|^2 + |psi_i|^4 / 2) (Eq. mass lumping).
 * *energy_host = F (FP64 sums).  Synchronises `stream`. */
GL_API gl_status gl_energy(gl_mesh mesh, const void *psi_dev, double *energy_host, void *stream);

/* Discrete Jacobian (Sec. 3):
 *   y_i = (K phi)_i + (-1 + 2|psi_i|^2) phi_i + psi_i^2 conj(phi_i).
 * psi, phi, y: n complex FP64; y may not alias psi or phi.  GL_FP64: the stored
 * K.  GL_APPLY_FP64_TABLES: the same operator formed matrix-free from the lattice
 * stencil's FP64 tables (meshes with an even number of nodes per side whose
 * stored K matches the tables to 16 ulp of its largest entry; GL_ERR_ARG on
 * others).  With GL_MIXED the operator and arithmetic are FP32 (inputs rounded
 * to FP32, output widened).
 * With GL_MIXED_PRECOND: the double-FP32 form that GL_MIXED_PRECOND solves use on
 * meshes with an even number of nodes per side (edge magnitudes and phases of
 * the checked lattice stencil as FP32 hi + lo pairs, error-free transformations,
 * about 48 significant bits) applied to phi rounded to FP32 (in the solve the
 * vectors it meets are FP32 values, so there the rounding is exact); y in FP64.
 * GL_ERR_ARG on a mesh without that stencil (odd N).  Synchronises `stream`. */
GL_API gl_status gl_jacobian_apply(gl_mesh mesh, const void *psi_dev, const void *phi_dev, void *y_dev,
                            int precision, void *stream);

/* The same Jacobian apply (FP64) as gl_jacobian_apply, for callers that cannot
 * let the library allocate device memory during the call: applications with a
 * fixed device-memory budget or their own pool (an allocation behind their back
 * can fail or fragment it), and latency-critical loops (cudaMalloc/cudaFree may
 * synchronise the device).  The paper has no counterpart; this is an interface
 * convenience.
 * It allocates nothing: its working buffers live in one static device array of
 * GL_NOALLOC_MAX_NODES = 262144 nodes x 3 complex doubles (12 MiB) that every
 * GPU loading the library holds until exit.  Meshes with more nodes are rejected
 * with GL_ERR_CAPACITY.  All calls on a device share that array (it keeps the
 * last call's contents; nothing needs to start at zero), so calls whose work
 * overlaps on the GPU race.  The first call on each device looks up the array's
 * device address with that device current; that first call should come before
 * any stream capture.
 * Arguments and layouts as gl_jacobian_apply. */
GL_API gl_status gl_jacobian_apply_noalloc(gl_mesh mesh, const void *psi_dev, const void *phi_dev, void *y_dev,
                                           void *stream);

/* Sets up R_k(psi) = AMG_k(K-hat + 2 D |psi|^2, D .) (Eq. prec2, Sec. 4.1):
 * smoothed-aggregation AMG with symmetric Gauss-Seidel smoothing.  Uses
 * opt->cycles, max_coarse, max_levels, power_its, precision (GL_MIXED also
 * builds FP32 copies of every level).  Synchronises `stream`. */
GL_API gl_status gl_precond_setup(gl_mesh mesh, const void *psi_dev, const gl_options *opt, void *stream,
                           gl_prec *out);

/* gl_precond_setup for a new psi (and the mesh's current mu) that takes over
 * from `like`, an earlier preconditioner of the same mesh set up with the same
 * max_coarse, max_levels and coloring, everything that depends on the sparsity
 * alone: the aggregates (strength threshold 0), the colourings and the kernel
 * choices its setup timed.  The hierarchy's values are computed afresh, so the
 * result equals a gl_precond_setup whose timing picked the same kernels; along
 * a continuation the sparsity never changes.  A `like` that does not match is
 * ignored (a full setup runs).  `like` stays valid and owned by the caller. */
GL_API gl_status gl_precond_setup_like(gl_mesh mesh, const void *psi_dev, const gl_options *opt, gl_prec like,
                                       void *stream, gl_prec *out);

/* z = R_k x: k V-cycles for (K-hat + 2 D|psi|^2) z = D x from z = 0 (Eq. prec2);
 * with cycles = GL_CYCLES_INF, R_inf: cycles until the residual test of
 * GL_CYCLES_INF holds (a device-side loop; no host round trip per cycle).
 * x_dev, z_dev: n complex FP64, may not alias.  FP64 arithmetic.  Synchronises
 * `stream` to read the coarse sweeps' error word: GL_ERR_TIMEOUT if one of their
 * bounded waits ran out (z is then not R x; the synchronisation state is reset,
 * so the next call runs normally). */
GL_API gl_status gl_precond_apply(gl_prec prec, const void *x_dev, void *z_dev, void *stream);

/* gl_precond_apply with the V-cycle in a chosen arithmetic: GL_FP64 as
 * gl_precond_apply; GL_MIXED or GL_MIXED_PRECOND the FP32 V-cycle those solves
 * run (x rounded to FP32 on entry, FP32 level operators and sweeps, the lattice
 * stencil on the finest level where options.lattice allows it, the coarsest
 * solve in FP64, z widened to FP64).  Builds the FP32 copies on first use.
 * Errors as gl_precond_apply; GL_ERR_ARG for R_inf in FP32. */
GL_API gl_status gl_precond_apply_precision(gl_prec prec, const void *x_dev, void *z_dev, int precision,
                                            void *stream);

/* Fault injection for tests of the failure handling; no counterpart in the
 * paper.  GL_DEBUG_STALL_SWEEPS: every wait of the next coarse-level sweeps
 * waits for a count that no CTA reaches, so it runs out after its 1 s bound,
 * the call that ran it returns GL_ERR_TIMEOUT and resets the state (later calls
 * run normally).  GL_DEBUG_NEGATE_COARSEST: multiplies the coarsest level's
 * dense inverse by -1, which makes R_k indefinite on a one-level hierarchy
 * (solves then end with GL_ERR_BREAKDOWN); permanent for this handle.
 * Synchronises the device. */
#define GL_DEBUG_STALL_SWEEPS 1
#define GL_DEBUG_NEGATE_COARSEST 2
GL_API gl_status gl_precond_debug(gl_prec prec, int action);
GL_API gl_status gl_precond_destroy(gl_prec prec);

/* Cost of applying R_k (k = cycles >= 1) in matrix-vector-product equivalents,
 * the measure of Fig. 1: matrix entries visited by k V-cycles and the k - 1
 * finest-level residuals between them, divided by the entries of K-hat.  A
 * V-cycle visits, per level, both symmetric Gauss-Seidel steps (a colour visit
 * reads its rows' off-diagonals and diagonals; from the zero guess the first
 * colour reads only diagonals; the backward pass skips the repeated last
 * colour), the residual, the restriction and the prolongation (nnz(P) each), and
 * n_c^2 entries of the dense coarsest inverse.  Host result; no GPU work. */
GL_API gl_status gl_precond_cost(gl_prec prec, int cycles, double *matvecs);

/* Hierarchy introspection (for parity checks).  Level 0 is the finest.
 * Node numbering is the canonical one: the mesh's node ids on level 0 and the
 * aggregate ids (roots in ascending id order) below.  Host outputs. */
GL_API gl_status gl_precond_levels(gl_prec prec, int *nlevels);
GL_API gl_status gl_precond_level_info(gl_prec prec, int level, int64_t *n, int64_t *nnz, int32_t *ncolors,
                                int64_t *p_nnz, double *omega);
/* How level l's Gauss-Seidel steps run in the given precision's V-cycle
 * (GL_FP64, or GL_MIXED / GL_MIXED_PRECOND for the FP32 V-cycle once built):
 * *lanes = lanes per row, *sync = 0 for a cooperative grid with a grid
 * barrier between colours, 1 for neighbour flags (*ctas = CTAs of the launch),
 * 3 for one thread-block cluster (*ctas = its size); 0 / -1 / 0 on the lattice
 * and the coarsest level, which have no such sweep.  Any output may be NULL. */
GL_API gl_status gl_precond_level_sweep(gl_prec prec, int level, int precision, int *lanes, int *sync, int *ctas);

/* agg_host: n int32, the coarse node of each node of this level (not the coarsest). */
GL_API gl_status gl_precond_level_aggregates(gl_prec prec, int level, int32_t *agg_host);
/* color_host: n int32 smoothing colours of this level. */
GL_API gl_status gl_precond_level_colors(gl_prec prec, int level, int32_t *color_host);
/* CSR of the level operator (Hermitian; level 0 = K-hat + 2 D|psi|^2), columns
 * ascending: rp_host n+1 int64, ci_host nnz int32, v_host nnz complex FP64. */
GL_API gl_status gl_precond_level_matrix(gl_prec prec, int level, int64_t *rp_host, int32_t *ci_host, void *v_host);
/* CSR of the prolongator from level+1 to level: n rows, p_nnz entries. */
GL_API gl_status gl_precond_level_P(gl_prec prec, int level, int64_t *rp_host, int32_t *ci_host, void *v_host);

/* Mesh introspection (host outputs): edges (j < k) in lexicographic order with
 * alpha and theta; and K-hat as CSR with ascending columns. */
GL_API gl_status gl_mesh_nedges(gl_mesh mesh, int64_t *nedges);
GL_API gl_status gl_mesh_edges(gl_mesh mesh, int32_t *ej_host, int32_t *ek_host, double *alpha_host,
                        double *theta_host);
GL_API gl_status gl_mesh_khat(gl_mesh mesh, int64_t *rp_host, int32_t *ci_host, void *v_host);

/* Solves J(psi) x = b (the Newton system, Eq. Newton system) by preconditioned
 * MINRES in <.,.>_R = Re sum |V_i| conj(x_i) y_i (Sec. 4, Eq. disc inner2) with
 * preconditioner R_k(psi).  prec: a handle set up for the same psi, or NULL to
 * set one up inside the call (timed in info->setup_ms).  x_dev: on entry the
 * initial guess (zeros for x0 = 0), on exit the solution.  The iteration stops
 * once the recurrence estimate and then the FP64 true residual
 * ||b - J x||_D / ||b||_D are both <= opt->tol.  GL_MIXED: FP64 defect
 * correction around FP32 inner MINRES solves.  Returns GL_ERR_NOT_CONVERGED at
 * the iteration cap with x the last iterate.  Synchronises `stream`. */
GL_API gl_status gl_jacobian_solve(gl_mesh mesh, const void *psi_dev, gl_prec prec, const void *b_dev, void *x_dev,
                            const gl_options *opt, gl_solve_info *info, void *stream);

/* One Newton step (Eq. Newton system): r = GL(psi), solve J(psi) d = -r with
 * R_k(psi), psi <- psi + d.  *gl_norm_out (nullable) = ||GL(psi)||_R of the
 * state on entry.  Synchronises `stream`. */
GL_API gl_status gl_newton_step(gl_mesh mesh, void *psi_dev, const gl_options *opt, gl_solve_info *info,
                         double *gl_norm_out, void *stream);

/* Many independent Newton systems at once (the continuation setting of Sec. 4,
 * where each step needs a Jacobian solve).  gl_batch_create sets up R_1(psi_s)
 * for every instance (meshes of any sizes; psi_dev[s] has that mesh's n complex
 * FP64 values).  gl_batch_run solves J(psi_s) x_s = b_s for all instances in ONE
 * CUDA-graph launch: every instance is a branch of the graph and iterates inside
 * a device-side WHILE conditional node until its own stopping test holds (same
 * test as gl_jacobian_solve); x_dev[s] holds the initial guess on entry.  With
 * precision GL_MIXED or GL_MIXED_PRECOND the V-cycles run in FP32 inside FP64
 * MINRES, and instances on lattice meshes with the checked stencil (even N) apply
 * J in double-FP32 arithmetic as gl_jacobian_solve does; an instance whose true
 * residual that ~48-bit apply holds above tol continues after the graph from its
 * x with the FP64 Jacobian (infos[s].stall_restarts = 1).  The graph is built on
 * the first run and rebuilt when the b/x pointers
 * change.  infos (nullable): count entries.  Returns the first non-GL_OK status.
 * Synchronises `stream`. */
GL_API gl_status gl_batch_create(int count, const gl_mesh *meshes, const void *const *psi_dev, const gl_options *opt,
                                 void *stream, gl_batch *out);
GL_API gl_status gl_batch_run(gl_batch batch, const void *const *b_dev, void *const *x_dev, gl_solve_info *infos,
                              void *stream);
GL_API gl_status gl_batch_destroy(gl_batch batch);

/* gl_batch_create + gl_batch_run + gl_batch_destroy in one call. */
GL_API gl_status gl_batch_solve(int count, const gl_mesh *meshes, const void *const *psi_dev, const void *const *b_dev,
                                void *const *x_dev, const gl_options *opt, gl_solve_info *infos, void *stream);

/* Measured arithmetic peak of the current GPU for the rooflines (not a paper
 * quantity): fused multiply-adds of independent chains on every SM, timed with
 * CUDA events; precision GL_FP64 for FP64, GL_MIXED for FP32.  *gflops_host =
 * GFLOP/s (2 per FMA), the best of repetitions grown to >= 20 ms.  Synchronises
 * `stream`. */
GL_API gl_status gl_measure_fma_peak(int precision, double *gflops_host, void *stream);

/* Measured latencies that bound one phase of the coarse-level Gauss-Seidel
 * sweeps (not a paper quantity), in ns, into ns4_host[4]: [0] the median and
 * [1] the largest one-way hand-off between CTA 0 and every other SM's CTA (a
 * release store seen by an acquiring poll, 200 round trips per pair); [2] one
 * dependent L2 load (__ldcg along a 1 MiB chain); [3] a store followed by a
 * GPU-scope fence.  Every wait is bounded (1 s; GL_ERR_TIMEOUT).  Synchronises
 * `stream`. */
GL_API gl_status gl_measure_sync_latency(double *ns4_host, void *stream);

/* Measurement instrumentation (no counterpart in the paper).
 * gl_profile_begin resets the count of hot-path kernel launches and, when
 * kernel_class is not NULL, records a pair of CUDA events on the launching
 * stream around each of the next max_launches launches of that class:
 *   "gs0"  Gauss-Seidel colour sweeps on the finest level (byte model: per row
 *          the diagonal, b and the written x; the stored off-diagonals as value +
 *          32-bit column; each neighbour value once)
 *   "jz"   the fused Jacobian apply + dot of MINRES (byte model: stored
 *          off-diagonals, K_ii, |V|, psi, z and the written result per row)
 *   "gs", "resid0", "resid", "restrict", "prolong" (timed, no byte model).
 * gl_profile_end synchronises the device and returns the launches since
 * begin, the number of timed launches, their summed duration in ms and their
 * summed algorithmic bytes.  Not thread-safe; one profile at a time. */
GL_API gl_status gl_profile_begin(const char *kernel_class, int max_launches);
GL_API gl_status gl_profile_end(int64_t *launches, int64_t *timed, double *total_ms, double *alg_bytes);
/* Arithmetic of the launches timed by the last gl_profile_begin / gl_profile_end
 * pair, for the classes whose kernels may be bound by an arithmetic pipe (the
 * FP64 Jacobian, the FP64 sweeps, the double-FP32 Jacobian: flops, an FMA or
 * an FP32 operation of an error-free transformation counted as 2); 0 for
 * other classes.  Host output. */
GL_API gl_status gl_profile_flops(double *alg_flops_host);

/* ---------------------------------------------------------------------------
 * Learned warm start.  The paper has no counterpart: its Newton-Krylov solves
 * start from x0 = 0 (Sec. 4).  The network predicts the initial guess of the
 * solve of J(psi) x = b (Eq. (16)) as
 *     x0 = ||b||_D * y(psi, b / ||b||_D) / K_ii,    ||b||_D^2 = sum_i |V_i| |b_i|^2,
 * with y a 4-layer, 64-channel graph network whose aggregation is the magnetic
 * Jacobi operator S = I - diag(K)^-1 K of Eq. (10) (edge weights and phases,
 * normalised per row), relu activations, channel 63 held at 1 (biases), and a
 * 2 x 64 linear head.  Its dense layers run as BF16 tensor-core MMAs with FP32
 * accumulation; activations are BF16.  Training minimises the squared relative
 * true-Jacobian residual ||b - J x0||_D^2 / ||b||_D^2 with Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8).  All vectors are n complex FP64 in node order on the
 * device; every call runs on `stream` and synchronises it.
 * ------------------------------------------------------------------------- */

/* New network with the given parameters (host, GL_WS_NPARAM floats; NULL =
 * zeros).  The handle owns its parameters, Adam moments and work buffers
 * (about 900 bytes per mesh node of the largest mesh it has seen). */
GL_API gl_status gl_warmstart_create(const float *params_host, gl_warmstart *out);
GL_API gl_status gl_warmstart_destroy(gl_warmstart ws);
/* Copy the FP32 parameters out / in (set also resets the Adam state). */
GL_API gl_status gl_warmstart_get_params(gl_warmstart ws, float *params_host);
GL_API gl_status gl_warmstart_set_params(gl_warmstart ws, const float *params_host);
/* x0 = network guess for (psi, b); x0_dev must not alias psi or b.  hint_dev
 * (nullable, n complex FP64, node order): a vector the solution is expected to
 * resemble; the guess is then
 *     x0 = alpha a + ||r||_D y(psi, r / ||r||_D, a / ||a||_D) / K_ii,
 *     alpha = <J a, b>_R / <J a, J a>_R (0 when J a = 0),   r = b - alpha J a,
 * alpha the multiple of the hint with the smallest ||b - J alpha a||_D (FP64), and
 * the normalised hint the network's input channel pair (6, 7). */
GL_API gl_status gl_warmstart_predict(gl_warmstart ws, gl_mesh mesh, const void *psi_dev, const void *b_dev,
                                      const void *hint_dev, void *x0_dev, void *stream);
/* Loss ||r^ - J x^||_D^2 of one sample (r = b without a hint) and its gradient
 * (host, GL_WS_NPARAM floats, nullable) with respect to the parameters. */
GL_API gl_status gl_warmstart_grad(gl_warmstart ws, gl_mesh mesh, const void *psi_dev, const void *b_dev,
                                   const void *hint_dev, float *grad_host, double *loss_out, void *stream);
/* `steps` Adam steps with learning rate lr; step t averages the losses and
 * gradients of samples (t * batch + j) mod count, j < batch.  Sample k is
 * (meshes[k], psi_dev[k], b_dev[k], hint_dev[k]); meshes may differ between
 * samples; hint_dev (nullable array, nullable entries) gives the hints.
 * loss_out (host, nullable) receives the mean loss of every step. */
GL_API gl_status gl_warmstart_train(gl_warmstart ws, int count, const gl_mesh *meshes, const void *const *psi_dev,
                                    const void *const *b_dev, const void *const *hint_dev, int steps, int batch,
                                    float lr, double *loss_out, void *stream);
/* One Adam step with the given gradient (host, GL_WS_NPARAM floats). */
GL_API gl_status gl_warmstart_adam_step(gl_warmstart ws, const float *grad_host, float lr);

/* ---------------------------------------------------------------------------
 * Pseudo-arclength parameter continuation in mu (Sec. 4, "Numerical parameter
 * continuation"): a predictor-corrector in (psi, mu) whose corrector is the
 * Newton-Krylov process of this library.
 *   metric:     ||(phi, nu)||^2 = <phi, phi>_R / |Omega| + nu^2 (Eq. disc inner2);
 *   start:      Newton at the mesh's mu; first tangent (c, 1) / norm with
 *               J c = -dGL/dmu (increasing mu); later tangents are secants;
 *   predictor:  (psi, mu) + ds t;
 *   corrector:  Newton on GL(psi, mu) = 0 and <t_psi, psi - psi_s>_R / |Omega|
 *               + t_mu (mu - mu_s) = ds, each step solving J a = -GL and
 *               J c = -dGL/dmu with one R_k(psi) and eliminating the border:
 *               dmu = (-n - <t_psi, a>) / (t_mu + <t_psi, c>), dpsi = a + dmu c;
 *               converged when ||GL||_R / sqrt|Omega| <= newton_tol;
 *   step size:  halved (same point) when Newton fails; after a step that took
 *               <= 2 Newton steps ds grows 1.5x (<= ds_max), >= 5 shrinks 0.7x.
 * ------------------------------------------------------------------------- */
typedef struct {
    double ds, ds_min, ds_max; /* arclength step: start, bounds (defaults 0.05, 1e-4, 0.2) */
    double mu_max;             /* stop once mu >= mu_max (default 1) */
    int max_steps;             /* accepted steps at most (default 100) */
    double newton_tol;         /* ||GL||_R / sqrt|Omega| target (default 1e-9) */
    int newton_maxit;          /* Newton steps per point before ds is halved (default 8) */
    gl_options solver;         /* the Jacobian solves (default: gl_options_default with tol 1e-8, the
                                  paper's continuation tolerance); cycles >= 1 */
} gl_cont_options;

typedef struct {
    double mu;           /* field strength of the point */
    double energy;       /* F / |Omega| (Eq. discr energy per unit volume; -1/2 for psi = 1, mu = 0) */
    double gl_norm;      /* ||GL(psi)||_R / sqrt|Omega| at acceptance */
    double ds;           /* arclength step that produced the point (0 for the start) */
    int newton_steps;    /* Newton steps of the point */
    int iters_last;      /* MINRES iterations of the last Newton step's J a = -GL solve (Fig. 4, right) */
    int iters_total;     /* all MINRES iterations of the point (both solves, retries included) */
    int retries;         /* step halvings before the point was accepted */
    double setup_ms;     /* preconditioner setups of the point */
    double solve_ms;     /* Jacobian solves of the point */
} gl_cont_point;

GL_API gl_status gl_cont_options_default(gl_cont_options *opt);

/* Runs the continuation from (psi_dev, the mesh's mu).  psi_dev: n complex FP64
 * in node order, in: the start state, out: the last accepted state; the mesh is
 * left at that state's mu (gl_mesh_set_mu).  points_host: room for max_points
 * entries; *npoints_out = points written (the start is the first).
 * states_dev (nullable): max_points device pointers, each n complex FP64,
 * receiving psi of every point.  Stops at mu >= mu_max, max_steps, a full
 * points array, or ds < ds_min (then GL_ERR_NOT_CONVERGED with the points so
 * far).  Synchronises `stream`. */
GL_API gl_status gl_continuation(gl_mesh mesh, void *psi_dev, const gl_cont_options *opt, gl_cont_point *points_host,
                                 int max_points, int *npoints_out, void *const *states_dev, void *stream);

/* Message describing the last failure on this host thread ("" if none). */
GL_API const char *gl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GL_GB300_H */
