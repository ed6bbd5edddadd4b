// gl_internal.cuh -- handle layouts of gl_mesh / gl_prec and the internal entry
// points shared between the translation units of the library.
#pragma once

#include "gl_common.cuh"

struct gl_mesh_s {
    int dim = 0, N = 0;
    int64_t n = 0;
    double h = 0, mu = 0, bhat[3] = {0, 0, 1};
    double edge = 1;                      // side of the square / cube
    int dipole = 0;                       // 1: A = mu A_d (dipole field) instead of (mu/2) bhat x x
    int64_t version = 0;                  // bumped by every change of mu (gl_mesh_set_mu)
    // canonical (node-order) data
    gl::CsrDev khat;                      // K-hat, columns ascending
    gl::DBuf<double> vol;                 // |V_j|
    int64_t nedges = 0;
    gl::DBuf<int32_t> ej, ek;             // edges j < k, lexicographic
    gl::DBuf<double> ealpha, etheta, etheta1;  // etheta1: phase per unit mu
    gl::DBuf<double> kal, kth1;           // per stored K-hat entry: alpha and phase per unit mu (0 on the diagonal)
    gl::DBuf<int32_t> color0;             // finest-level colour of each node (red-black on a lattice)
    // solve ordering: position p holds node perm[p]; red nodes occupy [0, nred);
    // colour c occupies [cstart0[c], cstart0[c + 1]) (ncolors0 colours: 2 on a
    // lattice, more on a general simplicial mesh)
    int64_t nred = 0;
    int ncolors0 = 2;
    std::vector<int64_t> cstart0;
    gl::DBuf<int32_t> perm, iperm;
    gl::Sell<double2> K;                  // off-diagonals of K = D^-1 K-hat (solve ordering)
    gl::DBuf<double> kdiag, volp;         // K_ii and |V_i| (solve ordering)
    bool has32 = false;
    gl::Sell<float2> K32;
    gl::DBuf<float> kdiag32, volp32;
    // closed-form finest-level stencil (gl_lattice.cu): phase tables per axis
    bool lat_checked = false, lat_ok = false;
    int64_t lat_per_axis = 0;
    gl::DBuf<float2> lat_tab;
    // the FP64 tables, used by the FP64 Jacobian when every stored entry of K
    // matches them to 16 ulp of the largest entry (lat64_ok)
    bool lat64_ok = false;
    gl::DBuf<double2> lat_tab64;
    // the same tables as double-float magnitude a = |K-hat| / h^d and unit phase,
    // the FP64 remainders K_ii - sum_k |K_ik| (solve ordering) and h^d
    gl::DBuf<float2> lat_a;
    gl::DBuf<float4> lat_u;
    gl::DBuf<double> lat_krem;
    double lat_hd = 0;
    // scratch for the node-order public calls
    gl::DBuf<double2> t0, t1, t2;
};

namespace gl {

constexpr int MAX_LEVELS = 16;
// grid-barrier state of a level's cooperative sweeps: one 64-bit arrival
// counter for the FP32 and one for the FP64 sweep
constexpr int GRID_BARRIER_WORDS = 4;
constexpr int MAX_COARSE_DENSE = 4096;
// neighbour-flag form of the coarse sweeps: one completed-phase counter per
// CTA, FLAG_STRIDE 64-bit words apart, at most MAX_FLAG_CTAS CTAs per launch,
// and at most FLAG_MAXN neighbour CTAs per (CTA, colour)
constexpr int FLAG_STRIDE = 16;
constexpr int MAX_FLAG_CTAS = 1024;
constexpr int FLAG_MAXN = 32;
// status word value a bounded device-side wait writes when it runs out
constexpr int STATUS_TIMEOUT = 6;
// bound of every device-side wait of the coarse sweeps (globaltimer ns)
constexpr long long SWEEP_WAIT_NS = 1000000000ll;

// Partition and dependency lists of the neighbour-flag sweep of one level in one
// precision: CTA b owns chunk b of nb equal contiguous chunks of every colour's
// positions (ascending node ids within a colour, so chunk b of every colour lies
// in about the same part of the level); before a phase it waits only for the
// CTAs owning columns of its rows in that phase's colour.
struct FlagPlan {
    int nb = 0;                  // CTAs of the launch (0: no plan)
    int G = 0;                   // lanes per row the plan was built for
    DBuf<int64_t> rstart;        // [colour][nb + 1]: first solve position of each CTA's rows in the colour
    DBuf<int32_t> nbr;           // [cta][colour][FLAG_MAXN]: CTAs whose rows those rows read
    DBuf<int32_t> nbrc;          // [cta][colour]: lengths of those lists
    // the row pointers of each CTA's rows, colour after colour (each colour's
    // rows and their end), which the sweep keeps in shared memory: CTA b's list
    // starts at rbase[b]; its colour c part at roff[b (nc + 1) + c]
    DBuf<int64_t> rpl, rbase;
    DBuf<int32_t> roff;
    int smem = 0;                // dynamic shared memory of the launch (bytes)
};
// what the sweep kernel reads of a FlagPlan
struct FlagView {
    const int64_t *rstart;
    const int32_t *nbr, *nbrc;
    const int64_t *rpl, *rbase;
    const int32_t *roff;
};
inline FlagView flag_view(const FlagPlan &F) {
    return FlagView{F.rstart.get(), F.nbr.get(), F.nbrc.get(), F.rpl.get(), F.rbase.get(), F.roff.get()};
}
constexpr int FLAG_SMEM_MAX = 40 * 1024;  // bound of a plan's shared-memory row pointers (bytes; with the
                                          // kernel's static shared memory below the 48 KiB default)

struct Level {
    int64_t n = 0;
    int ncolors = 0;
    std::vector<int64_t> cstart;    // colour c occupies solve positions [cstart[c], cstart[c+1])
    std::vector<int64_t> cnnz;      // stored off-diagonals of the rows of each colour
    // canonical numbering
    CsrDev A_can;                   // Hermitian level operator (level 0: K-hat + 2 D |psi|^2)
    DBuf<int32_t> agg;              // coarse node of each node (not on the coarsest level)
    DBuf<int32_t> color;
    DBuf<double> B;                 // near-null candidate
    CsrDev P_can;                   // prolongator from level + 1
    double rho = 0, omega = 0;
    // solve ordering (colour-major)
    DBuf<int32_t> perm_own, iperm_own;  // coarse levels own theirs; level 0 uses the mesh's
    const int32_t *perm = nullptr, *iperm = nullptr;
    Sell<double2> A_own;            // coarse levels: off-diagonals of A
    const Sell<double2> *A = nullptr;  // level 0 points at the mesh's K (row-scaled)
    DBuf<double> diag;              // level 0: K_ii + 2|psi_i|^2; else A_ii
    Sell<double2> P, PH;            // permuted prolongator / its adjoint
    CsrG<double2> Ag, PHg;          // grouped-CSR forms: coarse-level A (ell >= 1) and P^H
    DBuf<int64_t> cstart_dev;       // cstart on the device (cooperative sweeps)
    DBuf<unsigned> barrier;         // grid-barrier state of the cooperative coarse sweeps
    DBuf<unsigned long long> flags; // neighbour-flag sweeps: [precision][MAX_FLAG_CTAS][FLAG_STRIDE] counters
    FlagPlan fl32, fl64;            // their partitions (FP32 / FP64 sweep)
    int sync32 = 0, sync64 = 0;     // coarse sweep synchronisation: 0 grid barrier, 1 neighbour flags
    DBuf<double2> b, x, r;          // level vectors (solve ordering)
    DBuf<double2> Ainv;             // coarsest: dense inverse, row-major
    // FP32 copies (mixed precision)
    Sell<float2> A32_own;
    const Sell<float2> *A32 = nullptr;
    DBuf<float> diag32;
    Sell<float2> P32, PH32;
    CsrG<float2> Ag32, PHg32;
    CsrG<float2> PHg32b;            // level 0 with two colours: P^H without the colour-0 columns
    DBuf<float2> b32, x32, r32;
    DBuf<float4> Ainv_df;           // coarsest: the dense inverse as double-FP32 (re hi, re lo, im hi, im lo)
    int cl_size = 0, cl_chunk = 0;  // FP32 sweeps by one thread-block cluster (0: cooperative grid)
    int sgs_G32 = 1, sgs_G64 = 1;   // lanes per row of the coarse Gauss-Seidel sweeps
};

// R_inf (Eq. prec1): V-cycles until the scaled residual is RINF_TOL of the input
constexpr int CYCLES_INF = -1;
constexpr double RINF_TOL = 1e-12;
constexpr int RINF_MAXCYC = 200;
struct RinfDev {
    double v2;                     // ||v||_D^2 of the current application
    unsigned long long cycles;     // V-cycles applied since the last reset
    unsigned long long applies;    // applications since the last reset
    int k;                         // cycles of the current application
    int hit_max;                   // an application stopped at RINF_MAXCYC above the tolerance
};

}  // namespace gl

struct gl_prec_s {
    ~gl_prec_s();
    int64_t uid = 0;                  // unique per handle (keys cached CUDA graphs)
    gl_mesh_s *mesh = nullptr;
    int64_t mesh_version = 0;         // the mesh's version (mu) the operator was built for
    gl::DBuf<int> err;                // set by a device-side wait that ran out
    gl::DBuf<unsigned long long> wait_extra;  // added to every sweep wait target: 0, or huge after
                                      // gl_precond_debug(GL_DEBUG_STALL_SWEEPS) (reset with the error word)
    int nlev = 0;
    int cycles = 1;
    bool has32 = false;
    bool autotune = true;
    bool lattice = true;              // closed-form finest-level stencil in the FP32 V-cycle when available
    bool lattice64 = false;           // and MINRES's FP64 Jacobian from its FP64 tables (options.lattice = 2)
    bool cluster_sweeps = true;       // FP32 coarse sweeps by one thread-block cluster when the level fits
    gl::Level L[gl::MAX_LEVELS];
    gl::DBuf<double2> psi_p;          // psi in solve ordering
    gl::DBuf<double2> cyc_r, cyc_e;   // work vectors for k > 1 cycles
    gl::DBuf<float2> cyc_r32, cyc_e32;
    gl::DBuf<float2> mp_in, mp_out;   // FP32 V-cycle input/output inside FP64 MINRES
    gl::DBuf<double2> coarse_b64, coarse_x64;  // FP64 coarsest solve in mixed mode
    // cost model (matrix entries visited): one V-cycle, and the finest operator K-hat
    double cost_vcycle = 0, cost_fine = 0;
    // the hierarchy-shaping options the setup ran with (a template must match them)
    int64_t max_coarse_used = 0;
    int maxlev_used = 0, coloring_used = 0;
    // kernel choices taken over from a template instead of timing them again
    struct Tuned {
        int ag64 = 1, phg64 = 1, sgs64 = 1, ag32 = 1, phg32 = 1, sgs32 = 1, cl_size = 0, cl_chunk = 0;
        int sync64 = 0, nb64 = 0, sync32 = 0, nb32 = 0;
    } tuned[gl::MAX_LEVELS];
    int sweep_sync = 0;               // gl_options.sweep_sync the setup ran with
    bool coarse_df = true;            // FP32 V-cycle: double-FP32 coarsest product (else FP64)
    bool tuned64 = false, tuned32 = false;
    // R_inf: device loop state, the stream its loop body is captured on, and the
    // stream and events of an application outside stream capture
    bool rinf = false;
    gl::DBuf<double> rinf_part;
    gl::DBuf<gl::RinfDev> rinf_dev;
    cudaStream_t rinf_body = nullptr, rinf_eager = nullptr;
    cudaEvent_t rinf_ev[2] = {nullptr, nullptr};
};

namespace gl {

// gl_mesh.cu
// dip_x0, dip_m (both or neither): A = mu A_d, the field of a dipole of moment dip_m at dip_x0
void mesh_create(gl_mesh_s *m, int dim, int N, double edge, double mu, const double *bhat, cudaStream_t s,
                 const double *dip_x0 = nullptr, const double *dip_m = nullptr);
// new field strength: rewrites every phase-dependent value in place (K-hat, K, the
// FP32 copy and the lattice tables); bumps m->version
void mesh_set_mu(gl_mesh_s *m, double mu, cudaStream_t s);
// a general simplicial mesh from host arrays (gl_mesh.cu)
void mesh_create_simplicial(gl_mesh_s *m, int dim, int64_t n, const double *xyz_host, int64_t ns,
                            const int32_t *simp_host, double mu, const double *bhat, const double *dip_x0,
                            const double *dip_m, cudaStream_t s);
// round-based smallest-last colouring of a graph (gl_setup.cu); returns the colour count
int colour_graph_psl(const CsrDev &A, int32_t *color, cudaStream_t s);
void mesh_ensure_fp32(gl_mesh_s *m, cudaStream_t s);
template <typename C>
void build_sell(int64_t nrows, int64_t ncols, const int32_t *perm, const int32_t *icol, const CsrDev &A,
                const double *row_scale, bool drop_diag, Sell<C> &out, double *diag_out, cudaStream_t s);
void to_float(const double *in, float *out, int64_t n, cudaStream_t s);
// grouped CSR of A's rows perm[0..nrows) with columns mapped by icol; columns
// (after the map) below col_lo are left out
template <typename C>
void build_csrg(int64_t nrows, const int32_t *perm, const int32_t *icol, const CsrDev &A, bool drop_diag,
                CsrG<C> &out, double *diag_out, cudaStream_t s, int64_t col_lo = 0);

// gl_lattice.cu: validates the closed-form finest-level stencil against the
// assembled K and builds its phase tables (sets lat_ok)
// Unsigned 32-bit division by a divisor fixed on the host, by a multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and the round-up multiplier
// m = floor(2^32 (2^l - d) / d) + 1 (< 2^32), n / d = (mulhi(m, n) + n) >> l for
// every 32-bit n (the sum formed in 64 bits).  The lattice kernels split node
// numbers into coordinates with it instead of the hardware-less integer division.
struct DivU32 {
    uint32_t d = 1, m = 1;
    int l = 0;
    static DivU32 make(uint32_t d_) {
        DivU32 r;
        r.d = d_;
        r.l = 0;
        while ((1ull << r.l) < d_) ++r.l;
        r.m = (uint32_t)((((1ull << 32) * ((1ull << r.l) - d_)) / d_) + 1);
        return r;
    }
#ifdef __CUDACC__
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return (uint32_t)(((uint64_t)__umulhi(m, n) + n) >> l);
    }
#endif
};

struct LatticeView {
    int dim, N;
    DivU32 dN;                     // division by N
    int64_t nred;
    const float *vol;              // |V| in the solve ordering
    const float2 *tx, *ty, *tz;    // K-hat of the +x, +y, +z edges by perpendicular position
};
void mesh_ensure_lattice(gl_mesh_s *m, cudaStream_t s);
// after a change of mu: the tables again, into the same buffers (checked again;
// a failed check turns the stencil off)
void mesh_refresh_lattice(gl_mesh_s *m, cudaStream_t s);
LatticeView lattice_view(const gl_mesh_s *m);
// the FP64 tables and |V| (solve ordering) for the FP64 Jacobian
struct LatticeView64 {
    int dim, N;
    DivU32 dN;
    int64_t nred;
    const double *vol;
    const double2 *tx, *ty, *tz;
    double ihd;        // 1 / h^d: |V_p| = h^d 2^-b_p (b_p boundary coordinates), so 1 / |V_p| = 2^b_p / h^d
};
LatticeView64 lattice_view64(const gl_mesh_s *m);
// double-float view of the same stencil (row scaled by 2^b / h^d, b = boundary coordinates)
struct LatticeDfView {
    int dim, N;
    DivU32 dN;
    int64_t nred;
    int64_t per_axis;
    const float2 *a;   // |K-hat| / h^d as (hi, lo), axis-major tables
    const float4 *u;   // exp(-i theta) of the +e edge as (re_hi, re_lo, im_hi, im_lo)
};
LatticeDfView lattice_df_view(const gl_mesh_s *m);

// gl_setup.cu
// `like` (nullable): an earlier preconditioner of the same mesh set up with the
// same max_coarse / max_levels / coloring; its aggregates, colours and timed
// kernel choices are taken over (they depend on the sparsity only), everything
// numeric is computed for psi and the mesh's current mu
void precond_setup(gl_prec_s *p, gl_mesh_s *m, const double2 *psi_nat, const gl_options &o, cudaStream_t s,
                   const gl_prec_s *like = nullptr);
// cost of R_k in matrix-vector-product equivalents (entries visited / entries of K-hat)
double precond_cost(const gl_prec_s *p, int k);
// R_inf counters: zeroed before a solve, read after it (synchronises s)
void rinf_reset(gl_prec_s *p, cudaStream_t s);
RinfDev rinf_read(gl_prec_s *p, cudaStream_t s);
void precond_ensure_fp32(gl_prec_s *p, cudaStream_t s);
// multiplies the coarsest level's dense inverse by -1 (gl_precond_debug)
void precond_negate_coarsest(gl_prec_s *p, cudaStream_t s);

// gl_ops.cu (solve ordering)
void permute_in(int64_t n, const int32_t *perm, const double2 *nat, double2 *sol, cudaStream_t s);
void permute_out(int64_t n, const int32_t *perm, const double2 *sol, double2 *nat, cudaStream_t s);
void jacobian_apply_p(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s);
void jacobian_apply_lat64_p(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s);
void jacobian_apply_p32(const gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s);
// gl_solve.cu: the double-float lattice Jacobian of the GL_MIXED_PRECOND solve on
// phi rounded to FP32 (solve ordering; GL_ERR_ARG without a lattice stencil)
void jacobian_apply_pdf(gl_mesh_s *m, const double2 *psi, const double2 *phi, double2 *y, cudaStream_t s);
void residual_p(const gl_mesh_s *m, const double2 *psi, double2 *r, cudaStream_t s);
// node order: r <- -r, returns ||r||_R (part: RED_BLOCKS doubles, scal: 1 double)
double newton_rhs(const gl_mesh_s *m, double2 *r, double *part, double *scal, cudaStream_t s);
void newton_update(int64_t n, const double2 *d, double2 *psi, cudaStream_t s);

// gl_vcycle.cu: z = R_k v in solve ordering; `stop` (nullable) is a device flag
// that turns every kernel into a no-op when nonzero.
void precond_apply_p(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s);
void precond_apply_p32(gl_prec_s *p, const float2 *v, float2 *z, const int *stop, cudaStream_t s);
// autotuner: picks the lanes-per-row width of every grouped-CSR operator by timing
void autotune_levels(gl_prec_s *p, bool fp32, cudaStream_t s);
// picks, per coarse level, the lanes per row of the Gauss-Seidel sweep, its
// synchronisation (grid barrier or neighbour flags) and (FP32) the
// thread-block-cluster form (timed when autotuning)
void plan_sweeps(gl_prec_s *p, bool fp32, cudaStream_t s);
// rebuilds the neighbour-flag partitions of the sweep choices taken over from a template
void rebuild_flag_plans(gl_prec_s *p, bool fp32, cudaStream_t s);
// after a wait of the coarse sweeps ran out: zeroes every level's barrier
// counters and flags and the error word, so later launches start in step
void sweeps_reset(gl_prec_s *p, cudaStream_t s);
// 1 if a device-side wait of p's sweeps ran out since the last reset (synchronises s)
int sweeps_failed(gl_prec_s *p, cudaStream_t s);
// the coarsest level's dense inverse as double-FP32 pairs for the FP32 V-cycle
void coarse_inverse_df(Level &L, cudaStream_t s);
// z = R_k v with FP64 vectors and an FP32 V-cycle
void precond_apply_p64_via32(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s);

// gl_warmstart.cu (solve ordering): x_p = network guess for b_p (with the hint
// hint_nat, node order, nullable), replaced by 0 when ||b - J x||_D >= ||b||_D;
// warmstart_used() reads that decision (after a sync)
void warmstart_apply_p(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, double2 *x_p,
                       cudaStream_t s, const double2 *hint_nat = nullptr);
void hint_guess_p(gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, const double2 *hint_nat, double2 *x_p,
                  cudaStream_t s);
int warmstart_used(gl_warmstart_s *w, cudaStream_t s);

// gl_solve.cu
gl_batch_s *batch_new();
void batch_delete(gl_batch_s *B);
size_t batch_size(const gl_batch_s *B);
void batch_create(gl_batch_s *B, int count, gl_mesh_s *const *meshes, const double2 *const *psi, const gl_options &o,
                  cudaStream_t s);
gl_status batch_run(gl_batch_s *B, const double2 *const *b, double2 *const *x, gl_solve_info *infos, cudaStream_t s);
gl_status jacobian_solve_p(gl_mesh_s *m, gl_prec_s *p, const double2 *psi_p, const double2 *b_p, double2 *x_p,
                           const gl_options &o, gl_solve_info *info, cudaStream_t s);

}  // namespace gl
