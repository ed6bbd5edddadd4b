// gl_vcycle.cu -- the V-cycle that applies R_k = AMG_k(K-hat + 2 D|psi|^2, D .)
// (Eq. prec2): on each level one symmetric Gauss-Seidel step before and after
// the coarse correction (Sec. 4: one pre- and one post-smoothing step), the
// Gauss-Seidel sweeps taken colour by colour (forward: colours ascending,
// backward: descending), and a dense solve on the coarsest level.
//
// All vectors are in the solve ordering, where each colour is a contiguous
// range of positions.  On level 0 the operator is used in its row-scaled form
// K + 2|psi|^2 = D^-1 (K-hat + 2 D|psi|^2): Gauss-Seidel on D^-1 A with right-hand
// side v is Gauss-Seidel on A with right-hand side D v, and the residual handed
// to the restriction is multiplied by D.
#include <cooperative_groups.h>

#include "gl_internal.cuh"
#include "gl_kernels.cuh"
#include "gl_profile.cuh"

namespace gl {

template <typename T>
struct LevelOps;
template <>
struct LevelOps<double> {
    using C = double2;
    static const Sell<C> &A(const Level &L) { return *L.A; }
    static const double *diag(const Level &L) { return L.diag.get(); }
    static const Sell<C> &P(const Level &L) { return L.P; }
    static const Sell<C> &PH(const Level &L) { return L.PH; }
    static const CsrG<C> &Ag(const Level &L) { return L.Ag; }
    static const CsrG<C> &PHg(const Level &L) { return L.PHg; }
    static C *b(Level &L) { return L.b.get(); }
    static C *x(Level &L) { return L.x.get(); }
    static C *r(Level &L) { return L.r.get(); }
};
template <>
struct LevelOps<float> {
    using C = float2;
    static const Sell<C> &A(const Level &L) { return *L.A32; }
    static const float *diag(const Level &L) { return L.diag32.get(); }
    static const Sell<C> &P(const Level &L) { return L.P32; }
    static const Sell<C> &PH(const Level &L) { return L.PH32; }
    static const CsrG<C> &Ag(const Level &L) { return L.Ag32; }
    static const CsrG<C> &PHg(const Level &L) { return L.PHg32; }
    static C *b(Level &L) { return L.b32.get(); }
    static C *x(Level &L) { return L.x32.get(); }
    static C *r(Level &L) { return L.r32.get(); }
};

// x_i <- (b_i - sum_{k != i} A_ik x_k) / A_ii for the rows of one colour [lo, hi).
// `first`: first forward pass from x = 0, where only positions < lo hold values.
template <typename C, typename R>
__global__ void __launch_bounds__(256) k_gs(int64_t lo, int64_t hi, SellView<C> A, const R *__restrict__ diag,
                                            const C *__restrict__ b, C *__restrict__ x, int first,
                                            const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t p = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= hi) return;
    C acc;
    if (first && lo == 0) {  // every neighbour of the first colour still holds zero
        acc.x = 0;
        acc.y = 0;
    } else {
        acc = first ? sell_row_before<C, C>(A, p, x, lo) : sell_row<C, C>(A, p, x);
    }
    C bb = b[p];
    R d = (R)1 / diag[p];
    x[p] = mk((bb.x - acc.x) * d, (bb.y - acc.y) * d);
}

// r = (b - A x) * scale (scale = |V| on level 0, none below)
template <typename C, typename R>
__global__ void __launch_bounds__(256) k_resid(int64_t n, SellView<C> A, const R *__restrict__ diag,
                                               const C *__restrict__ b, const C *__restrict__ x,
                                               const R *__restrict__ scale, C *__restrict__ r,
                                               const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    C acc = sell_row<C, C>(A, p, x);
    C xx = x[p], bb = b[p];
    R d = diag[p];
    R sc = scale ? scale[p] : (R)1;
    r[p] = mk((bb.x - acc.x - d * xx.x) * sc, (bb.y - acc.y - d * xx.y) * sc);
}

// the two kernels above on the finest level of an even-N lattice, with the
// tabulated stencil instead of the stored one (FP32).  Each thread takes
// LAT_RPT rows, blockDim.x apart, and issues the neighbour reads of all of them
// before any write: a colour's rows read only the other colour's x.
constexpr int LAT_RPT = 1;

__global__ void __launch_bounds__(256) k_gs_lat(int64_t lo, int64_t hi, LatticeView L, const float *__restrict__ diag,
                                                const float2 *__restrict__ b, float2 *__restrict__ x, int first,
                                                const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int64_t p0 = lo + (int64_t)blockIdx.x * blockDim.x * LAT_RPT + threadIdx.x;
    // from x = 0 the first colour has no nonzero neighbour and the second sees
    // only the first (two colours, each node's neighbours of the other colour)
    const bool none = first && lo == 0;
    float2 acc[LAT_RPT];
#pragma unroll
    for (int u = 0; u < LAT_RPT; ++u) {
        const int64_t p = p0 + (int64_t)u * blockDim.x;
        acc[u] = (p < hi && !none) ? lattice_row(L, p, x) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < LAT_RPT; ++u) {
        const int64_t p = p0 + (int64_t)u * blockDim.x;
        if (p < hi) {
            const float2 bb = b[p];
            const float d = 1.f / diag[p];
            x[p] = make_float2((bb.x - acc[u].x) * d, (bb.y - acc[u].y) * d);
        }
    }
}
// k_gs_lat with two consecutive positions of a colour per thread: for N % 4 == 0
// positions 2t and 2t + 1 of a colour are the nodes v and v + 2 of one x-line,
// so b, diag, |V| and the written x move as 16- and 8-byte vectors, and the
// neighbours of the pair along y and z (and two of the three along x) are
// adjacent positions of the other colour, read as one 16-byte vector each.
// Per row the edges are summed in the order of lattice_row_f.  (Node v of
// colour c sits at position v >> 1; with p even, v = 2p + a, a = 1 when the
// parity of the line start differs from c.)
__global__ void __launch_bounds__(256) k_gs_lat2(int64_t lo, int64_t hi, LatticeView L,
                                                     const float *__restrict__ diag, const float2 *__restrict__ b,
                                                     float2 *__restrict__ x, int first, const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int64_t p = lo + 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (p >= hi) return;
    const bool none = first && lo == 0;
    const uint32_t c = p >= L.nred ? 1u : 0u;
    const int64_t base = c ? L.nred : 0;
    const int64_t other = c ? 0 : L.nred;
    const uint32_t N = (uint32_t)L.N;
    const uint32_t r = (uint32_t)(p - base);  // even
    const uint32_t v0 = 2u * r;
    const uint32_t row = L.dN.div(v0), k = L.dN.div(row);
    const uint32_t i0 = v0 - row * N, j = row - k * N;
    const uint32_t a = ((i0 + j + k) & 1u) != c ? 1u : 0u;
    const uint32_t i = i0 + a;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    if (!none) {
        const float2 *xo = x + other;
        auto e = [](float2 &acc, float2 t, float2 xv, bool plus) {
            const float ty = plus ? t.y : -t.y;
            acc.x += t.x * xv.x - ty * xv.y;
            acc.y += t.x * xv.y + ty * xv.x;
        };
        // x-direction: positions r - 1 + a .. r + 1 + a of the other colour
        const float4 xm = *reinterpret_cast<const float4 *>(xo + r);  // r, r + 1
        const float2 xlo = make_float2(xm.x, xm.y), xhi = make_float2(xm.z, xm.w);
        float2 xe = make_float2(0.f, 0.f);
        if (a == 0u) {
            if (i > 0) xe = xo[r - 1];
        } else {
            if (i + 3 < N) xe = xo[r + 2];
        }
        // node 1 (v0 + a): x+ -> (v + 1) >> 1, x- -> (v - 1) >> 1
        // a = 0: x+ = r, x- = r - 1; a = 1: x+ = r + 1, x- = r
        // node 2 (v + 2): a = 0: x+ = r + 1, x- = r; a = 1: x+ = r + 2, x- = r + 1
        const float2 t = __ldg(L.tx + (j + N * k));
        if (a == 0u) {
            e(acc0, t, xlo, true);
            if (i > 0) e(acc0, t, xe, false);
            if (i + 3 < N) e(acc1, t, xhi, true);
            e(acc1, t, xlo, false);
        } else {
            e(acc0, t, xhi, true);
            e(acc0, t, xlo, false);
            if (i + 3 < N) e(acc1, t, xe, true);
            e(acc1, t, xhi, false);
        }
        const uint32_t hN = N / 2;
        {
            const float2 t0 = __ldg(L.ty + (i + N * k)), t1 = __ldg(L.ty + (i + 2 + N * k));
            if (j + 1 < N) {
                const float4 q = *reinterpret_cast<const float4 *>(xo + r + hN);
                e(acc0, t0, make_float2(q.x, q.y), true);
                e(acc1, t1, make_float2(q.z, q.w), true);
            }
            if (j > 0) {
                const float4 q = *reinterpret_cast<const float4 *>(xo + r - hN);
                e(acc0, t0, make_float2(q.x, q.y), false);
                e(acc1, t1, make_float2(q.z, q.w), false);
            }
        }
        if (L.dim == 3) {
            const uint32_t hP = N * N / 2;
            const float2 t0 = __ldg(L.tz + (i + N * j)), t1 = __ldg(L.tz + (i + 2 + N * j));
            if (k + 1 < N) {
                const float4 q = *reinterpret_cast<const float4 *>(xo + r + hP);
                e(acc0, t0, make_float2(q.x, q.y), true);
                e(acc1, t1, make_float2(q.z, q.w), true);
            }
            if (k > 0) {
                const float4 q = *reinterpret_cast<const float4 *>(xo + (int64_t)r - hP);
                e(acc0, t0, make_float2(q.x, q.y), false);
                e(acc1, t1, make_float2(q.z, q.w), false);
            }
        }
        const float2 vv = *reinterpret_cast<const float2 *>(L.vol + p);
        const float iv0 = 1.f / vv.x, iv1 = 1.f / vv.y;
        acc0 = make_float2(acc0.x * iv0, acc0.y * iv0);
        acc1 = make_float2(acc1.x * iv1, acc1.y * iv1);
    }
    const float4 bb = *reinterpret_cast<const float4 *>(b + p);
    const float2 dd = *reinterpret_cast<const float2 *>(diag + p);
    const float d0 = 1.f / dd.x, d1 = 1.f / dd.y;
    *reinterpret_cast<float4 *>(x + p) =
        make_float4((bb.x - acc0.x) * d0, (bb.y - acc0.y) * d0, (bb.z - acc1.x) * d1, (bb.w - acc1.y) * d1);
}
// the first two half-sweeps from x = 0 in one launch: red rows x = b / diag,
// black rows relaxed against their red neighbours' b / diag (the values those
// rows get in the same launch)
__global__ void __launch_bounds__(256) k_gs_lat_first2(int64_t n, LatticeView L, const float *__restrict__ diag,
                                                       const float2 *__restrict__ b, float2 *__restrict__ x,
                                                       const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float2 acc = make_float2(0.f, 0.f);
    if (p >= L.nred)
        acc = lattice_row_f(L, p, [&](int64_t q) {
            const float2 bq = b[q];
            const float dq = 1.f / diag[q];
            return make_float2(bq.x * dq, bq.y * dq);
        });
    const float2 bb = b[p];
    const float d = 1.f / diag[p];
    x[p] = make_float2((bb.x - acc.x) * d, (bb.y - acc.y) * d);
}

// the residual of the rows [lo, n) (the rows below lo are not written)
__global__ void __launch_bounds__(256) k_resid_lat(int64_t lo, int64_t n, LatticeView L,
                                                   const float *__restrict__ diag, const float2 *__restrict__ b,
                                                   const float2 *__restrict__ x, const float *__restrict__ scale,
                                                   float2 *__restrict__ r, const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int64_t p0 = lo + (int64_t)blockIdx.x * blockDim.x * LAT_RPT + threadIdx.x;
    float2 acc[LAT_RPT];
#pragma unroll
    for (int u = 0; u < LAT_RPT; ++u) {
        const int64_t p = p0 + (int64_t)u * blockDim.x;
        acc[u] = p < n ? lattice_row(L, p, x) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < LAT_RPT; ++u) {
        const int64_t p = p0 + (int64_t)u * blockDim.x;
        if (p < n) {
            const float2 xx = x[p], bb = b[p];
            const float d = diag[p];
            const float sc = scale ? scale[p] : 1.f;
            r[p] = make_float2((bb.x - acc[u].x - d * xx.x) * sc, (bb.y - acc[u].y - d * xx.y) * sc);
        }
    }
}

// y = S x (add = 0) or y += S x (add = 1) for the rows [lo, n) of a rectangular
// sliced-ELL S
template <typename C>
__global__ void __launch_bounds__(256) k_spmv(int64_t lo, int64_t n, SellView<C> S, const C *__restrict__ x,
                                              C *__restrict__ y, int add, const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t p = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    C acc = sell_row<C, C>(S, p, x);
    if (add) acc = cadd(acc, y[p]);
    y[p] = acc;
}

// ---------------------------------------------------------------- grouped-CSR rows
// sum over the stored entries of row `row` (columns below `lim` only) by the G
// lanes of a group; every lane of the warp must call this (shuffles), rows past
// the end pass row < 0.  The result is complete in the group's first lane.
template <int G, typename C>
__device__ __forceinline__ C group_row(const CsrGView<C> &A, int64_t row, int lane, const C *__restrict__ x,
                                       int64_t lim) {
    C acc;
    acc.x = 0;
    acc.y = 0;
    if (row >= 0) {
        const int64_t q1 = A.rp[row + 1];
        int64_t q = A.rp[row] + lane;
        // four entries per step with all their loads issued first (long rows, such
        // as a restriction to a small coarse level, would otherwise wait for one
        // column and one gather per entry in turn); the sum runs in the same order
        for (; q + 3 * G < q1; q += 4 * G) {
            int32_t c[4];
            C v[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) c[u] = __ldg(A.col + q + u * G);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = A.val[q + u * G];
                if (c[u] < lim) xv[u] = x[c[u]];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c[u] < lim) cfma(acc, v[u], xv[u]);
        }
        for (; q < q1; q += G) {
            int32_t c = __ldg(A.col + q);
            if (c < lim) cfma(acc, A.val[q], x[c]);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, G);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, G);
    }
    return acc;
}

// y = S x (add = 0) or y += S x (add = 1), grouped CSR
template <int G, typename C>
__global__ void __launch_bounds__(256) k_spmv_g(CsrGView<C> S, const C *__restrict__ x, C *__restrict__ y, int add,
                                                const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = t / G;
    int lane = (int)(t % G);
    bool ok = row < S.nrows;
    C acc = group_row<G, C>(S, ok ? row : -1, lane, x, INT64_MAX);
    if (ok && lane == 0) y[row] = add ? cadd(acc, y[row]) : acc;
}

// r = b - A x (coarse levels, no scaling), grouped CSR
template <int G, typename C, typename R>
__global__ void __launch_bounds__(256) k_resid_g(CsrGView<C> A, const R *__restrict__ diag, const C *__restrict__ b,
                                                 const C *__restrict__ x, C *__restrict__ r,
                                                 const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = t / G;
    int lane = (int)(t % G);
    bool ok = row < A.nrows;
    C acc = group_row<G, C>(A, ok ? row : -1, lane, x, INT64_MAX);
    if (ok && lane == 0) {
        C xx = x[row], bb = b[row];
        R d = diag[row];
        r[row] = mk(bb.x - acc.x - d * xx.x, bb.y - acc.y - d * xx.y);
    }
}

// ---------------------------------------------------------------- coarse-level SGS
// Every wait of the coarse sweeps is bounded by SWEEP_WAIT_NS of the global
// timer.  A wait that runs out sets the preconditioner's error word and, when
// the launch belongs to a solve, the solve's status word to STATUS_TIMEOUT, so
// every later kernel of the solve returns at once and the host reports
// GL_ERR_TIMEOUT; every sweep launch returns at once while the error word is
// set, until the host resets the synchronisation state (sweeps_reset).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// spins until *p >= want; false if SWEEP_WAIT_NS passed first
__device__ __forceinline__ bool spin_geq(const unsigned long long *p, unsigned long long want) {
    if (ld_acquire_u64(p) >= want) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned spins = 1;; ++spins) {
        if (ld_acquire_u64(p) >= want) return true;
        if ((spins & 63u) == 0 && globaltimer_ns() - t0 > (unsigned long long)SWEEP_WAIT_NS) return false;
    }
}
__device__ __forceinline__ void report_timeout(int *err, int *stop) {
    atomicExch(err, 1);
    if (stop) atomicExch(stop, STATUS_TIMEOUT);
}
__device__ __forceinline__ bool sweep_halted(const int *stop, const int *err) {
    return (stop && *(volatile const int *)stop) || *(volatile const int *)err;
}

// Grid barrier of the cooperative sweeps: one 64-bit arrival counter per
// (level, precision) that only grows.  Every launch on a counter uses the same
// number of CTAs nb, so the counter is a multiple of nb between launches.  At
// its first barrier a CTA takes a ticket with an atomic add (the round trip
// tells it the launch's base: the ticket rounded down to a multiple of nb); at
// every later barrier it only adds one with a release reduction that it does
// not wait for.  Barrier k is passed when the counter reaches base + (k+1) nb,
// which one thread per CTA observes with acquiring loads.  So the critical path
// from the last CTA's work to everybody's next phase is one release reduction
// and the loads that see it.  The release/acquire pair, after a CTA-wide
// __syncthreads on both sides, orders every thread's x writes before the other
// CTAs' reads.  (A flag per CTA polled by one warp, and a counter reset by the
// last arriver, measured slower.)  A CTA that gives up a wait leaves the
// counter out of step; the host zeroes it (sweeps_reset) before the next use.
// arrival at barrier k; thread 0's base is set at k = 0
__device__ __forceinline__ void grid_arrive(unsigned long long *cnt, unsigned k, unsigned long long &base) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (k == 0) {
            unsigned long long t;
            asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(t) : "l"(cnt) : "memory");
            base = t - t % gridDim.x;
        } else {
            asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
        }
    }
}
// waits for barrier k; false if the wait ran out (thread 0 holds base and the
// extra offset of every wait target, nonzero only when a test has asked for
// waits that cannot end)
__device__ __forceinline__ bool grid_wait(const unsigned long long *cnt, unsigned k, unsigned long long base,
                                          unsigned long long extra, int *err, int *stop) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        const unsigned long long want = base + (unsigned long long)(k + 1) * gridDim.x + extra;
        ok = spin_geq(cnt, want) ? 1 : 0;
        if (!ok) report_timeout(err, stop);
    }
    __syncthreads();
    return ok;
}

// One symmetric Gauss-Seidel step on a coarse level in a single cooperative
// launch: colours 0..nc-1 forward then nc-2..0 backward, a grid barrier between
// colours.  zero_start: the forward pass starts from x = 0 (only columns of
// earlier colours are read).  Between arriving at and leaving a barrier each
// group loads the structure, values, b and diagonal of its row in the next
// colour (they do not depend on x), so after the barrier only the neighbour
// gathers remain.  The gathers are plain cached loads: other blocks wrote the
// values, but every phase starts behind an acquiring load of the wait (and a CTA
// barrier), which the memory model orders before them, and within a phase no
// block writes the colours its rows read; the rows of a colour share many
// neighbours, which then come from L1 (measured 3% faster than L2-only loads).
constexpr int PF = 8;  // prefetched entries per lane

template <typename R>
constexpr int coop_threads() {
    return sizeof(R) == 8 ? 512 : 1024;  // FP64 rows need more registers per thread
}

// relaxes the rows [lo, hi) of colour c (first round prefetched) with gpn groups
// of G lanes; `lim`: only columns below it are read (first sweep from zero)
template <int G, typename C, typename R>
struct SweepRows {
    CsrGView<C> A;
    const R *__restrict__ diag;
    const C *__restrict__ b;
    C *x;
    int lane;
    int32_t pcol[PF];
    C pval[PF];
    C pb;
    R pd = 1;
    int64_t pq0 = 0, pq1 = 0;
    __device__ SweepRows(const CsrGView<C> &A_, const R *d_, const C *b_, C *x_, int lane_)
        : A(A_), diag(d_), b(b_), x(x_), lane(lane_) {
        pb.x = 0;
        pb.y = 0;
    }
    // loads the x-independent data of row `row` (first round of a phase)
    __device__ __forceinline__ void prefetch(int64_t row, bool ok) {
        if (ok)
            prefetch_q(row, true, A.rp[row], A.rp[row + 1]);
        else
            prefetch_q(row, false, 0, 0);
    }
    // the same with the row's entry range [q0, q1) given
    __device__ __forceinline__ void prefetch_q(int64_t row, bool ok, int64_t q0, int64_t q1) {
        pq0 = pq1 = 0;
        if (ok) {
            pq0 = q0;
            pq1 = q1;
            pb = b[row];
            pd = diag[row];
        }
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            int64_t q = pq0 + lane + (int64_t)k * G;
            if (q < pq1) {
                pcol[k] = __ldg(A.col + q);
                pval[k] = A.val[q];
            }
        }
    }
    // one round: row (of this group) relaxed; k == 0 uses the prefetched data;
    // none: every neighbour still holds zero (first colour from a zero guess)
    __device__ __forceinline__ void relax(int64_t row, bool ok, int64_t k, int64_t lim, bool none) {
        C acc;
        acc.x = 0;
        acc.y = 0;
        if (!none) {
            if (k == 0) {
#pragma unroll
                for (int e = 0; e < PF; ++e) {
                    int64_t q = pq0 + lane + (int64_t)e * G;
                    if (q < pq1 && pcol[e] < lim) cfma(acc, pval[e], __ldca(x + pcol[e]));
                }
                for (int64_t q = pq0 + lane + (int64_t)PF * G; q < pq1; q += G) {
                    int32_t cc = __ldg(A.col + q);
                    if (cc < lim) cfma(acc, A.val[q], __ldca(x + cc));
                }
            } else if (ok) {
                for (int64_t q = A.rp[row] + lane; q < A.rp[row + 1]; q += G) {
                    int32_t cc = __ldg(A.col + q);
                    if (cc < lim) cfma(acc, A.val[q], __ldca(x + cc));
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, G);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, G);
        }
        if (ok && lane == 0) {
            C bb = (k == 0) ? pb : b[row];
            R d = (R)1 / ((k == 0) ? pd : diag[row]);
            x[row] = mk((bb.x - acc.x) * d, (bb.y - acc.y) * d);
        }
    }
};

template <int G, typename C, typename R>
__global__ void __launch_bounds__(coop_threads<R>()) k_sgs_coop(CsrGView<C> A, const R *__restrict__ diag,
                                                                const int64_t *__restrict__ cstart, int ncolors,
                                                                const C *__restrict__ b, C *x, int zero_start,
                                                                unsigned *bar, const unsigned long long *extra_p,
                                                                int *err, int *stop) {
    if (sweep_halted(stop, err)) return;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(bar) + (sizeof(R) == 4 ? 0 : 1);
    unsigned long long base = 0;
    const unsigned long long extra = threadIdx.x == 0 ? *extra_p : 0ull;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t grp = t / G, ngroups = (int64_t)gridDim.x * blockDim.x / G;
    SweepRows<G, C, R> S(A, diag, b, x, (int)(t % G));
    int nphase = 2 * ncolors - 1;
    auto colour_of = [&](int ph) { return ph < ncolors ? ph : 2 * ncolors - 2 - ph; };
    {
        int c = colour_of(0);
        S.prefetch(cstart[c] + grp, cstart[c] + grp < cstart[c + 1]);
    }
    for (int ph = 0; ph < nphase; ++ph) {
        int c = colour_of(ph);
        bool first = zero_start && ph < ncolors;
        int64_t lo = cstart[c], hi = cstart[c + 1];
        int64_t lim = first ? lo : INT64_MAX;
        int64_t rounds = (hi - lo + ngroups - 1) / ngroups;
        for (int64_t k = 0; k < rounds; ++k) {
            int64_t row = lo + k * ngroups + grp;
            S.relax(row, row < hi, k, lim, first && lo == 0);
        }
        if (ph + 1 < nphase) {
            // arrive, load the next colour's x-independent data, then wait
            grid_arrive(cnt, (unsigned)ph, base);
            int cn = colour_of(ph + 1);
            S.prefetch(cstart[cn] + grp, cstart[cn] + grp < cstart[cn + 1]);
            if (!grid_wait(cnt, (unsigned)ph, base, extra, err, stop)) return;
        }
    }
}

// The same symmetric step with neighbour flags instead of the grid barrier.
// CTA b owns a chunk of every colour's rows (FlagPlan) and after each
// phase publishes, with a release store, the number of phases it has
// completed; before phase ph (colour c) it waits, with acquiring loads, only
// until every CTA owning a column of its colour-c rows has completed phase
// ph - 1.  That CTA's last write of any such column came in a phase <= ph - 1,
// and its reads of b's colour-c rows since their previous relaxation also lie
// in phases <= ph - 1, so every row reads exactly the values the grid-barrier
// sweep gives it: the two forms are bit-identical for the same G.  CTAs far
// apart may then run several phases apart.  Counters only grow: a launch adds
// 2 nc - 1 to each, so all CTAs of a launch start from the same value (a CTA
// reads its own at the start); a CTA without rows in a colour only counts the
// phase.
//
// The phase is a chain of latencies (the hand-off from the CTAs it reads, the
// gathers of their x, the fence behind this CTA's writes), so the kernel keeps
// everything else off it: warp 0 holds no rows and only publishes and polls,
// starting its poll right after the release; the other warps relax the rows
// and, before the phase is published, issue the loads of the next phase's
// x-independent data (columns, values, b, diagonal) with row pointers from
// shared memory, where the CTA's row pointers of all colours sit for the whole
// launch, so no load waits on another.
template <int G, typename C, typename R>
__global__ void __launch_bounds__(coop_threads<R>()) k_sgs_flags(CsrGView<C> A, const R *__restrict__ diag,
                                                                 const int64_t *__restrict__ cstart, int ncolors,
                                                                 FlagView F, const C *__restrict__ b, C *x,
                                                                 int zero_start, unsigned long long *flags,
                                                                 const unsigned long long *extra_p, int *err,
                                                                 int *stop) {
    if (sweep_halted(stop, err)) return;
    constexpr int NT = coop_threads<R>();
    constexpr int GPB = (NT - 32) / G;  // row groups (rows per round) of the worker warps
    // dynamic shared memory: this CTA's rows [s_lo[c], s_hi[c]) of every colour,
    // the offsets s_roff[c] of their row pointers in s_rp, and the row pointers
    extern __shared__ int64_t s_dyn[];
    int64_t *s_lo = s_dyn, *s_hi = s_dyn + ncolors;
    int32_t *s_roff = reinterpret_cast<int32_t *>(s_dyn + 2 * ncolors);
    int64_t *s_rp = s_dyn + 2 * ncolors + (ncolors + 2) / 2;
    const int nb = gridDim.x, cta = blockIdx.x;
    const bool worker = threadIdx.x >= 32;
    const int grp = worker ? (int)(threadIdx.x - 32) / G : 0;
    unsigned long long *mine = flags + (size_t)cta * FLAG_STRIDE;
    // the launch's starting count, and the offset of every wait target (nonzero
    // only when a test asks for waits that cannot end), kept in shared memory
    __shared__ unsigned long long s_base, s_target0;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_base = *(volatile unsigned long long *)mine;
        s_target0 = s_base + *extra_p;
    }
    for (int c = threadIdx.x; c <= ncolors; c += NT) {
        s_roff[c] = F.roff[(int64_t)cta * (ncolors + 1) + c];
        if (c < ncolors) {
            s_lo[c] = F.rstart[(int64_t)c * (nb + 1) + cta];
            s_hi[c] = F.rstart[(int64_t)c * (nb + 1) + cta + 1];
        }
    }
    __syncthreads();
    {
        const int64_t *src = F.rpl + F.rbase[cta];
        const int total = s_roff[ncolors];
        for (int i0 = threadIdx.x; i0 < total; i0 += 4 * NT) {
            int64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * NT < total) v[u] = __ldg(src + i0 + u * NT);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * NT < total) s_rp[i0 + u * NT] = v[u];
        }
    }
    __syncthreads();
    SweepRows<G, C, R> S(A, diag, b, x, (int)(threadIdx.x % G));
    const int nphase = 2 * ncolors - 1;
    auto colour_of = [&](int ph) { return ph < ncolors ? ph : 2 * ncolors - 2 - ph; };
    auto rows_of = [&](int c, int64_t &lo, int64_t &hi) {
        lo = s_lo[c];
        hi = s_hi[c];
    };
    // the x-independent data of this group's first row of colour c (later rounds
    // of a phase, rare, load their own)
    auto prefetch = [&](int c) {
        int64_t lo, hi;
        rows_of(c, lo, hi);
        const bool ok = lo + grp < hi;
        const int32_t i = s_roff[c] + grp;
        S.prefetch_q(lo + grp, ok, ok ? s_rp[i] : 0, ok ? s_rp[i + 1] : 0);
    };
    if (worker) prefetch(colour_of(0));
    for (int ph = 0; ph < nphase; ++ph) {
        const int c = colour_of(ph);
        const bool first = zero_start && ph < ncolors;
        const int64_t clo = cstart[c];
        const int64_t lim = first ? clo : INT64_MAX;
        int64_t lo, hi;
        rows_of(c, lo, hi);
        if (ph > 0 && hi > lo) {
            if (!worker) {
                const int64_t li = (int64_t)cta * ncolors + c;
                const int cnt = F.nbrc[li];
                bool ok = true;
                if ((int)threadIdx.x < cnt)
                    ok = spin_geq(flags + (size_t)F.nbr[li * FLAG_MAXN + threadIdx.x] * FLAG_STRIDE,
                                  s_target0 + (unsigned long long)ph);
                ok = __all_sync(0xffffffffu, ok);
                if (threadIdx.x == 0) {
                    s_ok = ok ? 1 : 0;
                    if (!ok) report_timeout(err, stop);
                }
            }
            __syncthreads();
            if (!s_ok) return;
        }
        if (worker) {
            const int64_t rounds = (hi - lo + GPB - 1) / GPB;
            for (int64_t k = 0; k < rounds; ++k) {
                const int64_t row = lo + k * GPB + grp;
                S.relax(row, row < hi, k, lim, first && clo == 0);
            }
            // the next phase's x-independent data, before this phase is published
            if (ph + 1 < nphase) prefetch(colour_of(ph + 1));
        }
        __syncthreads();
        if (threadIdx.x == 0) st_release_u64(mine, s_base + (unsigned long long)ph + 1);
    }
}

// ---- partition of the neighbour-flag sweep
// Each colour's positions are split into nb equal contiguous chunks: CTA b owns
// positions [cstart[c] + floor(b m_c / nb), cstart[c] + floor((b + 1) m_c / nb))
// of colour c (m_c its size).  The positions of a colour hold ascending node
// ids, so chunk b of every colour covers about the same part of the level
// (node ids follow space), and no CTA has more than ceil(m_c / nb) rows of a
// colour, which keeps every phase to one round of rows where a partition by
// node id would give some CTAs a second one.
__device__ __forceinline__ int64_t chunk_start(int64_t m, int nb, int b) { return m * b / nb; }
// owner CTA of solve position q
__device__ __forceinline__ int flag_owner(int64_t q, const int64_t *__restrict__ cstart, int ncolors, int nb) {
    int lo = 0, hi = ncolors - 1;  // colour c with cstart[c] <= q < cstart[c + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (cstart[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t m = cstart[lo + 1] - cstart[lo], r = q - cstart[lo];
    int64_t o = m > 0 ? r * nb / m : 0;
    while (o + 1 < nb && chunk_start(m, nb, (int)o + 1) <= r) ++o;
    while (o > 0 && chunk_start(m, nb, (int)o) > r) --o;
    return (int)o;
}
// rstart[c (nb + 1) + b] = first position of CTA b's chunk of colour c
__global__ void k_flag_rstart(int nb, int ncolors, const int64_t *__restrict__ cstart,
                              int64_t *__restrict__ rstart) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)ncolors * (nb + 1)) return;
    const int c = (int)(i / (nb + 1));
    const int bb = (int)(i % (nb + 1));
    rstart[i] = cstart[c] + chunk_start(cstart[c + 1] - cstart[c], nb, bb);
}
// the CTAs owning a column of CTA b's colour-c rows (b itself left out); the
// list length is stored even when it exceeds FLAG_MAXN (the host then drops
// the plan)
template <typename C>
__global__ void __launch_bounds__(256) k_flag_nbrs(CsrGView<C> A, int nb, int ncolors,
                                                   const int64_t *__restrict__ cstart,
                                                   const int64_t *__restrict__ rstart, int32_t *__restrict__ nbr,
                                                   int32_t *__restrict__ nbrc) {
    __shared__ unsigned bits[MAX_FLAG_CTAS / 32];
    const int bb = blockIdx.x, c = blockIdx.y;
    for (int w = threadIdx.x; w < MAX_FLAG_CTAS / 32; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    const int64_t lo = rstart[(int64_t)c * (nb + 1) + bb], hi = rstart[(int64_t)c * (nb + 1) + bb + 1];
    for (int64_t row = lo + threadIdx.x; row < hi; row += blockDim.x)
        for (int64_t q = A.rp[row]; q < A.rp[row + 1]; ++q) {
            const int o = flag_owner(A.col[q], cstart, ncolors, nb);
            if (o != bb) atomicOr(&bits[o >> 5], 1u << (o & 31));
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t li = (int64_t)bb * ncolors + c;
        int cnt = 0;
        for (int w = 0; w < MAX_FLAG_CTAS / 32; ++w) {
            unsigned m = bits[w];
            while (m) {
                const int o = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                if (cnt < FLAG_MAXN) nbr[li * FLAG_MAXN + cnt] = o;
                ++cnt;
            }
        }
        nbrc[li] = cnt;
    }
}

// rpl[rbase[b] + roff[b][c] + i] = A.rp[lo + i], i = 0 .. hi - lo, for CTA b's
// rows [lo, hi) of colour c
template <typename C>
__global__ void __launch_bounds__(256) k_flag_rpl(CsrGView<C> A, int nb, int ncolors,
                                                  const int64_t *__restrict__ rstart, const int32_t *__restrict__ roff,
                                                  const int64_t *__restrict__ rbase, int64_t *__restrict__ rpl) {
    const int bb = blockIdx.x, c = blockIdx.y;
    const int64_t lo = rstart[(int64_t)c * (nb + 1) + bb], hi = rstart[(int64_t)c * (nb + 1) + bb + 1];
    int64_t *dst = rpl + rbase[bb] + roff[(int64_t)bb * (ncolors + 1) + c];
    for (int64_t i = threadIdx.x; i <= hi - lo; i += blockDim.x) dst[i] = A.rp[lo + i];
}

// resident CTAs per SM of a sweep kernel and the SM count (queried once per kernel)
template <typename K>
static void sweep_residency(K kern, int threads, int &per_sm, int &nsm, size_t smem = 0) {
    int dev = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    GL_REQUIRE(per_sm > 0, GL_ERR_CUDA, "cooperative sweep kernel cannot be resident");
}

template <typename K, typename... Args>
static void launch_coop_smem(K kern, int grid, int threads, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GL_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}
template <typename K, typename... Args>
static void launch_coop(K kern, int grid, int threads, cudaStream_t s, Args... args) {
    launch_coop_smem(kern, grid, threads, 0, s, args...);
}

template <int G, typename C, typename R>
static void launch_sgs_coop(const CsrG<C> &A, const R *diag, const int64_t *cstart, int nc, const C *b, C *x,
                            int zero_start, unsigned *bar, const unsigned long long *extra, int *err, int *stop,
                            int64_t max_colour, cudaStream_t s) {
    static int per_sm = -1, nsm = 0;
    const int threads = coop_threads<R>();
    if (per_sm < 0) sweep_residency(k_sgs_coop<G, C, R>, threads, per_sm, nsm);
    int64_t want = (max_colour * G + threads - 1) / threads;
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)per_sm * nsm);
    launch_coop(k_sgs_coop<G, C, R>, grid, threads, s, A.view(), diag, cstart, nc, b, x, zero_start, bar, extra, err,
                stop);
}

// most CTAs a neighbour-flag sweep of G lanes per row may use (all resident,
// with the largest shared memory a plan may ask for)
template <int G, typename C, typename R>
static int flags_max_ctas() {
    static int per_sm = -1, nsm = 0;
    if (per_sm < 0) sweep_residency(k_sgs_flags<G, C, R>, coop_threads<R>(), per_sm, nsm, FLAG_SMEM_MAX);
    return std::min(per_sm * nsm, MAX_FLAG_CTAS);
}

template <int G, typename C, typename R>
static void launch_sgs_flags(const CsrG<C> &A, const R *diag, const int64_t *cstart, int nc, const FlagPlan &F,
                             const C *b, C *x, int zero_start, unsigned long long *flags,
                             const unsigned long long *extra, int *err, int *stop, cudaStream_t s) {
    const bool matches = F.nb > 0 && F.nb <= flags_max_ctas<G, C, R>() && F.G == G && F.smem <= FLAG_SMEM_MAX;
    GL_REQUIRE(matches, GL_ERR_ARG, "neighbour-flag sweep without a matching partition");
    launch_coop_smem(k_sgs_flags<G, C, R>, F.nb, coop_threads<R>(), (size_t)F.smem, s, A.view(), diag, cstart, nc,
                     flag_view(F), b, x, zero_start, flags, extra, err, stop);
}

// Builds the neighbour-flag partition of a coarse level for nb CTAs of G lanes
// per row.  Returns the longest neighbour list (the plan is usable if it is at
// most FLAG_MAXN); synchronises s.
template <typename C>
static int build_flag_plan(const Level &L, const CsrG<C> &A, int G, int nb, FlagPlan &F, cudaStream_t s) {
    F.nb = 0;
    F.G = G;
    GL_REQUIRE(nb >= 1 && nb <= MAX_FLAG_CTAS, GL_ERR_ARG, "neighbour-flag sweep: bad CTA count");
    const int nc = L.ncolors;
    F.rstart.alloc((size_t)nc * (nb + 1));
    F.nbr.alloc((size_t)nb * nc * FLAG_MAXN);
    F.nbrc.alloc((size_t)nb * nc);
    k_flag_rstart<<<grid_for((int64_t)nc * (nb + 1), 256), 256, 0, s>>>(nb, nc, L.cstart_dev.get(), F.rstart.get());
    GL_LAUNCH_CHECK();
    k_flag_nbrs<C><<<dim3(nb, nc), 256, 0, s>>>(A.view(), nb, nc, L.cstart_dev.get(), F.rstart.get(), F.nbr.get(),
                                                F.nbrc.get());
    GL_LAUNCH_CHECK();
    std::vector<int32_t> cnt((size_t)nb * nc);
    std::vector<int64_t> rs((size_t)nc * (nb + 1));
    GL_CUDA(cudaMemcpyAsync(cnt.data(), F.nbrc.get(), cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaMemcpyAsync(rs.data(), F.rstart.get(), rs.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    int mx = 0;
    for (int32_t v : cnt) mx = std::max(mx, (int)v);
    // each CTA's row pointers, colour after colour: its rows of colour c and their end
    std::vector<int32_t> roff((size_t)nb * (nc + 1));
    std::vector<int64_t> rbase(nb + 1);
    int64_t most = 0;
    rbase[0] = 0;
    for (int bb = 0; bb < nb; ++bb) {
        int32_t o = 0;
        for (int c = 0; c < nc; ++c) {
            roff[(size_t)bb * (nc + 1) + c] = o;
            o += (int32_t)(rs[(size_t)c * (nb + 1) + bb + 1] - rs[(size_t)c * (nb + 1) + bb]) + 1;
        }
        roff[(size_t)bb * (nc + 1) + nc] = o;
        rbase[bb + 1] = rbase[bb] + o;
        most = std::max<int64_t>(most, o);
    }
    // the kernel's layout: lo and hi per colour, nc + 1 offsets (int32), the row pointers
    F.smem = (int)std::min<int64_t>((2 * nc + (nc + 2) / 2 + most) * (int64_t)sizeof(int64_t), INT32_MAX);
    F.roff.alloc(roff.size());
    F.rbase.alloc(nb + 1);
    F.rpl.alloc((size_t)std::max<int64_t>(rbase[nb], 1));
    GL_CUDA(cudaMemcpyAsync(F.roff.get(), roff.data(), roff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    GL_CUDA(cudaMemcpyAsync(F.rbase.get(), rbase.data(), rbase.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_flag_rpl<<<dim3(nb, nc), 256, 0, s>>>(A.view(), nb, nc, F.rstart.get(), F.roff.get(), F.rbase.get(), F.rpl.get());
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamSynchronize(s));
    if (mx <= FLAG_MAXN && F.smem <= FLAG_SMEM_MAX) F.nb = nb;
    return F.smem <= FLAG_SMEM_MAX ? mx : FLAG_MAXN + 1;
}

// ---------------------------------------------------------------- cluster sweeps
// One thread-block cluster runs a whole symmetric Gauss-Seidel step of a coarse
// level in FP32.  The level's x lives in the distributed shared memory of the
// cluster: CTA r holds positions [r chunk, (r + 1) chunk).  Rows of a colour are
// spread over all the cluster's threads (G lanes per row); neighbour values are
// read from the owning CTA's shared memory and new values written there, and
// consecutive colours are separated by the cluster's hardware barrier, split
// into arrive and wait so that the next colour's x-independent data (row
// bounds, columns, values, b, diagonal) is loaded in between.  The same colour
// order and the same first-sweep rule (from x = 0, later colours are still 0) as
// the cooperative kernel.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

constexpr int CLUSTER_THREADS = 1024;

template <int G>
__global__ void __launch_bounds__(CLUSTER_THREADS) k_sgs_cluster(CsrGView<float2> A, const float *__restrict__ diag,
                                                                 const int64_t *__restrict__ cstart, int ncolors,
                                                                 const float2 *__restrict__ b, float2 *x,
                                                                 int zero_start, int chunk, float inv_chunk,
                                                                 const int *__restrict__ stop) {
    extern __shared__ float2 xs[];
    if (stop && *stop) return;
    namespace cgs = cooperative_groups;
    cgs::cluster_group cl = cgs::this_cluster();
    const int rank = (int)cl.block_rank();
    const int nblk = (int)cl.num_blocks();
    const int64_t n = A.nrows;
    const int64_t base = (int64_t)rank * chunk;
    const int64_t mine = std::max<int64_t>(0, std::min<int64_t>(chunk, n - base));
    for (int64_t i = threadIdx.x; i < mine; i += blockDim.x) xs[i] = zero_start ? make_float2(0.f, 0.f) : x[base + i];
    // owning CTA and offset of position c
    auto owner_of = [&](int32_t c) {
        int o = (int)((float)c * inv_chunk);
        if ((int64_t)o * chunk > c) --o;
        else if ((int64_t)(o + 1) * chunk <= c) ++o;
        return o;
    };
    auto xget = [&](int32_t c) {
        const int o = owner_of(c);
        return cl.map_shared_rank(xs, o)[c - (int64_t)o * chunk];
    };
    const int64_t t = (int64_t)rank * blockDim.x + threadIdx.x;
    const int64_t grp = t / G, ngroups = (int64_t)nblk * blockDim.x / G;
    const int lane = (int)(t % G);
    const int nphase = 2 * ncolors - 1;
    int32_t pcol[PF];
    float2 pval[PF];
    float2 pb = make_float2(0.f, 0.f);
    float pd = 1.f;
    int64_t pq0 = 0, pq1 = 0;
    auto colour_of = [&](int ph) { return ph < ncolors ? ph : 2 * ncolors - 2 - ph; };
    auto prefetch = [&](int64_t row, bool ok) {
        pq0 = pq1 = 0;
        if (ok) {
            pq0 = A.rp[row];
            pq1 = A.rp[row + 1];
            pb = b[row];
            pd = diag[row];
        }
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            int64_t q = pq0 + lane + (int64_t)k * G;
            if (q < pq1) {
                pcol[k] = __ldg(A.col + q);
                pval[k] = A.val[q];
            }
        }
    };
    cluster_arrive();
    {
        int c = colour_of(0);
        prefetch(cstart[c] + grp, cstart[c] + grp < cstart[c + 1]);
    }
    cluster_wait();
    for (int ph = 0; ph < nphase; ++ph) {
        const int c = colour_of(ph);
        const bool first = zero_start && ph < ncolors;
        const int64_t lo = cstart[c], hi = cstart[c + 1];
        const int64_t rounds = (hi - lo + ngroups - 1) / ngroups;
        for (int64_t k = 0; k < rounds; ++k) {
            const int64_t row = lo + k * ngroups + grp;
            const bool ok = row < hi;
            float2 acc = make_float2(0.f, 0.f);
            if (!(first && lo == 0)) {
                if (k == 0) {
#pragma unroll
                    for (int e = 0; e < PF; ++e) {
                        int64_t q = pq0 + lane + (int64_t)e * G;
                        if (q < pq1) cfma(acc, pval[e], xget(pcol[e]));
                    }
                    for (int64_t q = pq0 + lane + (int64_t)PF * G; q < pq1; q += G)
                        cfma(acc, A.val[q], xget(__ldg(A.col + q)));
                } else if (ok) {
                    for (int64_t q = A.rp[row] + lane; q < A.rp[row + 1]; q += G)
                        cfma(acc, A.val[q], xget(__ldg(A.col + q)));
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, G);
                acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, G);
            }
            if (ok && lane == 0) {
                const float2 bb = (k == 0) ? pb : b[row];
                const float d = 1.f / ((k == 0) ? pd : diag[row]);
                const int o = owner_of((int32_t)row);
                cl.map_shared_rank(xs, o)[row - (int64_t)o * chunk] =
                    make_float2((bb.x - acc.x) * d, (bb.y - acc.y) * d);
            }
        }
        cluster_arrive();
        if (ph + 1 < nphase) {
            const int cn = colour_of(ph + 1);
            prefetch(cstart[cn] + grp, cstart[cn] + grp < cstart[cn + 1]);
        }
        cluster_wait();
    }
    for (int64_t i = threadIdx.x; i < mine; i += blockDim.x) x[base + i] = xs[i];
}

// cluster size (16 with the non-portable opt-in, else 8) and chunk for a level
// of n rows whose x fits the cluster's shared memory; size 0 if none fits
template <int G>
static void plan_sgs_cluster(int64_t n, int &size, int &chunk) {
    size = 0;
    chunk = 0;
    if (n <= 0) return;
    GL_CUDA(cudaFuncSetAttribute(k_sgs_cluster<G>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int cs : {16, 8}) {
        int64_t ch = (n + cs - 1) / cs;
        int64_t smem = ch * (int64_t)sizeof(float2);
        if (smem > 200 * 1024) continue;
        GL_CUDA(cudaFuncSetAttribute(k_sgs_cluster<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(CLUSTER_THREADS);
        cfg.dynamicSmemBytes = (size_t)smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_sgs_cluster<G>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters >= 1) {
            size = cs;
            chunk = (int)ch;
            return;
        }
    }
}

template <int G>
static void launch_sgs_cluster(const CsrG<float2> &A, const float *diag, const int64_t *cstart, int nc,
                               const float2 *b, float2 *x, int zero_start, int size, int chunk, const int *stop,
                               cudaStream_t s) {
    const size_t smem = (size_t)chunk * sizeof(float2);
    GL_CUDA(cudaFuncSetAttribute(k_sgs_cluster<G>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    GL_CUDA(cudaFuncSetAttribute(k_sgs_cluster<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(size);
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GL_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_cluster<G>, A.view(), diag, cstart, nc, b, x, zero_start, chunk,
                               1.0f / (float)chunk, stop));
}

// dispatch on the group width
#define GL_DISPATCH_G(G_, CALL)                       \
    switch (G_) {                                     \
        case 1: { constexpr int GG = 1; CALL; break; }   \
        case 2: { constexpr int GG = 2; CALL; break; }   \
        case 4: { constexpr int GG = 4; CALL; break; }   \
        case 8: { constexpr int GG = 8; CALL; break; }   \
        case 16: { constexpr int GG = 16; CALL; break; } \
        default: { constexpr int GG = 32; CALL; break; } \
    }

template <typename C>
static void spmv_g(const CsrG<C> &S, const C *x, C *y, int add, const int *stop, cudaStream_t s) {
    GL_DISPATCH_G(S.G, (k_spmv_g<GG, C><<<grid_for(S.nrows * GG, 256), 256, 0, s>>>(S.view(), x, y, add, stop)));
}

// Autotuner: times the grouped-CSR SpMV of one operator for every group width
// (lanes per row) on this GPU and keeps the fastest.  x must hold the
// operator's column count, y its row count (contents irrelevant).
template <typename C>
static void tune_groups(CsrG<C> &S, const C *x, C *y, cudaStream_t s) {
    if (S.nrows <= 0 || S.nnz <= 0) return;
    cudaEvent_t e0, e1;
    GL_CUDA(cudaEventCreate(&e0));
    GL_CUDA(cudaEventCreate(&e1));
    int best = S.G;
    float best_ms = 1e30f;
    for (int g = 1; g <= 32; g *= 2) {
        S.G = g;
        spmv_g<C>(S, x, y, 0, nullptr, s);  // warm
        GL_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 5; ++r) spmv_g<C>(S, x, y, 0, nullptr, s);
        GL_CUDA(cudaEventRecord(e1, s));
        GL_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        GL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            best = g;
        }
    }
    S.G = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

void autotune_levels(gl_prec_s *p, bool fp32, cudaStream_t s) {
    for (int l = 0; l + 1 < p->nlev; ++l) {
        Level &L = p->L[l], &Lc = p->L[l + 1];
        if (fp32) {
            if (l > 0) tune_groups<float2>(L.Ag32, L.x32.get(), L.r32.get(), s);
            tune_groups<float2>(L.PHg32, L.r32.get(), Lc.b32.get(), s);
        } else {
            if (l > 0) tune_groups<double2>(L.Ag, L.x.get(), L.r.get(), s);
            tune_groups<double2>(L.PHg, L.r.get(), Lc.b.get(), s);
        }
    }
    GL_LAUNCH_CHECK();
}

// x = M b for the dense coarsest inverse (FP64).  The product is bound by the
// FP64 pipe (four FMAs per complex entry), so one warp takes one row and every
// lane keeps four independent accumulators to keep FMAs in flight; b comes
// through L1 (the same 16 n bytes for every row).
constexpr int DMV_WARPS = 8;
__global__ void __launch_bounds__(32 * DMV_WARPS) k_dense_mv(int64_t n, const double2 *__restrict__ M,
                                                             const double2 *__restrict__ b, double2 *__restrict__ x,
                                                             const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * DMV_WARPS + (threadIdx.x >> 5);
    if (row >= n) return;
    const double2 *mr = M + row * n;
    double2 a0 = make_double2(0, 0), a1 = a0, a2 = a0, a3 = a0;
    int64_t j = lane;
    for (; j + 96 < n; j += 128) {
        cfma(a0, mr[j], __ldg(b + j));
        cfma(a1, mr[j + 32], __ldg(b + j + 32));
        cfma(a2, mr[j + 64], __ldg(b + j + 64));
        cfma(a3, mr[j + 96], __ldg(b + j + 96));
    }
    for (; j < n; j += 32) cfma(a0, mr[j], __ldg(b + j));
    double sx = (a0.x + a1.x) + (a2.x + a3.x), sy = (a0.y + a1.y) + (a2.y + a3.y);
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) x[row] = make_double2(sx, sy);
}

// x = M b for the FP32 V-cycle: b is an FP32 vector (exact), M the dense
// coarsest inverse as double-FP32 pairs, every product error-free and every sum
// compensated (Dot2), so the value carries about 48 significant bits before it
// is rounded to FP32 - the FP64 product's value, at the FP32 pipe's rate (the
// FP64 form of this product is bound by the FP64 pipe).  The product is a
// stream of the matrix (16 B per entry): one warp takes a row, so every row of a
// coarsest level of a few thousand nodes is resident at once (one wave; wider
// blocks left a second, mostly idle wave: 31 us against 25 us at 2720 nodes),
// and every lane keeps U entries in flight; partial (sum, compensation) pairs
// are combined by shuffles.
constexpr int DMV_DF_THREADS = 32;  // one warp
__global__ void __launch_bounds__(DMV_DF_THREADS) k_dense_mv_df(int64_t n, const float4 *__restrict__ M,
                                                                const float2 *__restrict__ b,
                                                                float2 *__restrict__ x, const int *__restrict__ stop) {
    if (stop && *stop) return;
    const int64_t row = blockIdx.x;
    const float4 *mr = M + row * n;
    float rs[2] = {0.f, 0.f}, rc[2] = {0.f, 0.f}, is[2] = {0.f, 0.f}, ic[2] = {0.f, 0.f};
    int64_t j = threadIdx.x;
    constexpr int U = 8;
    for (; j + (U - 1) * DMV_DF_THREADS < n; j += U * DMV_DF_THREADS) {
        float4 m[U];
        float2 bb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            m[u] = mr[j + u * DMV_DF_THREADS];
            bb[u] = __ldg(b + j + u * DMV_DF_THREADS);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int a = u & 1;
            dot2_df(rs[a], rc[a], make_float2(m[u].x, m[u].y), bb[u].x);
            dot2_df(rs[a], rc[a], make_float2(-m[u].z, -m[u].w), bb[u].y);
            dot2_df(is[a], ic[a], make_float2(m[u].x, m[u].y), bb[u].y);
            dot2_df(is[a], ic[a], make_float2(m[u].z, m[u].w), bb[u].x);
        }
    }
    for (; j < n; j += DMV_DF_THREADS) {
        const float4 m = mr[j];
        const float2 bb = __ldg(b + j);
        dot2_df(rs[0], rc[0], make_float2(m.x, m.y), bb.x);
        dot2_df(rs[0], rc[0], make_float2(-m.z, -m.w), bb.y);
        dot2_df(is[0], ic[0], make_float2(m.x, m.y), bb.y);
        dot2_df(is[0], ic[0], make_float2(m.z, m.w), bb.x);
    }
    dot2_add(rs[0], rc[0], rs[1]);
    rc[0] = __fadd_rn(rc[0], rc[1]);
    dot2_add(is[0], ic[0], is[1]);
    ic[0] = __fadd_rn(ic[0], ic[1]);
    for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_down_sync(0xffffffffu, rs[0], o), ac = __shfl_down_sync(0xffffffffu, rc[0], o);
        const float c = __shfl_down_sync(0xffffffffu, is[0], o), cc = __shfl_down_sync(0xffffffffu, ic[0], o);
        dot2_add(rs[0], rc[0], a);
        rc[0] = __fadd_rn(rc[0], ac);
        dot2_add(is[0], ic[0], c);
        ic[0] = __fadd_rn(ic[0], cc);
    }
    if (threadIdx.x == 0) x[row] = make_float2(__fadd_rn(rs[0], rc[0]), __fadd_rn(is[0], ic[0]));
}

__global__ void k_split_dense_df(int64_t nn, const double2 *__restrict__ a, float4 *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float2 re = split_df(a[i].x), im = split_df(a[i].y);
    out[i] = make_float4(re.x, re.y, im.x, im.y);
}

void coarse_inverse_df(Level &L, cudaStream_t s) {
    const int64_t nn = L.n * L.n;
    // an existing buffer of the right size is kept (captured solve graphs hold its address)
    if (L.Ainv_df.n != (size_t)nn) L.Ainv_df.alloc(nn);
    k_split_dense_df<<<grid_for(nn, 256), 256, 0, s>>>(nn, L.Ainv.get(), L.Ainv_df.get());
    GL_LAUNCH_CHECK();
}

template <typename C>
__global__ void k_axpy_t(int64_t n, const C *__restrict__ e, C *__restrict__ z, const int *__restrict__ stop) {
    if (stop && *stop) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = cadd(z[i], e[i]);
}

__global__ void k_f2d(int64_t n, const float2 *a, double2 *b, const int *stop) {
    if (stop && *stop) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = to64(a[i]);
}
__global__ void k_d2f2(int64_t n, const double2 *a, float2 *b, const int *stop) {
    if (stop && *stop) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = to32(a[i]);
}

template <typename T>
static void coarse_solve(gl_prec_s *p, Level &L, const typename LevelOps<T>::C *b, typename LevelOps<T>::C *x,
                         const int *stop, cudaStream_t s);
template <>
void coarse_solve<double>(gl_prec_s *, Level &L, const double2 *b, double2 *x, const int *stop, cudaStream_t s) {
    ProfScope ps("coarse", (double)L.n * L.n * sizeof(double2), s);
    k_dense_mv<<<grid_for(L.n, DMV_WARPS), 32 * DMV_WARPS, 0, s>>>(L.n, L.Ainv.get(), b, x, stop);
}
template <>
void coarse_solve<float>(gl_prec_s *p, Level &L, const float2 *b, float2 *x, const int *stop, cudaStream_t s) {
    if (L.Ainv_df.get()) {
        // double-FP32 product of the FP32 right-hand side
        ProfScope ps("coarse", (double)L.n * L.n * sizeof(float4), s);
        k_dense_mv_df<<<(unsigned)L.n, DMV_DF_THREADS, 0, s>>>(L.n, L.Ainv_df.get(), b, x, stop);
        return;
    }
    // the FP32 right-hand side widened once, the FP64 solve, the result narrowed
    note_launch(2);
    k_f2d<<<grid_for(L.n, 256), 256, 0, s>>>(L.n, b, p->coarse_b64.get(), stop);
    {
        ProfScope ps("coarse", (double)L.n * L.n * sizeof(double2), s);
        k_dense_mv<<<grid_for(L.n, DMV_WARPS), 32 * DMV_WARPS, 0, s>>>(L.n, L.Ainv.get(), p->coarse_b64.get(),
                                                                       p->coarse_x64.get(), stop);
    }
    k_d2f2<<<grid_for(L.n, 256), 256, 0, s>>>(L.n, p->coarse_x64.get(), x, stop);
}

template <typename T>
static void gs_sweep(Level &L, int level, const typename LevelOps<T>::C *b, typename LevelOps<T>::C *x, int c,
                     bool first, const int *stop, cudaStream_t s, const LatticeView *lat = nullptr) {
    using O = LevelOps<T>;
    using C = typename O::C;
    int64_t lo = L.cstart[c], hi = L.cstart[c + 1];
    if (hi <= lo) return;
    if constexpr (sizeof(T) == 4) {
        if (lat) {
            // diagonal, b and the written x per row; the other colour's x once and
            // the phase tables, unless the colour is relaxed from a zero guess
            double bytes = (double)(hi - lo) * (sizeof(T) + 2 * sizeof(C));
            if (!(first && lo == 0))
                bytes += (double)(L.n - (hi - lo)) * sizeof(C) + (double)lat->N * lat->N * lat->dim * 8.0;
            ProfScope ps("gs0", bytes, s);
            if (lat->N % 4 == 0)  // colour ranges of even length, pairs within one x-line
                k_gs_lat2<<<grid_for((hi - lo) / 2, 256), 256, 0, s>>>(lo, hi, *lat, O::diag(L), b, x, first ? 1 : 0,
                                                                       stop);
            else
                k_gs_lat<<<grid_for(hi - lo, 256 * LAT_RPT), 256, 0, s>>>(lo, hi, *lat, O::diag(L), b, x,
                                                                         first ? 1 : 0, stop);
            return;
        }
    }
    // algorithmic bytes: diagonal, b and the written x for each row; the stored
    // off-diagonals (value + column) and each neighbour value once, unless the
    // colour is relaxed from an all-zero guess
    double rows = (double)(hi - lo);
    double bytes = rows * (sizeof(T) + 2 * sizeof(C));
    if (!(first && lo == 0))
        bytes += (double)L.cnnz[c] * (sizeof(C) + 4) + (double)(first ? lo : L.n - (hi - lo)) * sizeof(C);
    // a complex FMA (8 flops) per entry read, (b - acc) / diag per row (6)
    const double flops = (first && lo == 0 ? 0.0 : 8.0 * (double)L.cnnz[c]) + 6.0 * rows;
    ProfScope ps(level == 0 ? "gs0" : "gs", bytes, s, flops);
    k_gs<C, T><<<grid_for(hi - lo, 256), 256, 0, s>>>(lo, hi, O::A(L).view(), O::diag(L), b, x, first ? 1 : 0, stop);
}

// symmetric Gauss-Seidel: forward over colours, then backward; the backward pass
// starts one colour early because re-relaxing the last forward colour with
// unchanged neighbours reproduces the same values
template <typename T>
static void sgs(Level &L, int level, const typename LevelOps<T>::C *b, typename LevelOps<T>::C *x, bool zero_start,
                const int *stop, cudaStream_t s, const LatticeView *lat = nullptr) {
    int nc = L.ncolors;
    if constexpr (sizeof(T) == 4) {
        if (lat && zero_start && nc == 2) {
            // both forward colours in one launch; per row b, diagonal and the written
            // x, the red rows' b and diagonal once more for the black rows, the tables
            double bytes = (double)L.n * (sizeof(T) + 2 * sizeof(typename LevelOps<T>::C)) +
                           (double)L.cstart[1] * (sizeof(T) + sizeof(typename LevelOps<T>::C)) +
                           (double)lat->N * lat->N * lat->dim * 8.0;
            {
                ProfScope ps("gs0", bytes, s);
                k_gs_lat_first2<<<grid_for(L.n, 256), 256, 0, s>>>(L.n, *lat, LevelOps<T>::diag(L), b, x, stop);
            }
            gs_sweep<T>(L, level, b, x, 0, false, stop, s, lat);
            return;
        }
    }
    for (int c = 0; c < nc; ++c) gs_sweep<T>(L, level, b, x, c, zero_start, stop, s, lat);
    for (int c = nc - 2; c >= 0; --c) gs_sweep<T>(L, level, b, x, c, false, stop, s, lat);
}

// closed-form finest-level stencil for the FP32 V-cycle, when the mesh has one
template <typename T>
static bool lattice_for(const gl_prec_s *p, LatticeView &v) {
    if constexpr (sizeof(T) == 4) {
        if (p->lattice && p->mesh->lat_ok && p->L[0].ncolors == 2) {
            v = lattice_view(p->mesh);
            return true;
        }
    }
    return false;
}

// pre- or post-smoothing on level l: per-colour launches on the lattice level
// (two colours, large sweeps), one cooperative launch on coarse levels
template <typename T>
static void smooth(gl_prec_s *p, int l, const typename LevelOps<T>::C *b, typename LevelOps<T>::C *x, bool zero_start,
                   const int *stop, cudaStream_t s) {
    using O = LevelOps<T>;
    using C = typename O::C;
    Level &L = p->L[l];
    if (l == 0) {
        LatticeView lv;
        bool lat = lattice_for<T>(p, lv);
        sgs<T>(L, l, b, x, zero_start, stop, s, lat ? &lv : nullptr);
        return;
    }
    const CsrG<C> &A = O::Ag(L);
    int64_t maxc = 0;
    for (int c = 0; c < L.ncolors; ++c) maxc = std::max(maxc, L.cstart[c + 1] - L.cstart[c]);
    // algorithmic bytes of one symmetric step: every visit of a colour reads its
    // rows' stored entries (value + column) and b, diagonal and writes x; the
    // first colour from a zero guess reads no entries
    double bytes = 0, flops = 0;
    for (int ph = 0; ph < 2 * L.ncolors - 1; ++ph) {
        int c = ph < L.ncolors ? ph : 2 * L.ncolors - 2 - ph;
        double rows = (double)(L.cstart[c + 1] - L.cstart[c]);
        bytes += rows * (2 * sizeof(C) + sizeof(T));
        flops += 6.0 * rows;
        if (!(zero_start && ph == 0)) {
            bytes += (double)L.cnnz[c] * (sizeof(C) + 4);
            flops += 8.0 * (double)L.cnnz[c];
        }
    }
    ProfScope ps("gs", bytes, s, flops);
    const int sG = sizeof(T) == 4 ? L.sgs_G32 : L.sgs_G64;
    if constexpr (sizeof(T) == 4) {
        if (L.cl_size > 0 && p->cluster_sweeps) {
            GL_DISPATCH_G(sG, (launch_sgs_cluster<GG>(A, O::diag(L), L.cstart_dev.get(), L.ncolors, b, x,
                                                       zero_start ? 1 : 0, L.cl_size, L.cl_chunk, stop, s)));
            return;
        }
    }
    // the status word of the solve this sweep belongs to: a wait that runs out writes it
    int *status = const_cast<int *>(stop);
    const int sync = sizeof(T) == 4 ? L.sync32 : L.sync64;
    if (sync == 1) {
        const FlagPlan &F = sizeof(T) == 4 ? L.fl32 : L.fl64;
        unsigned long long *flags = L.flags.get() + (sizeof(T) == 4 ? 0 : (size_t)MAX_FLAG_CTAS * FLAG_STRIDE);
        GL_DISPATCH_G(sG, (launch_sgs_flags<GG, C, T>(A, O::diag(L), L.cstart_dev.get(), L.ncolors, F, b, x,
                                                       zero_start ? 1 : 0, flags, p->wait_extra.get(), p->err.get(),
                                                       status, s)));
        return;
    }
    GL_DISPATCH_G(sG, (launch_sgs_coop<GG, C, T>(A, O::diag(L), L.cstart_dev.get(), L.ncolors, b, x,
                                                  zero_start ? 1 : 0, L.barrier.get(), p->wait_extra.get(),
                                                  p->err.get(), status, maxc, s)));
}

template <typename T>
static void vcycle(gl_prec_s *p, int l, const typename LevelOps<T>::C *b, typename LevelOps<T>::C *x,
                   const int *stop, cudaStream_t s) {
    using O = LevelOps<T>;
    using C = typename O::C;
    Level &L = p->L[l];
    if (l == p->nlev - 1) {
        coarse_solve<T>(p, L, b, x, stop, s);
        return;
    }
    Level &Lc = p->L[l + 1];
    smooth<T>(p, l, b, x, true, stop, s);
    C *r = O::r(L);
    bool restrict_black = false;
    if (l == 0) {
        const T *scale;
        if constexpr (sizeof(T) == 8)
            scale = p->mesh->volp.get();
        else
            scale = p->mesh->volp32.get();
        ProfScope ps("resid0", 0, s);
        LatticeView lv;
        bool lat = lattice_for<T>(p, lv);
        if constexpr (sizeof(T) == 4) {
            if (lat) {
                // the pre-smoothing ended by relaxing the red rows against black
                // neighbours it left unchanged, so their residual is zero (up to the
                // rounding of that relaxation): only the black rows are formed, and
                // the restriction below reads only black columns
                const int64_t lo = L.PHg32b.nrows > 0 ? L.cstart[1] : 0;
                k_resid_lat<<<grid_for(L.n - lo, 256 * LAT_RPT), 256, 0, s>>>(lo, L.n, lv, O::diag(L), b, x, scale,
                                                                              r, stop);
            }
        }
        if (!lat)
            k_resid<C, T><<<grid_for(L.n, 256), 256, 0, s>>>(L.n, O::A(L).view(), O::diag(L), b, x, scale, r, stop);
        restrict_black = lat && sizeof(T) == 4 && L.PHg32b.nrows > 0;
    } else {
        const CsrG<C> &A = O::Ag(L);
        ProfScope ps("resid", 0, s);
        GL_DISPATCH_G(A.G, (k_resid_g<GG, C, T><<<grid_for(L.n * GG, 256), 256, 0, s>>>(A.view(), O::diag(L), b, x,
                                                                                        r, stop)));
    }
    {
        ProfScope ps("restrict", 0, s);
        if constexpr (sizeof(T) == 4) {
            if (restrict_black) {
                spmv_g<C>(L.PHg32b, r, O::b(Lc), 0, stop, s);
            } else {
                spmv_g<C>(O::PHg(L), r, O::b(Lc), 0, stop, s);
            }
        } else {
            spmv_g<C>(O::PHg(L), r, O::b(Lc), 0, stop, s);
        }
    }
    vcycle<T>(p, l + 1, O::b(Lc), O::x(Lc), stop, s);
    {
        // x += P e_c.  The post-smoothing that follows relaxes colour 0 first, and a
        // Gauss-Seidel relaxation of a row does not read the row's own old value,
        // so the correction of colour-0 rows would be overwritten unread: only the
        // rows of the other colours are corrected (the same values, bit for bit)
        const int64_t lo = L.ncolors > 1 ? L.cstart[1] : 0;
        ProfScope ps("prolong", 0, s);
        k_spmv<C><<<grid_for(L.n - lo, 256), 256, 0, s>>>(lo, L.n, O::P(L).view(), O::x(Lc), x, 1, stop);
    }
    smooth<T>(p, l, b, x, false, stop, s);
    GL_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ R_inf
// partial sums of ||x||_D^2 = sum_i |V_i| |x_i|^2 (fixed grid RED_BLOCKS x RED_THREADS)
__global__ void __launch_bounds__(RED_THREADS) k_dnorm2_part(int64_t n, const double2 *__restrict__ x,
                                                             const double *__restrict__ vol,
                                                             double *__restrict__ part, const int *stop) {
    if (stop && *stop) return;
    __shared__ double sh[RED_THREADS];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 a = x[i];
        acc += vol[i] * (a.x * a.x + a.y * a.y);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// sum of the RED_BLOCKS partial sums by one block of RED_THREADS (every thread gets it)
__device__ double sum_parts(const double *__restrict__ part) {
    __shared__ double sh[RED_THREADS];
    double acc = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(RED_THREADS) k_rinf_begin(RinfDev *R, const double *__restrict__ part,
                                                            const int *stop) {
    if (stop && *stop) return;
    double v2 = sum_parts(part);
    if (threadIdx.x == 0) {
        R->v2 = v2;
        R->k = 0;
    }
}

// after a cycle: continue while ||r||_D^2 > tol^2 ||v||_D^2 and fewer than kmax
// cycles ran (a NaN stops the loop; MINRES reports it).  Always sets the
// condition, so the loop ends whatever the state.
__global__ void __launch_bounds__(RED_THREADS) k_rinf_decide(cudaGraphConditionalHandle h, RinfDev *R,
                                                             const double *__restrict__ part, const int *stop,
                                                             double tol2, int kmax) {
    const bool halted = stop && *stop;
    double r2 = 0;
    if (!halted) r2 = sum_parts(part);
    if (threadIdx.x == 0) {
        unsigned go = 0;
        if (!halted) {
            int k = R->k + 1;
            R->k = k;
            bool above = r2 > tol2 * R->v2;
            go = (above && k < kmax) ? 1u : 0u;
            if (!go) {
                R->cycles += (unsigned long long)k;
                R->applies += 1ull;
                if (above) R->hit_max = 1;
            }
        }
        cudaGraphSetConditional(h, go);
    }
}

// z = R_inf v on a capturing stream: the first cycle from z = 0, its residual
// and the decision, then a WHILE node whose body runs one more cycle, the
// correction, the residual and the decision.
static void rinf_enqueue(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s) {
    using O = LevelOps<double>;
    Level &L = p->L[0];
    const int64_t n = L.n;
    double2 *r = p->cyc_r.get(), *e = p->cyc_e.get();
    RinfDev *R = p->rinf_dev.get();
    double *part = p->rinf_part.get();
    const double *vol = p->mesh->volp.get();
    const double tol2 = RINF_TOL * RINF_TOL;
    note_launch(5);
    k_dnorm2_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, v, vol, part, stop);
    k_rinf_begin<<<1, RED_THREADS, 0, s>>>(R, part, stop);
    vcycle<double>(p, 0, v, z, stop, s);
    k_resid<double2, double><<<grid_for(n, 256), 256, 0, s>>>(n, O::A(L).view(), O::diag(L), v, z, nullptr, r, stop);
    k_dnorm2_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, r, vol, part, stop);
    GL_LAUNCH_CHECK();
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    GL_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h;
    GL_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
    k_rinf_decide<<<1, RED_THREADS, 0, s>>>(h, R, part, stop, tol2, RINF_MAXCYC);
    GL_LAUNCH_CHECK();
    GL_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    GL_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    GL_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t sb = p->rinf_body;
    GL_CUDA(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        vcycle<double>(p, 0, r, e, stop, sb);
        note_launch(4);
        k_axpy_t<double2><<<grid_for(n, 256), 256, 0, sb>>>(n, e, z, stop);
        k_resid<double2, double><<<grid_for(n, 256), 256, 0, sb>>>(n, O::A(L).view(), O::diag(L), v, z, nullptr,
                                                                    r, stop);
        k_dnorm2_part<<<RED_BLOCKS, RED_THREADS, 0, sb>>>(n, r, vol, part, stop);
        k_rinf_decide<<<1, RED_THREADS, 0, sb>>>(h, R, part, stop, tol2, RINF_MAXCYC);
        GL_LAUNCH_CHECK();
    } catch (...) {
        cudaStreamEndCapture(sb, &body);
        throw;
    }
    GL_CUDA(cudaStreamEndCapture(sb, &body));
}

// R_inf on any stream: inserted into the graph being captured, or (outside
// capture) captured into a graph of its own and launched once.  No event nodes
// of the profiler go into the loop body.
static void rinf_apply(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s) {
    Profiler &pr = profiler();
    const bool was_active = pr.active;
    pr.active = false;
    struct Restore {
        Profiler &pr;
        bool a;
        ~Restore() { pr.active = a; }
    } restore{pr, was_active};
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    GL_CUDA(cudaStreamIsCapturing(s, &st));
    if (st == cudaStreamCaptureStatusActive) {
        rinf_enqueue(p, v, z, stop, s);
        return;
    }
    cudaStream_t se = p->rinf_eager;
    GL_CUDA(cudaEventRecord(p->rinf_ev[0], s));
    GL_CUDA(cudaStreamWaitEvent(se, p->rinf_ev[0], 0));
    cudaGraph_t g = nullptr;
    GL_CUDA(cudaStreamBeginCapture(se, cudaStreamCaptureModeThreadLocal));
    try {
        rinf_enqueue(p, v, z, stop, se);
    } catch (...) {
        cudaStreamEndCapture(se, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    GL_CUDA(cudaStreamEndCapture(se, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    GL_CUDA(ie);
    cudaError_t le = cudaGraphLaunch(ex, se);
    cudaGraphExecDestroy(ex);  // released when the launch completes
    GL_CUDA(le);
    GL_CUDA(cudaEventRecord(p->rinf_ev[1], se));
    GL_CUDA(cudaStreamWaitEvent(s, p->rinf_ev[1], 0));
}

template <typename T>
static void precond_apply_t(gl_prec_s *p, const typename LevelOps<T>::C *v, typename LevelOps<T>::C *z,
                            const int *stop, cudaStream_t s) {
    using O = LevelOps<T>;
    using C = typename O::C;
    if (p->rinf) {
        if constexpr (sizeof(T) == 8) {
            rinf_apply(p, v, z, stop, s);
            return;
        } else {
            GL_REQUIRE(false, GL_ERR_ARG, "R_inf runs in FP64 only");
        }
    }
    if (p->cycles <= 1) {
        vcycle<T>(p, 0, v, z, stop, s);
    } else {
        // R_k: k steps of z <- z + V(v - (K + 2|psi|^2) z) from z = 0
        Level &L = p->L[0];
        C *r, *e;
        if constexpr (sizeof(T) == 8) {
            r = p->cyc_r.get();
            e = p->cyc_e.get();
        } else {
            r = p->cyc_r32.get();
            e = p->cyc_e32.get();
        }
        for (int k = 0; k < p->cycles; ++k) {
            if (k == 0) {
                vcycle<T>(p, 0, v, z, stop, s);
                continue;
            }
            note_launch(2);
            k_resid<C, T><<<grid_for(L.n, 256), 256, 0, s>>>(L.n, O::A(L).view(), O::diag(L), v, z, nullptr, r, stop);
            vcycle<T>(p, 0, r, e, stop, s);
            k_axpy_t<C><<<grid_for(L.n, 256), 256, 0, s>>>(L.n, e, z, stop);
        }
    }
    GL_LAUNCH_CHECK();
}

void precond_apply_p(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s) {
    precond_apply_t<double>(p, v, z, stop, s);
}
void precond_apply_p32(gl_prec_s *p, const float2 *v, float2 *z, const int *stop, cudaStream_t s) {
    precond_apply_t<float>(p, v, z, stop, s);
}
void precond_apply_p64_via32(gl_prec_s *p, const double2 *v, double2 *z, const int *stop, cudaStream_t s) {
    int64_t n = p->mesh->n;
    note_launch(2);
    k_d2f2<<<grid_for(n, 256), 256, 0, s>>>(n, v, p->mp_in.get(), stop);
    precond_apply_t<float>(p, p->mp_in.get(), p->mp_out.get(), stop, s);
    k_f2d<<<grid_for(n, 256), 256, 0, s>>>(n, p->mp_out.get(), z, stop);
    GL_LAUNCH_CHECK();
}

// CTAs of a neighbour-flag sweep by default: about 3/4 of a round of rows per
// CTA in the largest colour (the node-range partition spreads a colour unevenly)
template <typename T>
static int flags_default_nb(const Level &L, int G, int max_ctas) {
    int64_t maxc = 0;
    for (int c = 0; c < L.ncolors; ++c) maxc = std::max(maxc, L.cstart[c + 1] - L.cstart[c]);
    // rows per round of the flag sweep (its warp 0 only synchronises), three quarters full
    const int64_t per = std::max<int64_t>(1, (int64_t)((coop_threads<T>() - 32) / G) * 3 / 4);
    return (int)std::min<int64_t>(std::max<int64_t>((maxc + per - 1) / per, 1), max_ctas);
}

template <typename T>
static int flags_max_ctas_g(int G) {
    using C = typename LevelOps<T>::C;
    int r = 0;
    GL_DISPATCH_G(G, (r = flags_max_ctas<GG, C, T>()));
    return r;
}

static void zero_flags(Level &L, bool fp32, cudaStream_t s) {
    const size_t words = (size_t)MAX_FLAG_CTAS * FLAG_STRIDE;
    GL_CUDA(cudaMemsetAsync(L.flags.get() + (fp32 ? 0 : words), 0, words * sizeof(unsigned long long), s));
}

// chooses how every coarse level runs its symmetric Gauss-Seidel steps: the
// lanes-per-row width G (a latency-bound kernel wants more lanes per row than
// the throughput-bound SpMV that set the operator's own G), the synchronisation
// between colours (grid barrier, or neighbour flags with nb CTAs) and, in FP32,
// the thread-block-cluster sweep for levels whose vector fits a cluster.  With
// autotuning every candidate (G = 2, 4, 8, 16; the flags with CTAs in
// proportion to the level's largest colour) is timed on this GPU (best of two after
// a warm-up launch, on zero vectors) and the fastest kept; without it the
// operator's G, the flags where their partition fits (else the grid barrier),
// and the cluster sweep wherever it fits.  options.sweep_sync = 1 or 2 keeps
// only the grid-barrier or only the flag candidates (the flags fall back to the
// barrier where no partition fits).  All of them give the same rows for the
// same G.
template <typename T>
static void plan_sweeps_t(gl_prec_s *p, cudaStream_t s) {
    using O = LevelOps<T>;
    using C = typename O::C;
    constexpr bool fp32 = sizeof(T) == 4;
    cudaEvent_t e0, e1;
    GL_CUDA(cudaEventCreate(&e0));
    GL_CUDA(cudaEventCreate(&e1));
    const bool try_grid = p->sweep_sync != 2, try_flags = p->sweep_sync != 1;
    for (int l = 1; l < p->nlev - 1; ++l) {
        Level &L = p->L[l];
        const CsrG<C> &A = O::Ag(L);
        int &sG = fp32 ? L.sgs_G32 : L.sgs_G64;
        int &sync = fp32 ? L.sync32 : L.sync64;
        FlagPlan &F = fp32 ? L.fl32 : L.fl64;
        sG = A.G;
        sync = 0;
        F = FlagPlan{};
        if constexpr (fp32) {
            L.cl_size = 0;
            L.cl_chunk = 0;
        }
        int size = 0, chunk = 0;
        if constexpr (fp32) {
            if (p->cluster_sweeps && p->sweep_sync == 0 && L.n <= INT32_MAX)
                GL_DISPATCH_G(A.G, (plan_sgs_cluster<GG>(L.n, size, chunk)));
        }
        if (!p->autotune) {
            if (try_flags) {
                const int nb = flags_default_nb<T>(L, sG, flags_max_ctas_g<T>(sG));
                if (build_flag_plan<C>(L, A, sG, nb, F, s) <= FLAG_MAXN)
                    sync = 1;
                else
                    F = FlagPlan{};
            }
            if constexpr (fp32) {
                L.cl_size = size;
                L.cl_chunk = chunk;
            }
            zero_flags(L, fp32, s);
            continue;
        }
        int64_t maxc = 0;
        for (int c = 0; c < L.ncolors; ++c) maxc = std::max(maxc, L.cstart[c + 1] - L.cstart[c]);
        C *b = O::b(L), *x = O::x(L);
        GL_CUDA(cudaMemsetAsync(b, 0, L.n * sizeof(C), s));
        GL_CUDA(cudaMemsetAsync(x, 0, L.n * sizeof(C), s));
        auto time_it = [&](auto &&launch) {
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                GL_CUDA(cudaEventRecord(e0, s));
                launch();
                GL_CUDA(cudaEventRecord(e1, s));
                GL_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                GL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0) best = std::min(best, ms);
            }
            return best;
        };
        float best = 1e30f;
        int bestG = A.G, best_sync = 0, best_nb = 0;
        bool best_cluster = false;
        unsigned long long *flags = L.flags.get() + (fp32 ? 0 : (size_t)MAX_FLAG_CTAS * FLAG_STRIDE);
        for (int g : {2, 4, 8, 16}) {
            if (try_grid) {
                // a new grid size on this level's barrier counter: start it from zero
                GL_CUDA(cudaMemsetAsync(L.barrier.get(), 0, GRID_BARRIER_WORDS * sizeof(unsigned), s));
                float t = time_it([&] {
                    GL_DISPATCH_G(g, (launch_sgs_coop<GG, C, T>(A, O::diag(L), L.cstart_dev.get(), L.ncolors, b, x,
                                                                 0, L.barrier.get(), p->wait_extra.get(),
                                                                 p->err.get(), nullptr, maxc, s)));
                });
                if (t < best) best = t, bestG = g, best_sync = 0, best_cluster = false;
                if (verbose()) fprintf(stderr, "gl: level %d (n %lld, %d colours, %s) sweep G %d grid: %.1f us\n", l,
                                       (long long)L.n, L.ncolors, fp32 ? "FP32" : "FP64", g, 1e3 * t);
            }
            if (try_flags) {
                // CTAs in proportion to the level (never the whole GPU for a small
                // level: in a batch, instances' sweeps run side by side)
                const int nb0 = flags_default_nb<T>(L, g, flags_max_ctas_g<T>(g));
                for (int nb : {nb0}) {
                    FlagPlan cand;
                    const int longest = build_flag_plan<C>(L, A, g, nb, cand, s);
                    if (longest > FLAG_MAXN) {
                        if (verbose()) fprintf(stderr, "gl: level %d flags G %d nb %d: %d neighbours, too many\n", l,
                                               g, nb, longest);
                        continue;
                    }
                    zero_flags(L, fp32, s);
                    float t = time_it([&] {
                        GL_DISPATCH_G(g, (launch_sgs_flags<GG, C, T>(A, O::diag(L), L.cstart_dev.get(), L.ncolors,
                                                                      cand, b, x, 0, flags, p->wait_extra.get(),
                                                                      p->err.get(), nullptr, s)));
                    });
                    if (verbose())
                        fprintf(stderr, "gl: level %d sweep G %d flags nb %d (<= %d neighbours): %.1f us\n", l, g,
                                nb, longest, 1e3 * t);
                    if (t < best) {
                        best = t, bestG = g, best_sync = 1, best_nb = nb, best_cluster = false;
                        F = std::move(cand);
                    }
                }
            }
            if constexpr (fp32) {
                if (size > 0) {
                    float tc = time_it([&] {
                        GL_DISPATCH_G(g, (launch_sgs_cluster<GG>(A, O::diag(L), L.cstart_dev.get(), L.ncolors, b, x, 0,
                                                                  size, chunk, nullptr, s)));
                    });
                    if (tc < best) best = tc, bestG = g, best_cluster = true, best_sync = 0;
                    if (verbose()) fprintf(stderr, "gl: level %d cluster sweep G %d: %.1f us\n", l, g, 1e3 * tc);
                }
            }
        }
        sG = bestG;
        sync = best_sync;
        if (sync != 1) F = FlagPlan{};
        if (verbose())
            fprintf(stderr, "gl: level %d %s sweep: G %d%s%s (largest colour %lld rows)\n", l, fp32 ? "FP32" : "FP64",
                    bestG, best_cluster ? ", cluster" : "",
                    best_sync == 1 ? (std::string(", flags nb ") + std::to_string(best_nb)).c_str() : "",
                    (long long)maxc);
        // the timing ran other launch shapes on this level's counters
        GL_CUDA(cudaMemsetAsync(L.barrier.get(), 0, GRID_BARRIER_WORDS * sizeof(unsigned), s));
        zero_flags(L, fp32, s);
        GL_CUDA(cudaMemsetAsync(p->err.get(), 0, sizeof(int), s));
        if constexpr (fp32) {
            if (best_cluster) {
                L.cl_size = size;
                L.cl_chunk = chunk;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// the partitions of sweep choices taken over from a template (same sparsity)
template <typename T>
static void rebuild_flag_plans_t(gl_prec_s *p, const int *nbs, cudaStream_t s) {
    using O = LevelOps<T>;
    using C = typename O::C;
    constexpr bool fp32 = sizeof(T) == 4;
    for (int l = 1; l < p->nlev - 1; ++l) {
        Level &L = p->L[l];
        int &sync = fp32 ? L.sync32 : L.sync64;
        FlagPlan &F = fp32 ? L.fl32 : L.fl64;
        F = FlagPlan{};
        if (sync == 1) {
            const int G = fp32 ? L.sgs_G32 : L.sgs_G64;
            if (nbs[l] < 1 || nbs[l] > flags_max_ctas_g<T>(G) || build_flag_plan<C>(L, O::Ag(L), G, nbs[l], F, s) > FLAG_MAXN) {
                F = FlagPlan{};
                sync = 0;
            }
        }
        zero_flags(L, fp32, s);
    }
}

void rebuild_flag_plans(gl_prec_s *p, bool fp32, cudaStream_t s) {
    int nbs[MAX_LEVELS];
    for (int l = 0; l < MAX_LEVELS; ++l) nbs[l] = fp32 ? p->tuned[l].nb32 : p->tuned[l].nb64;
    if (fp32)
        rebuild_flag_plans_t<float>(p, nbs, s);
    else
        rebuild_flag_plans_t<double>(p, nbs, s);
}

void sweeps_reset(gl_prec_s *p, cudaStream_t s) {
    for (int l = 1; l < p->nlev - 1; ++l) {
        Level &L = p->L[l];
        if (L.barrier.get()) GL_CUDA(cudaMemsetAsync(L.barrier.get(), 0, GRID_BARRIER_WORDS * sizeof(unsigned), s));
        if (L.flags.get()) GL_CUDA(cudaMemsetAsync(L.flags.get(), 0, L.flags.bytes(), s));
    }
    GL_CUDA(cudaMemsetAsync(p->err.get(), 0, sizeof(int), s));
    GL_CUDA(cudaMemsetAsync(p->wait_extra.get(), 0, sizeof(unsigned long long), s));
}

int sweeps_failed(gl_prec_s *p, cudaStream_t s) {
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, p->err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return h;
}

void plan_sweeps(gl_prec_s *p, bool fp32, cudaStream_t s) {
    if (fp32)
        plan_sweeps_t<float>(p, s);
    else
        plan_sweeps_t<double>(p, s);
}

}  // namespace gl
