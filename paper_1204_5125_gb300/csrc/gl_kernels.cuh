// gl_kernels.cuh -- device building blocks shared by the operator, V-cycle and
// Krylov kernels.
#pragma once

#include "gl_internal.cuh"

namespace gl {

// ---- double-FP32 arithmetic (hi + lo FP32 pairs, about 48 significant bits)
__device__ __forceinline__ float2 split_df(double x) {
    float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}
// (s, c) += p exactly: s + p = t + e (TwoSum), the error e joins the compensation c
__device__ __forceinline__ void dot2_add(float &s, float &c, float p) {
    float t = __fadd_rn(s, p);
    float bp = __fadd_rn(t, -s);
    float e = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -bp)), __fadd_rn(p, -bp));
    s = t;
    c = __fadd_rn(c, e);
}
// (s, c) += a b, a = a.x + a.y: the exact product of the high part (TwoProd) and
// the low part's product into the compensation
__device__ __forceinline__ void dot2_df(float &s, float &c, float2 a, float b) {
    float p = __fmul_rn(a.x, b);
    float e = __fmaf_rn(a.x, b, -p);
    dot2_add(s, c, p);
    c = __fadd_rn(c, e);
    c = __fmaf_rn(a.y, b, c);
}


// sum_k A[p][k] * x[col[p][k]] over the stored off-diagonals of row p of a sliced
// ELL matrix (a warp reads 32 consecutive entries per k)
template <typename C, typename X>
__device__ __forceinline__ C sell_row(const SellView<C> &A, int64_t p, const X *__restrict__ x) {
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = __ldg(A.sptr + s);
    int w = (int)((__ldg(A.sptr + s + 1) - beg) >> 5);
    const int32_t *cp = A.col + beg + lane;
    const C *vp = A.val + beg + lane;
    C acc;
    acc.x = 0;
    acc.y = 0;
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
        int32_t c = __ldg(cp + (int64_t)k * SELL_C);
        C a = vp[(int64_t)k * SELL_C];
        X xv = x[c];
        C xc;
        xc.x = xv.x;
        xc.y = xv.y;
        cfma(acc, a, xc);
    }
    return acc;
}

// same, over the columns below `lo` only: on the first Gauss-Seidel pass from a
// zero guess the colours before the current one hold values, the current colour
// has no couplings to itself (a proper colouring) and the later colours are
// still zero.  Padding entries point at the row itself, which lies in the
// current colour, so they are skipped too (its x is not yet written).
template <typename C, typename X>
__device__ __forceinline__ C sell_row_before(const SellView<C> &A, int64_t p, const X *__restrict__ x, int64_t lo) {
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = __ldg(A.sptr + s);
    int w = (int)((__ldg(A.sptr + s + 1) - beg) >> 5);
    const int32_t *cp = A.col + beg + lane;
    const C *vp = A.val + beg + lane;
    C acc;
    acc.x = 0;
    acc.y = 0;
    for (int k = 0; k < w; ++k) {
        int32_t c = __ldg(cp + (int64_t)k * SELL_C);
        if (c >= lo) continue;
        C a = vp[(int64_t)k * SELL_C];
        X xv = x[c];
        C xc;
        xc.x = xv.x;
        xc.y = xv.y;
        cfma(acc, a, xc);
    }
    return acc;
}

// Jacobian row given the off-diagonal sum: acc + (K_ii - 1 + 2|psi|^2) phi + psi^2 conj(phi)
template <typename C, typename R>
__device__ __forceinline__ C jacobian_epilogue(C acc, R kd, C ps, C ph) {
    R a2 = ps.x * ps.x + ps.y * ps.y;
    R d = kd - (R)1 + (R)2 * a2;
    C p2 = mk(ps.x * ps.x - ps.y * ps.y, (R)2 * ps.x * ps.y);  // psi^2
    C r;
    r.x = acc.x + d * ph.x + (p2.x * ph.x + p2.y * ph.y);  // psi^2 conj(phi): (a+ib)(c-id)
    r.y = acc.y + d * ph.y + (p2.y * ph.x - p2.x * ph.y);
    return r;
}

// sum_{k != p} K_pk x_k with the tabulated finest-level stencil (FP32) at solve
// position p of an even-N lattice: red nodes ((i + j + k) even) first, node v of
// either colour at position v / 2 within its colour, neighbours of the other
// colour; K-hat of a +e edge from the per-axis table at the perpendicular
// position, its conjugate for the -e edge; the row scaled by 1 / |V_p|.
template <typename F>
__device__ __forceinline__ float2 lattice_row_f(const LatticeView &L, int64_t p, F xval);

__device__ __forceinline__ float2 lattice_row(const LatticeView &L, int64_t p, const float2 *__restrict__ x) {
    return lattice_row_f(L, p, [x](int64_t q) { return x[q]; });
}

// the same with the neighbour values supplied by xval(position)
template <typename F>
__device__ __forceinline__ float2 lattice_row_f(const LatticeView &L, int64_t p, F xval) {
    const uint32_t c = p >= L.nred ? 1u : 0u;
    const uint32_t N = (uint32_t)L.N;
    uint32_t v = 2u * (uint32_t)(p - (c ? L.nred : 0));
    const uint32_t r = L.dN.div(v), k = L.dN.div(r);
    uint32_t i = v - r * N;
    const uint32_t j = r - k * N;
    if (((i + j + k) & 1u) != c) {
        ++v;
        ++i;
    }
    const int64_t other = c ? 0 : L.nred;
    float2 acc = make_float2(0.f, 0.f);
    // acc += t x_u (plus) or conj(t) x_u (minus)
    auto edge = [&](float2 t, uint32_t u, bool plus) {
        const float2 xv = xval((int64_t)(u >> 1) + other);
        const float ty = plus ? t.y : -t.y;
        acc.x += t.x * xv.x - ty * xv.y;
        acc.y += t.x * xv.y + ty * xv.x;
    };
    {
        const float2 t = __ldg(L.tx + (j + N * k));
        if (i + 1 < N) edge(t, v + 1, true);
        if (i > 0) edge(t, v - 1, false);
    }
    {
        const float2 t = __ldg(L.ty + (i + N * k));
        if (j + 1 < N) edge(t, v + N, true);
        if (j > 0) edge(t, v - N, false);
    }
    if (L.dim == 3) {
        const float2 t = __ldg(L.tz + (i + N * j));
        if (k + 1 < N) edge(t, v + N * N, true);
        if (k > 0) edge(t, v - N * N, false);
    }
    const float iv = 1.f / L.vol[p];
    return make_float2(acc.x * iv, acc.y * iv);
}

// sum_{k != p} K_pk x_k in FP64 from the FP64 tables (same layout, edge order and
// conjugation as lattice_row_f), the row scaled by 1 / |V_p| = 2^b / h^d (b the
// node's boundary coordinates; no division: this kernel is bound by the FP64 pipe)
__device__ __forceinline__ double2 lattice_row64(const LatticeView64 &L, int64_t p, const double2 *__restrict__ x) {
    const uint32_t c = p >= L.nred ? 1u : 0u;
    const uint32_t N = (uint32_t)L.N;
    uint32_t v = 2u * (uint32_t)(p - (c ? L.nred : 0));
    const uint32_t r = L.dN.div(v), k = L.dN.div(r);
    uint32_t i = v - r * N;
    const uint32_t j = r - k * N;
    if (((i + j + k) & 1u) != c) {
        ++v;
        ++i;
    }
    const int64_t other = c ? 0 : L.nred;
    double2 acc = make_double2(0.0, 0.0);
    auto edge = [&](double2 t, uint32_t u, bool plus) {
        const double2 xv = x[(int64_t)(u >> 1) + other];
        const double ty = plus ? t.y : -t.y;
        acc.x += t.x * xv.x - ty * xv.y;
        acc.y += t.x * xv.y + ty * xv.x;
    };
    {
        const double2 t = __ldg(L.tx + (j + N * k));
        if (i + 1 < N) edge(t, v + 1, true);
        if (i > 0) edge(t, v - 1, false);
    }
    {
        const double2 t = __ldg(L.ty + (i + N * k));
        if (j + 1 < N) edge(t, v + N, true);
        if (j > 0) edge(t, v - N, false);
    }
    if (L.dim == 3) {
        const double2 t = __ldg(L.tz + (i + N * j));
        if (k + 1 < N) edge(t, v + N * N, true);
        if (k > 0) edge(t, v - N * N, false);
    }
    const int b = (i == 0 || i == N - 1) + (j == 0 || j == N - 1) + (L.dim == 3 && (k == 0 || k == N - 1));
    const double iv = L.ihd * (double)(1 << b);
    return make_double2(acc.x * iv, acc.y * iv);
}

}  // namespace gl
