// gl_setup.cu -- GPU setup of R_k(psi) = AMG_k(K-hat + 2 D |psi|^2, D .)
// (Eq. prec2, Sec. 4.1): smoothed-aggregation AMG with symmetric Gauss-Seidel.
// Every step runs in the kernels below; the host only sequences them.
//   * strength: every off-diagonal is a strong connection (threshold 0)
//   * aggregation: distance-2 maximal independent set in synchronous Luby rounds
//     with fixed hash priorities (Bell, Dalton & Olson 2012); roots numbered in
//     ascending node order; neighbours of a root join it; the rest join the
//     neighbouring aggregate with the smallest id
//   * tentative prolongator from the candidate B (B = 1 on the finest level,
//     aggregate norms below); P = (I - omega D^-1 A) P_tent, omega = 4/(3 rho),
//     rho from power iterations on D^-1 A and a D-Rayleigh quotient
//   * Galerkin A_c = P^H A P by a two-phase row-wise SpGEMM (hash symbolic pass,
//     deterministic numeric pass), made exactly Hermitian as (A_c + A_c^H)/2
//   * colours: red-black on the lattice level, Jones-Plassmann below
//   * coarsest level: dense FP64 inverse by Gauss-Jordan elimination
#include <atomic>

#include <chrono>

#include "gl_internal.cuh"

namespace gl {

// ------------------------------------------------------------------ priorities
// "lowbias32" integer mixer (C. Wellons) of the node id, paired with the id
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint64_t prio(int64_t i) {
    return ((((uint64_t)mix32((uint32_t)i)) << 32) | (uint64_t)(uint32_t)i) + 1ull;
}

// ------------------------------------------------------------------ level 0 operator
// A_can = K-hat + 2 D |psi|^2 (diagonal update only)
__global__ void k_add_diag(int64_t n, const int64_t *rp, const int32_t *ci, double2 *v, const double *vol,
                           const double2 *psi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (ci[q] == i) {
            double2 p = psi[i];
            v[q].x += 2.0 * vol[i] * (p.x * p.x + p.y * p.y);
        }
}

// ------------------------------------------------------------------ MIS(2) aggregation
enum : uint8_t { UNDECIDED = 0, ROOT = 1, OUT = 2 };

__global__ void k_mis_key(int64_t n, const uint8_t *state, uint64_t *key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) key[i] = (state[i] == UNDECIDED) ? prio(i) : 0ull;
}
__global__ void k_mis_max1(int64_t n, const int64_t *rp, const int32_t *ci, const uint64_t *key, uint64_t *m1) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) k = max(k, key[ci[q]]);
    m1[i] = k;
}
__global__ void k_mis_max2(int64_t n, const int64_t *rp, const int32_t *ci, const uint64_t *key, const uint64_t *m1,
                           uint8_t *state, uint8_t *newroot) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = m1[i];
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) k = max(k, m1[ci[q]]);
    uint8_t nr = (state[i] == UNDECIDED && key[i] == k) ? 1 : 0;
    newroot[i] = nr;
    if (nr) state[i] = ROOT;
}
__global__ void k_mis_d1(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *newroot, uint8_t *d1) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t f = newroot[i];
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) f |= newroot[ci[q]];
    d1[i] = f;
}
__global__ void k_mis_d2(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *d1, uint8_t *state,
                         uint8_t *undecided) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] != UNDECIDED) {
        undecided[i] = 0;
        return;
    }
    uint8_t f = d1[i];
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) f |= d1[ci[q]];
    if (f) state[i] = OUT;
    undecided[i] = f ? 0 : 1;
}
__global__ void k_root_flag(int64_t n, const uint8_t *state, int64_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (state[i] == ROOT) ? 1 : 0;
}
__global__ void k_agg_first(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *state,
                            const int64_t *rank, int32_t *first) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = -1;
    if (state[i] == ROOT) {
        a = (int32_t)rank[i];
    } else {
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
            if (state[ci[q]] == ROOT) a = (int32_t)rank[ci[q]];
    }
    first[i] = a;
}
__global__ void k_agg_final(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *first, int32_t *agg,
                            int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = first[i];
    if (a < 0)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int32_t b = first[ci[q]];
            if (b >= 0 && (a < 0 || b < a)) a = b;
        }
    if (a < 0) atomicExch(err, 1);
    agg[i] = a;
}

static int64_t aggregate(const CsrDev &A, int32_t *agg, cudaStream_t s) {
    int64_t n = A.n;
    DBuf<uint8_t> state(n), newroot(n), d1(n), und(n);
    DBuf<uint64_t> key(n), m1(n);
    GL_CUDA(cudaMemsetAsync(state.get(), 0, n, s));
    int G = grid_for(n, 256);
    for (int round = 0;; ++round) {
        GL_REQUIRE(round < 10000, GL_ERR_CAPACITY, "aggregation did not terminate");
        k_mis_key<<<G, 256, 0, s>>>(n, state.get(), key.get());
        k_mis_max1<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), key.get(), m1.get());
        k_mis_max2<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), key.get(), m1.get(), state.get(), newroot.get());
        k_mis_d1<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), newroot.get(), d1.get());
        k_mis_d2<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), d1.get(), state.get(), und.get());
        GL_LAUNCH_CHECK();
        if (count_nonzero_u8(und.get(), n, s) == 0) break;
    }
    DBuf<int64_t> rank(n + 1);
    DBuf<int32_t> first(n);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    k_root_flag<<<G, 256, 0, s>>>(n, state.get(), rank.get());
    GL_LAUNCH_CHECK();
    scan_exclusive(rank.get(), rank.get(), n, true, s);
    int64_t nagg = 0;
    GL_CUDA(cudaMemcpyAsync(&nagg, rank.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    k_agg_first<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), state.get(), rank.get(), first.get());
    k_agg_final<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), first.get(), agg, err.get());
    GL_LAUNCH_CHECK();
    int herr = 0;
    GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(herr == 0, GL_ERR_CAPACITY, "aggregation left a node unassigned");
    return nagg;
}

// ------------------------------------------------------------------ Jones-Plassmann colouring
__global__ void k_jp_pick(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *color, uint8_t *pick) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t ok = 0;
    if (color[i] < 0) {
        ok = 1;
        uint64_t k = prio(i);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int64_t j = ci[q];
            if (j != i && color[j] < 0 && prio(j) > k) ok = 0;
        }
    }
    pick[i] = ok;
}
__global__ void k_jp_assign(int64_t n, const int64_t *rp, const int32_t *ci, const uint8_t *pick, int32_t *color,
                            uint8_t *left, int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (pick[i]) {
        uint64_t used[4] = {0, 0, 0, 0};
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int64_t j = ci[q];
            int32_t c = color[j];
            if (j != i && c >= 0 && c < 256) used[c >> 6] |= 1ull << (c & 63);
        }
        int c = 0;
        while (c < 256 && (used[c >> 6] >> (c & 63)) & 1ull) ++c;
        if (c >= 256) atomicExch(err, 1);
        color[i] = c;
        left[i] = 0;
    } else {
        left[i] = color[i] < 0 ? 1 : 0;
    }
}
__global__ void k_fill_i32(int64_t n, int32_t *x, int32_t v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}
__global__ void k_max_i32(const int32_t *x, int64_t n, int32_t *out) {
    __shared__ int32_t sh[256];
    int32_t m = -1;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = max(m, x[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

static int color_jp(const CsrDev &A, int32_t *color, cudaStream_t s) {
    int64_t n = A.n;
    DBuf<uint8_t> pick(n), left(n);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    int G = grid_for(n, 256);
    k_fill_i32<<<G, 256, 0, s>>>(n, color, -1);
    for (int round = 0;; ++round) {
        GL_REQUIRE(round < 100000, GL_ERR_CAPACITY, "colouring did not terminate");
        k_jp_pick<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), color, pick.get());
        k_jp_assign<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), pick.get(), color, left.get(), err.get());
        GL_LAUNCH_CHECK();
        if (count_nonzero_u8(left.get(), n, s) == 0) break;
    }
    DBuf<int32_t> mx(1);
    k_max_i32<<<1, 256, 0, s>>>(color, n, mx.get());
    GL_LAUNCH_CHECK();
    int32_t hm = 0;
    int herr = 0;
    GL_CUDA(cudaMemcpyAsync(&hm, mx.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(herr == 0, GL_ERR_CAPACITY, "more than 256 colours needed");
    return hm + 1;
}

// Smallest-last colouring in removal rounds, on the device (the default):
// round r removes every remaining vertex whose remaining degree is within
// PSL_SLACK of the round's smallest (degrees as at the start of the round) and
// gives it level r; then Jones-Plassmann rounds with the key (level, prio)
// colour each vertex once all its higher-key neighbours are coloured, with the
// smallest colour none of them has - the greedy colouring in decreasing key
// order (a later-removed vertex first).  Few rounds in both phases (a few
// hundred on the 128^3 cube's level 1) and the one-at-a-time order's colour
// count there.
constexpr int PSL_SLACK = 4;
constexpr int PSL_BATCH = 32;  // rounds launched between two checks of the host

__global__ void k_psl_deg(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *deg, int32_t *level) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t d = 0;
    for (int64_t q = rp[v]; q < rp[v + 1]; ++q) d += (ci[q] != v);
    deg[v] = d;
    level[v] = -1;
}
__global__ void k_psl_min(int64_t n, const int32_t *level, const int32_t *deg, int32_t *mn) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n && level[v] < 0) atomicMin(mn, deg[v]);
}
__global__ void k_psl_mark(int64_t n, int32_t *level, const int32_t *deg, const int32_t *mn, int32_t r) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t m = *mn;
    if (v < n && m != INT32_MAX && level[v] < 0 && deg[v] <= m + PSL_SLACK) level[v] = r;
}
__global__ void k_psl_dec(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *level, int32_t *deg,
                          int32_t r) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n || level[v] != r) return;
    for (int64_t q = rp[v]; q < rp[v + 1]; ++q) {
        const int32_t u = ci[q];
        if (u != v && level[u] < 0) atomicSub(deg + u, 1);
    }
}
__global__ void k_psl_alive(int64_t n, const int32_t *level, uint8_t *alive) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) alive[v] = level[v] < 0 ? 1 : 0;
}
// an uncoloured vertex is picked when no uncoloured neighbour has a higher (level, prio) key
__global__ void k_jpl_pick(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *level,
                           const int32_t *color, uint8_t *pick) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t ok = 0;
    if (color[i] < 0) {
        ok = 1;
        const int32_t li = level[i];
        const uint64_t ki = prio(i);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            const int64_t j = ci[q];
            if (j != i && color[j] < 0 && (level[j] > li || (level[j] == li && prio(j) > ki))) ok = 0;
        }
    }
    pick[i] = ok;
}

static int color_psl(const CsrDev &A, int32_t *color, cudaStream_t s) {
    const int64_t n = A.n;
    const int G = grid_for(n, 256);
    DBuf<int32_t> deg(n), level(n), mn(PSL_BATCH);
    DBuf<uint8_t> flag(n), pick(n);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    k_psl_deg<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), deg.get(), level.get());
    GL_LAUNCH_CHECK();
    int32_t r = 0;
    for (;;) {
        GL_REQUIRE(r <= n + PSL_BATCH, GL_ERR_CAPACITY, "colouring rounds did not terminate");
        k_fill_i32<<<1, PSL_BATCH, 0, s>>>(PSL_BATCH, mn.get(), INT32_MAX);
        for (int k = 0; k < PSL_BATCH; ++k, ++r) {
            k_psl_min<<<G, 256, 0, s>>>(n, level.get(), deg.get(), mn.get() + k);
            k_psl_mark<<<G, 256, 0, s>>>(n, level.get(), deg.get(), mn.get() + k, r);
            k_psl_dec<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), level.get(), deg.get(), r);
        }
        GL_LAUNCH_CHECK();
        k_psl_alive<<<G, 256, 0, s>>>(n, level.get(), flag.get());
        if (count_nonzero_u8(flag.get(), n, s) == 0) break;
    }
    k_fill_i32<<<G, 256, 0, s>>>(n, color, -1);
    for (int round = 0;; round += 8) {
        GL_REQUIRE(round <= n + 8, GL_ERR_CAPACITY, "colouring did not terminate");
        for (int k = 0; k < 8; ++k) {
            k_jpl_pick<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), level.get(), color, pick.get());
            k_jp_assign<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), pick.get(), color, flag.get(), err.get());
        }
        GL_LAUNCH_CHECK();
        if (count_nonzero_u8(flag.get(), n, s) == 0) break;
    }
    DBuf<int32_t> mx(1);
    k_max_i32<<<1, 256, 0, s>>>(color, n, mx.get());
    GL_LAUNCH_CHECK();
    int32_t hm = 0;
    int herr = 0;
    GL_CUDA(cudaMemcpyAsync(&hm, mx.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(herr == 0, GL_ERR_CAPACITY, "more than 256 colours needed");
    return hm + 1;
}

// Smallest-last greedy colouring (Matula & Beck) of the level graph, on the
// host (option GL_COLOR_SL): a sequential order whose colour count is bounded by the graph's
// degeneracy + 1 (fewer colours, so fewer dependent phases in every
// multicolour sweep, than the parallel Jones-Plassmann colouring).  The order
// is deterministic: vertices wait in degree buckets (intrusive lists; entered
// in ascending id, each at the head), the head of the lowest non-empty bucket
// leaves next, and each of its remaining neighbours, in row order, moves to the
// head of the bucket one degree lower.  Colouring runs from the last vertex to
// leave to the first, each taking the smallest colour none of its coloured
// neighbours has.
int colour_graph_psl(const CsrDev &A, int32_t *color, cudaStream_t s) { return color_psl(A, color, s); }

static int color_smallest_last(const CsrDev &A, int32_t *color_dev, cudaStream_t s) {
    const int64_t n = A.n;
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> ci(A.nnz > 0 ? A.nnz : 1);
    GL_CUDA(cudaMemcpyAsync(rp.data(), A.rp.get(), (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (A.nnz > 0)
        GL_CUDA(cudaMemcpyAsync(ci.data(), A.ci.get(), A.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> d(n, 0);
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t q = rp[v]; q < rp[v + 1]; ++q) d[v] += (ci[q] != v);
        dmax = std::max(dmax, d[v]);
    }
    std::vector<int64_t> first(dmax + 1, -1), nxt(n, -1), prv(n, -1);
    auto unlink = [&](int64_t v) {
        if (prv[v] >= 0)
            nxt[prv[v]] = nxt[v];
        else
            first[d[v]] = nxt[v];
        if (nxt[v] >= 0) prv[nxt[v]] = prv[v];
    };
    auto push = [&](int64_t v) {
        prv[v] = -1;
        nxt[v] = first[d[v]];
        if (nxt[v] >= 0) prv[nxt[v]] = v;
        first[d[v]] = v;
    };
    for (int64_t v = 0; v < n; ++v) push(v);
    std::vector<int32_t> seq(n);
    std::vector<char> out(n, 0);
    int64_t b = 0;
    for (int64_t k = 0; k < n; ++k) {
        while (first[b] < 0) ++b;
        const int64_t v = first[b];
        unlink(v);
        out[v] = 1;
        seq[n - 1 - k] = (int32_t)v;
        for (int64_t q = rp[v]; q < rp[v + 1]; ++q) {
            const int64_t u = ci[q];
            if (u == v || out[u]) continue;
            unlink(u);
            --d[u];
            push(u);
        }
        b = b > 0 ? b - 1 : 0;
    }
    std::vector<int32_t> col(n, -1);
    std::vector<int64_t> seen(dmax + 2, -1);
    int32_t ncol = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t v = seq[k];
        for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
            if (ci[q] != v && col[ci[q]] >= 0) seen[col[ci[q]]] = v;
        int32_t c = 0;
        while (seen[c] == v) ++c;
        col[v] = c;
        ncol = std::max(ncol, c + 1);
    }
    GL_REQUIRE(ncol <= 256, GL_ERR_CAPACITY, "more than 256 colours needed");
    GL_CUDA(cudaMemcpyAsync(color_dev, col.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return ncol;
}

// ------------------------------------------------------------------ candidate norms
// members of each aggregate (the pattern of P_tent^T), sorted by node id
__global__ void k_count_cols(int64_t nnz, const int32_t *col, int64_t *cnt) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nnz) atomicAdd((unsigned long long *)(cnt + col[q]), 1ull);
}
__global__ void k_agg_members(int64_t n, const int32_t *agg, const int64_t *rp, int64_t *fill, int32_t *mem) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = agg[i];
    int64_t pos = rp[a] + (int64_t)atomicAdd((unsigned long long *)(fill + a), 1ull);
    mem[pos] = (int32_t)i;
}
__global__ void k_sort_small_i32(int64_t nrows, const int64_t *rp, int32_t *x) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int64_t a = rp[r] + 1; a < rp[r + 1]; ++a) {
        int32_t k = x[a];
        int64_t b = a - 1;
        while (b >= rp[r] && x[b] > k) {
            x[b + 1] = x[b];
            --b;
        }
        x[b + 1] = k;
    }
}
__global__ void k_bnorm(int64_t nc, const int64_t *rp, const int32_t *mem, const double *B, double *bn) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double s = 0;
    for (int64_t q = rp[c]; q < rp[c + 1]; ++q) s += B[mem[q]] * B[mem[q]];
    bn[c] = sqrt(s);
}

// ------------------------------------------------------------------ spectral radius of D^-1 A
__global__ void k_pow_init(int64_t n, double2 *x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = make_double2(1.0 + (double)(i % 7) / 7.0, 0.0);
}
__global__ void k_diag_of(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, double *d) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double r = 0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (ci[q] == i) r = v[q].x;
    d[i] = r;
}
// y = D^-1 A x, per-block partial of ||y||^2
__global__ void k_pow_step(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, const double *d,
                           const double2 *x, double2 *y, double *part) {
    __shared__ double sh[32];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 s = make_double2(0, 0);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) cfma(s, v[q], x[ci[q]]);
        double2 yi = make_double2(s.x / d[i], s.y / d[i]);
        y[i] = yi;
        acc += yi.x * yi.x + yi.y * yi.y;
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_sum_parts(const double *part, int np, double *out, int sqrt_it) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) *out = sqrt_it ? sqrt(t) : t;
}
__global__ void k_pow_scale(int64_t n, const double2 *y, const double *nrm, double2 *x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        double s = 1.0 / *nrm;
        x[i] = make_double2(y[i].x * s, y[i].y * s);
    }
}
// partials of Re(x^H A x) and x^H D x
__global__ void k_rayleigh(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, const double *d,
                           const double2 *x, double *pnum, double *pden) {
    __shared__ double sh[32];
    double an = 0, ad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 s = make_double2(0, 0);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) cfma(s, v[q], x[ci[q]]);
        double2 xi = x[i];
        an += xi.x * s.x + xi.y * s.y;
        ad += d[i] * (xi.x * xi.x + xi.y * xi.y);
    }
    double t = block_sum(an, sh);
    double u = block_sum(ad, sh);
    if (threadIdx.x == 0) {
        pnum[blockIdx.x] = t;
        pden[blockIdx.x] = u;
    }
}

static double spectral_radius(const CsrDev &A, int its, cudaStream_t s) {
    int64_t n = A.n;
    DBuf<double2> x(n), y(n);
    DBuf<double> d(n), part(2 * RED_BLOCKS), sc(3);
    int G = grid_for(n, 256);
    k_pow_init<<<G, 256, 0, s>>>(n, x.get());
    k_diag_of<<<G, 256, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), d.get());
    for (int it = 0; it < its; ++it) {
        k_pow_step<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), d.get(), x.get(), y.get(),
                                                      part.get());
        k_sum_parts<<<1, 1024, 0, s>>>(part.get(), RED_BLOCKS, sc.get(), 1);
        k_pow_scale<<<G, 256, 0, s>>>(n, y.get(), sc.get(), x.get());
    }
    k_rayleigh<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), d.get(), x.get(), part.get(),
                                                  part.get() + RED_BLOCKS);
    k_sum_parts<<<1, 1024, 0, s>>>(part.get(), RED_BLOCKS, sc.get() + 1, 0);
    k_sum_parts<<<1, 1024, 0, s>>>(part.get() + RED_BLOCKS, RED_BLOCKS, sc.get() + 2, 0);
    GL_LAUNCH_CHECK();
    double h[3];
    GL_CUDA(cudaMemcpyAsync(h, sc.get(), 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return h[1] / h[2];
}

// ------------------------------------------------------------------ smoothed prolongator
constexpr int MAX_ROW_AGGS = 256;

// number of distinct aggregates among the nodes of row i (diagonal included)
__global__ void k_p_count(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *agg, int64_t *len,
                          int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t seen[MAX_ROW_AGGS];
    int cnt = 0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        int32_t a = agg[ci[q]];
        bool dup = false;
        for (int t = 0; t < cnt; ++t)
            if (seen[t] == a) dup = true;
        if (!dup) {
            if (cnt >= MAX_ROW_AGGS) {
                atomicExch(err, 1);
                break;
            }
            seen[cnt++] = a;
        }
    }
    len[i] = cnt;
}
// P_ic = [c == agg(i)] B_i / bn_c - omega / A_ii sum_{j in row i, agg(j) = c} A_ij B_j / bn_c
__global__ void k_p_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, const int32_t *agg,
                         const double *B, const double *bn, double omega, const int64_t *prp, int32_t *pci,
                         double2 *pv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t base = prp[i];
    int cnt = (int)(prp[i + 1] - base);
    double dii = 0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (ci[q] == i) dii = v[q].x;
    // build the sorted distinct list
    int filled = 0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        int32_t a = agg[ci[q]];
        int pos = 0;
        bool dup = false;
        for (; pos < filled; ++pos) {
            int32_t b = pci[base + pos];
            if (b == a) {
                dup = true;
                break;
            }
            if (b > a) break;
        }
        if (dup) continue;
        for (int t = filled; t > pos; --t) pci[base + t] = pci[base + t - 1];
        pci[base + pos] = a;
        ++filled;
    }
    for (int t = 0; t < cnt; ++t) {
        int32_t c = pci[base + t];
        double2 acc = make_double2(0, 0);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int64_t j = ci[q];
            if (agg[j] != c) continue;
            double pt = B[j] / bn[c];
            acc.x += v[q].x * pt;
            acc.y += v[q].y * pt;
        }
        double pt_i = (agg[i] == c) ? B[i] / bn[c] : 0.0;
        pv[base + t] = make_double2(pt_i - omega / dii * acc.x, -omega / dii * acc.y);
    }
}

// ------------------------------------------------------------------ transpose (conjugate)
__global__ void k_tr_fill(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, const int64_t *trp,
                          int64_t *fill, int32_t *tci, double2 *tv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        int32_t c = ci[q];
        int64_t pos = trp[c] + (int64_t)atomicAdd((unsigned long long *)(fill + c), 1ull);
        tci[pos] = (int32_t)i;
        tv[pos] = make_double2(v[q].x, -v[q].y);
    }
}
__global__ void k_rowlen_max(int64_t n, const int64_t *rp, int64_t *part) {
    __shared__ int64_t sh[256];
    int64_t m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, rp[i + 1] - rp[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
static int64_t max_i64_parts(const int64_t *part, int np, cudaStream_t s) {
    std::vector<int64_t> h(np);
    GL_CUDA(cudaMemcpyAsync(h.data(), part, np * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    int64_t m = 0;
    for (auto x : h) m = std::max(m, x);
    return m;
}
static int64_t max_row_len(const CsrDev &A, cudaStream_t s) {
    DBuf<int64_t> part(256);
    k_rowlen_max<<<256, 256, 0, s>>>(A.n, A.rp.get(), part.get());
    GL_LAUNCH_CHECK();
    return max_i64_parts(part.get(), 256, s);
}

static void transpose_conj(const CsrDev &A, CsrDev &T, cudaStream_t s) {
    T.n = A.m;
    T.m = A.n;
    T.nnz = A.nnz;
    DBuf<int64_t> cnt(T.n + 1), fill(T.n + 1);
    GL_CUDA(cudaMemsetAsync(cnt.get(), 0, (T.n + 1) * sizeof(int64_t), s));
    GL_CUDA(cudaMemsetAsync(fill.get(), 0, (T.n + 1) * sizeof(int64_t), s));
    k_count_cols<<<grid_for(A.nnz, 256), 256, 0, s>>>(A.nnz, A.ci.get(), cnt.get());
    GL_LAUNCH_CHECK();
    T.rp.alloc(T.n + 1);
    scan_exclusive(cnt.get(), T.rp.get(), T.n, true, s);
    T.ci.alloc(T.nnz > 0 ? T.nnz : 1);
    T.v.alloc(T.nnz > 0 ? T.nnz : 1);
    k_tr_fill<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), A.v.get(), T.rp.get(), fill.get(),
                                                 T.ci.get(), T.v.get());
    GL_LAUNCH_CHECK();
    sort_rows_by_col(T.n, T.rp.get(), T.ci.get(), T.v.get(), max_row_len(T, s), s);
    GL_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ SpGEMM C = A B
// products per row of C
__global__ void k_sg_prod(int64_t n, const int64_t *arp, const int32_t *aci, const int64_t *brp, int64_t *prod) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t t = 0;
    for (int64_t q = arp[i]; q < arp[i + 1]; ++q) t += brp[aci[q] + 1] - brp[aci[q]];
    prod[i] = t;
}

constexpr int32_t HASH_EMPTY = -1;

__device__ __forceinline__ int hash_slots(int64_t prod, int64_t ncols, int cap) {
    int64_t u = prod < ncols ? prod : ncols;
    int h = 32;
    while (h < 2 * u && h < cap) h <<= 1;
    return h;
}

// insert every product column of row i into a shared open-addressing table;
// returns the number of distinct columns (block-uniform)
__device__ int hash_row(int64_t i, const int64_t *arp, const int32_t *aci, const int64_t *brp, const int32_t *bci,
                        int32_t *tab, int H, int *cnt, int *err) {
    for (int t = threadIdx.x; t < H; t += blockDim.x) tab[t] = HASH_EMPTY;
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    int64_t a0 = arp[i], a1 = arp[i + 1];
    // warp w walks A entries w, w + nwarps, ...; lanes walk the B row
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t q = a0 + wid; q < a1; q += nw) {
        int64_t k = aci[q];
        for (int64_t r = brp[k] + lane; r < brp[k + 1]; r += 32) {
            int32_t c = bci[r];
            uint32_t h = (mix32((uint32_t)c) & (uint32_t)(H - 1));
            for (int probe = 0;; ++probe) {
                if (probe >= H) {
                    atomicExch(err, 1);
                    break;
                }
                int32_t old = atomicCAS(tab + h, HASH_EMPTY, c);
                if (old == HASH_EMPTY) {
                    atomicAdd(cnt, 1);
                    break;
                }
                if (old == c) break;
                h = (h + 1) & (uint32_t)(H - 1);
            }
        }
    }
    __syncthreads();
    return *cnt;
}

__global__ void k_sg_symbolic(int64_t n, int64_t ncols, const int64_t *arp, const int32_t *aci, const int64_t *brp,
                              const int32_t *bci, const int64_t *prod, int cap, int64_t *cnt_out, int *err) {
    extern __shared__ int32_t tab[];
    __shared__ int cnt;
    int64_t i = blockIdx.x;
    int H = hash_slots(prod[i], ncols, cap);
    int u = hash_row(i, arp, aci, brp, bci, tab, H, &cnt, err);
    if (threadIdx.x == 0) cnt_out[i] = u;
}

__global__ void k_sg_numeric(int64_t n, int64_t ncols, const int64_t *arp, const int32_t *aci, const double2 *av,
                             const int64_t *brp, const int32_t *bci, const double2 *bv, const int64_t *prod, int cap,
                             const int64_t *crp, int32_t *cci, double2 *cv, int *err) {
    extern __shared__ int32_t tab[];
    __shared__ int cnt, fillc;
    int64_t i = blockIdx.x;
    int H = hash_slots(prod[i], ncols, cap);
    int u = hash_row(i, arp, aci, brp, bci, tab, H, &cnt, err);
    if (2 * u > H) {  // the sorted list below has H / 2 slots
        if (threadIdx.x == 0) atomicExch(err, 1);
        return;
    }
    int32_t *list = tab + H;
    int p2 = 1;
    while (p2 < u) p2 <<= 1;
    if (threadIdx.x == 0) fillc = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < H; t += blockDim.x)
        if (tab[t] != HASH_EMPTY) list[atomicAdd(&fillc, 1)] = tab[t];
    __syncthreads();
    for (int t = u + threadIdx.x; t < p2; t += blockDim.x) list[t] = INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)  // bitonic sort, ascending
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < p2; t += blockDim.x) {
                int o = t ^ j;
                if (o > t) {
                    bool up = ((t & k) == 0);
                    int32_t a = list[t], b = list[o];
                    if ((a > b) == up) {
                        list[t] = b;
                        list[o] = a;
                    }
                }
            }
            __syncthreads();
        }
    int64_t base = crp[i];
    int64_t a0 = arp[i], a1 = arp[i + 1];
    for (int t = threadIdx.x; t < u; t += blockDim.x) {
        int32_t c = list[t];
        double2 acc = make_double2(0, 0);
        for (int64_t q = a0; q < a1; ++q) {  // fixed order: ascending A column
            int64_t k = aci[q];
            int64_t lo = brp[k], hi = brp[k + 1] - 1;
            while (lo <= hi) {
                int64_t mid = (lo + hi) >> 1;
                int32_t mc = bci[mid];
                if (mc == c) {
                    cfma(acc, av[q], bv[mid]);
                    break;
                }
                if (mc < c)
                    lo = mid + 1;
                else
                    hi = mid - 1;
            }
        }
        cci[base + t] = c;
        cv[base + t] = acc;
    }
}

static void spgemm(const CsrDev &A, const CsrDev &B, CsrDev &C, cudaStream_t s) {
    int64_t n = A.n;
    C.n = n;
    C.m = B.m;
    DBuf<int64_t> prod(n + 1), cnt(n + 1);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    k_sg_prod<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), B.rp.get(), prod.get());
    GL_LAUNCH_CHECK();
    DBuf<int64_t> part(256);
    {
        // reuse the row-length maximum on a fake CSR view of the product counts
        CsrDev tmp;
        tmp.n = n;
        DBuf<int64_t> pre(n + 1);
        scan_exclusive(prod.get(), pre.get(), n, true, s);
        k_rowlen_max<<<256, 256, 0, s>>>(n, pre.get(), part.get());
        GL_LAUNCH_CHECK();
    }
    int64_t pmax = max_i64_parts(part.get(), 256, s);
    int cap = 1 << 15;  // up to 32768 hash slots: 128 KiB table + 64 KiB list
    int64_t u = pmax < B.m ? pmax : B.m;
    int H = 32;
    while (H < 2 * u && H < cap) H <<= 1;
    size_t sm_sym = (size_t)H * sizeof(int32_t);
    size_t sm_num = sm_sym + (size_t)(H / 2) * sizeof(int32_t);
    GL_CUDA(cudaFuncSetAttribute(k_sg_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sym));
    GL_CUDA(cudaFuncSetAttribute(k_sg_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_num));
    k_sg_symbolic<<<(unsigned)n, 128, sm_sym, s>>>(n, B.m, A.rp.get(), A.ci.get(), B.rp.get(), B.ci.get(), prod.get(),
                                                  cap, cnt.get(), err.get());
    GL_LAUNCH_CHECK();
    C.rp.alloc(n + 1);
    scan_exclusive(cnt.get(), C.rp.get(), n, true, s);
    GL_CUDA(cudaMemcpyAsync(&C.nnz, C.rp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    C.ci.alloc(C.nnz > 0 ? C.nnz : 1);
    C.v.alloc(C.nnz > 0 ? C.nnz : 1);
    k_sg_numeric<<<(unsigned)n, 128, sm_num, s>>>(n, B.m, A.rp.get(), A.ci.get(), A.v.get(), B.rp.get(), B.ci.get(),
                                                 B.v.get(), prod.get(), cap, C.rp.get(), C.ci.get(), C.v.get(),
                                                 err.get());
    GL_LAUNCH_CHECK();
    int herr = 0;
    GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(herr == 0, GL_ERR_CAPACITY, "SpGEMM row exceeded the shared hash table");
}

// (A + A^H) / 2 in place; the pattern is structurally symmetric
__global__ void k_symmetrize(int64_t n, const int64_t *rp, const int32_t *ci, double2 *v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
        int64_t j = ci[q];
        if (j < i) continue;
        if (j == i) {
            v[q].y = 0.0;
            continue;
        }
        int64_t lo = rp[j], hi = rp[j + 1] - 1, f = -1;
        while (lo <= hi) {
            int64_t mid = (lo + hi) >> 1;
            if (ci[mid] == i) {
                f = mid;
                break;
            }
            if (ci[mid] < i)
                lo = mid + 1;
            else
                hi = mid - 1;
        }
        double2 a = v[q], b = (f >= 0) ? v[f] : make_double2(0, 0);
        double2 sv = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        v[q] = sv;
        if (f >= 0) v[f] = make_double2(sv.x, -sv.y);
    }
}

// ------------------------------------------------------------------ coarsest level
// the stored entries of a CSR matrix into a zeroed dense row-major one
__global__ void k_to_dense(int64_t n, const int64_t *rp, const int32_t *ci, const double2 *v, double2 *M) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) M[i * n + ci[q]] = v[q];
}
// the pivot row scaled by 1 / pivot and the pivot column, as they are before
// step k (the pivot of an HPD matrix stays real positive; a non-positive one is
// reported)
__global__ void k_gj_snap(int64_t n, int64_t k, const double2 *M, double2 *rowk, double2 *colk, double *ipiv,
                          int *err) {
    const double piv = M[k * n + k].x;
    const double ip = 1.0 / piv;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) {
        const double2 r = M[k * n + t];
        rowk[t] = make_double2(r.x * ip, r.y * ip);
        colk[t] = M[t * n + k];
    }
    if (t == 0) {
        *ipiv = ip;
        if (!(piv > 0)) atomicExch(err, 1);
    }
}
// one Gauss-Jordan step on pivot k (in-place inversion, no pivoting: A is HPD):
// row i = blockIdx.y, columns blockIdx.x * blockDim.x + threadIdx.x; one complex
// product per entry off the pivot row and column
__global__ void __launch_bounds__(256) k_gj_step(int64_t n, int64_t k, double2 *M, const double2 *__restrict__ rowk,
                                                 const double2 *__restrict__ colk, const double *__restrict__ ipiv) {
    const int64_t i = blockIdx.y;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t t = i * n + j;
    double2 r;
    if (i == k) {
        r = (j == k) ? make_double2(*ipiv, 0.0) : rowk[j];
    } else if (j == k) {
        const double ip = *ipiv;
        r = make_double2(-colk[i].x * ip, -colk[i].y * ip);
    } else {
        const double2 cr = cmul(colk[i], rowk[j]);
        r = make_double2(M[t].x - cr.x, M[t].y - cr.y);
    }
    M[t] = r;
}

static void dense_inverse(const CsrDev &A, DBuf<double2> &Ainv, cudaStream_t s) {
    int64_t n = A.n;
    GL_REQUIRE(n <= MAX_COARSE_DENSE, GL_ERR_CAPACITY, "coarsest level too large for the dense solve");
    Ainv.alloc(n * n);
    DBuf<double2> rowk(n), colk(n);
    DBuf<double> ipiv(1);
    DBuf<int> err(1);
    GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    GL_CUDA(cudaMemsetAsync(Ainv.get(), 0, (size_t)n * n * sizeof(double2), s));
    k_to_dense<<<grid_for(n, 128), 128, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), Ainv.get());
    const dim3 step_grid((unsigned)((n + 255) / 256), (unsigned)n);
    for (int64_t k = 0; k < n; ++k) {
        k_gj_snap<<<grid_for(n, 256), 256, 0, s>>>(n, k, Ainv.get(), rowk.get(), colk.get(), ipiv.get(), err.get());
        k_gj_step<<<step_grid, 256, 0, s>>>(n, k, Ainv.get(), rowk.get(), colk.get(), ipiv.get());
    }
    GL_LAUNCH_CHECK();
    int herr = 0;
    GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    GL_REQUIRE(herr == 0, GL_ERR_BREAKDOWN, "coarsest operator is not positive definite");
}

// ------------------------------------------------------------------ solve ordering
__global__ void k_color_flag(int64_t n, const int32_t *color, int32_t c, int64_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (color[i] == c) ? 1 : 0;
}
__global__ void k_color_place(int64_t n, const int32_t *color, int32_t c, const int64_t *rank, int64_t off,
                              int32_t *perm, int32_t *iperm) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && color[i] == c) {
        int64_t p = off + rank[i];
        perm[p] = (int32_t)i;
        iperm[i] = (int32_t)p;
    }
}
__global__ void k_iota(int64_t n, int32_t *a, int32_t *b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = b[i] = (int32_t)i;
}
__global__ void k_pdiag(int64_t n, const double *kdiag, const double2 *psi, double *pd) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) pd[p] = kdiag[p] + 2.0 * (psi[p].x * psi[p].x + psi[p].y * psi[p].y);
}
__global__ void k_fill_d(int64_t n, double *x, double v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// M[p][q] = Ainv[perm[p]][perm[q]] vol[perm[q]]: the node-order inverse of the
// level-0 operator as the map from v to z = Ainv D v in the solve ordering
__global__ void k_dense_perm_scale(int64_t n, const double2 *__restrict__ Ainv, const int32_t *__restrict__ perm,
                                   const double *__restrict__ vol, double2 *__restrict__ M) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    const int64_t p = t / n, q = t % n;
    const int64_t i = perm[p], j = perm[q];
    const double2 a = Ainv[i * n + j];
    M[t] = make_double2(a.x * vol[j], a.y * vol[j]);
}

static void colour_ordering(Level &L, cudaStream_t s) {
    int64_t n = L.n;
    L.perm_own.alloc(n);
    L.iperm_own.alloc(n);
    L.cstart.assign(L.ncolors + 1, 0);
    DBuf<int64_t> rank(n + 1);
    int G = grid_for(n, 256);
    int64_t off = 0;
    for (int c = 0; c < L.ncolors; ++c) {
        k_color_flag<<<G, 256, 0, s>>>(n, L.color.get(), c, rank.get());
        GL_LAUNCH_CHECK();
        scan_exclusive(rank.get(), rank.get(), n, true, s);
        int64_t cntc = 0;
        GL_CUDA(cudaMemcpyAsync(&cntc, rank.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        k_color_place<<<G, 256, 0, s>>>(n, L.color.get(), c, rank.get(), off, L.perm_own.get(), L.iperm_own.get());
        GL_LAUNCH_CHECK();
        GL_CUDA(cudaStreamSynchronize(s));
        L.cstart[c] = off;
        off += cntc;
    }
    L.cstart[L.ncolors] = off;
    L.perm = L.perm_own.get();
    L.iperm = L.iperm_own.get();
}

static void copy_csr(const CsrDev &a, CsrDev &b, cudaStream_t s) {
    b.n = a.n;
    b.m = a.m;
    b.nnz = a.nnz;
    b.rp.alloc(a.n + 1);
    b.ci.alloc(a.nnz);
    b.v.alloc(a.nnz);
    GL_CUDA(cudaMemcpyAsync(b.rp.get(), a.rp.get(), (a.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    GL_CUDA(cudaMemcpyAsync(b.ci.get(), a.ci.get(), a.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    GL_CUDA(cudaMemcpyAsync(b.v.get(), a.v.get(), a.nnz * sizeof(double2), cudaMemcpyDeviceToDevice, s));
}

// ------------------------------------------------------------------ driver
void precond_setup(gl_prec_s *p, gl_mesh_s *m, const double2 *psi_nat, const gl_options &o, cudaStream_t s,
                   const gl_prec_s *like) {
    static std::atomic<int64_t> next_uid{1};
    p->uid = next_uid.fetch_add(1);
    p->mesh = m;
    p->mesh_version = m->version;
    // GL_VERBOSE: wall time of the setup's phases (synchronising at each mark)
    auto t_last = std::chrono::steady_clock::now();
    auto mark = [&](const char *what) {
        if (!verbose()) return;
        GL_CUDA(cudaStreamSynchronize(s));
        const auto t = std::chrono::steady_clock::now();
        fprintf(stderr, "gl: setup %-28s %8.2f ms\n", what, std::chrono::duration<double, std::milli>(t - t_last).count());
        t_last = t;
    };
    p->rinf = (o.cycles == CYCLES_INF);
    GL_REQUIRE(!p->rinf || o.precision == GL_FP64, GL_ERR_ARG, "R_inf (cycles = -1) needs precision GL_FP64");
    p->cycles = o.cycles > 0 ? o.cycles : 1;
    int maxlev = o.max_levels > 0 ? std::min(o.max_levels, MAX_LEVELS) : 10;
    int64_t max_coarse = o.max_coarse > 0 ? o.max_coarse : 512;
    GL_REQUIRE(max_coarse <= MAX_COARSE_DENSE, GL_ERR_ARG, "max_coarse above 4096");
    int power_its = o.power_its > 0 ? o.power_its : 20;
    int64_t n = m->n;
    p->max_coarse_used = max_coarse;
    p->maxlev_used = maxlev;
    p->coloring_used = o.coloring;
    const gl_prec_s *T = like;
    if (T && !(T->mesh == m && T->max_coarse_used == max_coarse && T->maxlev_used == maxlev &&
               T->coloring_used == o.coloring && T->nlev >= 1))
        T = nullptr;
    // level l of the template can stand in for level l here (same size, so the same graph)
    auto same = [&](int l, int64_t nl) { return T && l < T->nlev && T->L[l].n == nl; };

    // level 0: K-hat + 2 D |psi|^2 in node order
    Level &L0 = p->L[0];
    L0.n = n;
    copy_csr(m->khat, L0.A_can, s);
    k_add_diag<<<grid_for(n, 256), 256, 0, s>>>(n, L0.A_can.rp.get(), L0.A_can.ci.get(), L0.A_can.v.get(),
                                                m->vol.get(), psi_nat);
    GL_LAUNCH_CHECK();
    L0.B.alloc(n);
    k_fill_d<<<grid_for(n, 256), 256, 0, s>>>(n, L0.B.get(), 1.0);
    L0.color.alloc(n);
    GL_CUDA(cudaMemcpyAsync(L0.color.get(), m->color0.get(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    L0.ncolors = m->ncolors0;

    int l = 0;
    for (;;) {
        Level &L = p->L[l];
        int64_t nl = L.n;
        if (l > 0) {
            L.color.alloc(nl);
            if (same(l, nl) && T->L[l].color.n == (size_t)nl) {
                GL_CUDA(cudaMemcpyAsync(L.color.get(), T->L[l].color.get(), nl * sizeof(int32_t),
                                        cudaMemcpyDeviceToDevice, s));
                L.ncolors = T->L[l].ncolors;
            } else {
                L.ncolors = o.coloring == GL_COLOR_JP    ? color_jp(L.A_can, L.color.get(), s)
                            : o.coloring == GL_COLOR_PSL ? color_psl(L.A_can, L.color.get(), s)
                                                         : color_smallest_last(L.A_can, L.color.get(), s);
            }
        }
        if (nl <= max_coarse || l + 1 >= maxlev) break;
        L.agg.alloc(nl);
        int64_t nc;
        if (same(l, nl) && l + 1 < T->nlev && T->L[l].agg.n == (size_t)nl) {
            GL_CUDA(cudaMemcpyAsync(L.agg.get(), T->L[l].agg.get(), nl * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            nc = T->L[l + 1].n;
        } else {
            nc = aggregate(L.A_can, L.agg.get(), s);
        }
        if (nc >= nl || nc == 0) {
            L.agg.release();
            break;
        }
        // candidate norms per aggregate
        Level &Lc = p->L[l + 1];
        Lc.n = nc;
        Lc.B.alloc(nc);
        {
            DBuf<int64_t> cnt(nc + 1), fill(nc + 1), arp(nc + 1);
            DBuf<int32_t> mem(nl);
            GL_CUDA(cudaMemsetAsync(cnt.get(), 0, (nc + 1) * sizeof(int64_t), s));
            GL_CUDA(cudaMemsetAsync(fill.get(), 0, (nc + 1) * sizeof(int64_t), s));
            k_count_cols<<<grid_for(nl, 256), 256, 0, s>>>(nl, L.agg.get(), cnt.get());
            GL_LAUNCH_CHECK();
            scan_exclusive(cnt.get(), arp.get(), nc, true, s);
            k_agg_members<<<grid_for(nl, 256), 256, 0, s>>>(nl, L.agg.get(), arp.get(), fill.get(), mem.get());
            k_sort_small_i32<<<grid_for(nc, 128), 128, 0, s>>>(nc, arp.get(), mem.get());
            k_bnorm<<<grid_for(nc, 256), 256, 0, s>>>(nc, arp.get(), mem.get(), L.B.get(), Lc.B.get());
            GL_LAUNCH_CHECK();
            GL_CUDA(cudaStreamSynchronize(s));
        }
        // prolongator smoothing
        L.rho = spectral_radius(L.A_can, power_its, s);
        L.omega = 4.0 / (3.0 * L.rho);
        {
            CsrDev &P = L.P_can;
            P.n = nl;
            P.m = nc;
            DBuf<int64_t> len(nl + 1);
            DBuf<int> err(1);
            GL_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
            k_p_count<<<grid_for(nl, 128), 128, 0, s>>>(nl, L.A_can.rp.get(), L.A_can.ci.get(), L.agg.get(),
                                                        len.get(), err.get());
            GL_LAUNCH_CHECK();
            P.rp.alloc(nl + 1);
            scan_exclusive(len.get(), P.rp.get(), nl, true, s);
            GL_CUDA(cudaMemcpyAsync(&P.nnz, P.rp.get() + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            int herr = 0;
            GL_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
            GL_CUDA(cudaStreamSynchronize(s));
            GL_REQUIRE(herr == 0, GL_ERR_CAPACITY, "prolongator row touches too many aggregates");
            P.ci.alloc(P.nnz);
            P.v.alloc(P.nnz);
            k_p_fill<<<grid_for(nl, 128), 128, 0, s>>>(nl, L.A_can.rp.get(), L.A_can.ci.get(), L.A_can.v.get(),
                                                       L.agg.get(), L.B.get(), Lc.B.get(), L.omega, P.rp.get(),
                                                       P.ci.get(), P.v.get());
            GL_LAUNCH_CHECK();
        }
        // Galerkin coarse operator
        {
            CsrDev PH, T;
            transpose_conj(L.P_can, PH, s);
            spgemm(L.A_can, L.P_can, T, s);
            spgemm(PH, T, Lc.A_can, s);
            k_symmetrize<<<grid_for(nc, 128), 128, 0, s>>>(nc, Lc.A_can.rp.get(), Lc.A_can.ci.get(), Lc.A_can.v.get());
            GL_LAUNCH_CHECK();
            GL_CUDA(cudaStreamSynchronize(s));
        }
        ++l;
    }
    p->nlev = l + 1;

    // coarsest level: dense inverse, identity ordering
    Level &Lb = p->L[l];
    mark("hierarchy (aggregation, P, RAP)");
    dense_inverse(Lb.A_can, Lb.Ainv, s);
    mark("dense coarsest inverse");

    // solve-ordering structures
    for (int k = 0; k < p->nlev; ++k) {
        Level &L = p->L[k];
        bool coarsest = (k == p->nlev - 1);
        if (k == 0) {
            L.perm = m->perm.get();
            L.iperm = m->iperm.get();
            L.cstart = m->cstart0;
            L.A = &m->K;
        } else if (coarsest) {
            L.perm_own.alloc(L.n);
            L.iperm_own.alloc(L.n);
            k_iota<<<grid_for(L.n, 256), 256, 0, s>>>(L.n, L.perm_own.get(), L.iperm_own.get());
            GL_LAUNCH_CHECK();
            L.perm = L.perm_own.get();
            L.iperm = L.iperm_own.get();
        } else {
            colour_ordering(L, s);
        }
    }
    if (p->nlev == 1) {
        // the finest level is also the coarsest: the V-cycle there is z = P-hat^-1 D v
        // in the solve ordering, so the dense inverse is permuted and scaled by D
        DBuf<double2> M(n * n);
        k_dense_perm_scale<<<grid_for(n * n, 256), 256, 0, s>>>(n, Lb.Ainv.get(), m->perm.get(), m->vol.get(),
                                                               M.get());
        GL_LAUNCH_CHECK();
        Lb.Ainv = std::move(M);
    }
    mark("solve orderings");
    p->psi_p.alloc(n);
    permute_in(n, m->perm.get(), psi_nat, p->psi_p.get(), s);
    p->err.alloc(1);
    GL_CUDA(cudaMemsetAsync(p->err.get(), 0, sizeof(int), s));
    p->wait_extra.alloc(1);
    GL_CUDA(cudaMemsetAsync(p->wait_extra.get(), 0, sizeof(unsigned long long), s));
    for (int k = 0; k < p->nlev; ++k) {
        Level &L = p->L[k];
        bool coarsest = (k == p->nlev - 1);
        L.diag.alloc(L.n);
        if (k == 0) {
            k_pdiag<<<grid_for(n, 256), 256, 0, s>>>(n, m->kdiag.get(), p->psi_p.get(), L.diag.get());
            GL_LAUNCH_CHECK();
        } else if (!coarsest) {
            build_sell<double2>(L.n, L.n, L.perm, L.iperm, L.A_can, nullptr, true, L.A_own, L.diag.get(), s);
            L.A = &L.A_own;
            build_csrg<double2>(L.n, L.perm, L.iperm, L.A_can, true, L.Ag, nullptr, s);
            L.cstart_dev.alloc(L.ncolors + 1);
            GL_CUDA(cudaMemcpyAsync(L.cstart_dev.get(), L.cstart.data(), (L.ncolors + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s));
            L.barrier.alloc(GRID_BARRIER_WORDS);
            GL_CUDA(cudaMemsetAsync(L.barrier.get(), 0, GRID_BARRIER_WORDS * sizeof(unsigned), s));
            L.flags.alloc(2 * (size_t)MAX_FLAG_CTAS * FLAG_STRIDE);
            GL_CUDA(cudaMemsetAsync(L.flags.get(), 0, L.flags.bytes(), s));
        }
        if (!coarsest) {
            Level &Lc = p->L[k + 1];
            build_sell<double2>(L.n, Lc.n, L.perm, Lc.iperm, L.P_can, nullptr, false, L.P, nullptr, s);
            CsrDev PH;
            transpose_conj(L.P_can, PH, s);
            build_sell<double2>(Lc.n, L.n, Lc.perm, L.iperm, PH, nullptr, false, L.PH, nullptr, s);
            build_csrg<double2>(Lc.n, Lc.perm, L.iperm, PH, false, L.PHg, nullptr, s);
        }
        L.b.alloc(L.n);
        L.x.alloc(L.n);
        L.r.alloc(L.n);
    }
    // stored off-diagonals per colour (for the byte accounting of the sweeps)
    for (int k = 0; k < p->nlev - 1; ++k) {
        Level &L = p->L[k];
        std::vector<int64_t> hrp(L.n + 1);
        std::vector<int32_t> hc(L.n);
        GL_CUDA(cudaMemcpyAsync(hrp.data(), L.A_can.rp.get(), (L.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaMemcpyAsync(hc.data(), L.color.get(), L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
        L.cnnz.assign(L.ncolors, 0);
        for (int64_t i = 0; i < L.n; ++i) L.cnnz[hc[i]] += hrp[i + 1] - hrp[i] - 1;
    }
    // cost of one V-cycle in matrix entries visited: per level the two symmetric
    // Gauss-Seidel steps (a colour visit reads its rows' off-diagonals and
    // diagonals; from the zero guess the first colour reads only diagonals; the
    // backward pass skips the repeated last colour), the residual (all entries),
    // restriction and prolongation (nnz(P) each); the dense coarsest product
    // (n_c^2).  The finest operator K-hat has nnz_0 off-diagonals + n_0 diagonals.
    {
        double E = 0;
        for (int k = 0; k < p->nlev - 1; ++k) {
            const Level &L = p->L[k];
            double all = 0;
            std::vector<double> visit(L.ncolors);
            for (int c = 0; c < L.ncolors; ++c) {
                visit[c] = (double)L.cnnz[c] + (double)(L.cstart[c + 1] - L.cstart[c]);
                all += visit[c];
            }
            const double rows0 = (double)(L.cstart[1] - L.cstart[0]);
            const double back = all - visit[L.ncolors - 1];
            E += (all - visit[0] + rows0) + back;  // pre-smoothing from zero
            E += all + back;                       // post-smoothing
            E += all;                              // residual
            E += 2.0 * (double)L.P_can.nnz;        // restriction and prolongation
        }
        const Level &Lc = p->L[p->nlev - 1];
        E += (double)Lc.n * (double)Lc.n;
        p->cost_vcycle = E;
        // (the per-colour counts exist on the smoothed levels only)
        double fine = (double)m->khat.nnz;
        if (p->nlev > 1) {
            fine = (double)p->L[0].n;
            for (int c = 0; c < p->L[0].ncolors; ++c) fine += (double)p->L[0].cnnz[c];
        }
        p->cost_fine = fine;
    }
    if (p->rinf) {
        p->rinf_part.alloc(RED_BLOCKS);
        p->rinf_dev.alloc(1);
        GL_CUDA(cudaMemsetAsync(p->rinf_dev.get(), 0, sizeof(RinfDev), s));
        GL_CUDA(cudaStreamCreateWithFlags(&p->rinf_body, cudaStreamNonBlocking));
        GL_CUDA(cudaStreamCreateWithFlags(&p->rinf_eager, cudaStreamNonBlocking));
        for (auto &e : p->rinf_ev) GL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (p->cycles > 1 || p->rinf) {
        p->cyc_r.alloc(n);
        p->cyc_e.alloc(n);
    }
    GL_CUDA(cudaStreamSynchronize(s));
    p->autotune = o.autotune != 0;
    p->lattice = o.lattice != 0;
    p->lattice64 = o.lattice == 2;
    p->cluster_sweeps = o.cluster_sweeps != 0;
    p->sweep_sync = o.sweep_sync;
    p->coarse_df = o.coarse_df != 0;
    if (T && T->nlev == p->nlev && T->autotune == p->autotune && T->cluster_sweeps == p->cluster_sweeps &&
        T->sweep_sync == p->sweep_sync) {
        for (int k = 0; k < p->nlev; ++k) {
            const Level &S = T->L[k];
            auto &t = p->tuned[k];
            t.ag64 = S.Ag.G;
            t.phg64 = S.PHg.G;
            t.sgs64 = S.sgs_G64;
            t.ag32 = S.Ag32.G;
            t.phg32 = S.PHg32.G;
            t.sgs32 = S.sgs_G32;
            t.cl_size = S.cl_size;
            t.cl_chunk = S.cl_chunk;
            t.sync64 = S.sync64;
            t.nb64 = S.fl64.nb;
            t.sync32 = S.sync32;
            t.nb32 = S.fl32.nb;
        }
        p->tuned64 = true;
        p->tuned32 = T->has32;
    }
    mark("solve-order operators, cost");
    if (p->tuned64) {
        for (int k = 0; k < p->nlev; ++k) {
            Level &L = p->L[k];
            L.Ag.G = p->tuned[k].ag64;
            L.PHg.G = p->tuned[k].phg64;
            L.sgs_G64 = p->tuned[k].sgs64;
            L.sync64 = p->tuned[k].sync64;
        }
        rebuild_flag_plans(p, false, s);
    } else {
        if (p->autotune) autotune_levels(p, false, s);
        plan_sweeps(p, false, s);
    }
    mark("FP64 kernel choices");
    if (o.precision != GL_FP64) precond_ensure_fp32(p, s);
    mark("FP32 copies and choices");
}

// FP32 copies of every level (the coarsest solve stays FP64)
void precond_ensure_fp32(gl_prec_s *p, cudaStream_t s) {
    if (p->has32) return;
    gl_mesh_s *m = p->mesh;
    mesh_ensure_fp32(m, s);
    for (int k = 0; k < p->nlev; ++k) {
        Level &L = p->L[k];
        bool coarsest = (k == p->nlev - 1);
        L.diag32.alloc(L.n);
        to_float(L.diag.get(), L.diag32.get(), L.n, s);
        if (k == 0) {
            L.A32 = &m->K32;
        } else if (!coarsest) {
            build_sell<float2>(L.n, L.n, L.perm, L.iperm, L.A_can, nullptr, true, L.A32_own, nullptr, s);
            L.A32 = &L.A32_own;
            build_csrg<float2>(L.n, L.perm, L.iperm, L.A_can, true, L.Ag32, nullptr, s);
        }
        if (!coarsest) {
            Level &Lc = p->L[k + 1];
            build_sell<float2>(L.n, Lc.n, L.perm, Lc.iperm, L.P_can, nullptr, false, L.P32, nullptr, s);
            CsrDev PH;
            transpose_conj(L.P_can, PH, s);
            build_sell<float2>(Lc.n, L.n, Lc.perm, L.iperm, PH, nullptr, false, L.PH32, nullptr, s);
            build_csrg<float2>(Lc.n, Lc.perm, L.iperm, PH, false, L.PHg32, nullptr, s);
            // after the pre-smoothing of a red-black level 0 the residual of every
            // colour-0 row is zero, so its restriction needs only the other columns
            if (k == 0 && L.ncolors == 2)
                build_csrg<float2>(Lc.n, Lc.perm, L.iperm, PH, false, L.PHg32b, nullptr, s, L.cstart[1]);
        }
        L.b32.alloc(L.n);
        L.x32.alloc(L.n);
        L.r32.alloc(L.n);
    }
    if (p->cycles > 1) {
        p->cyc_r32.alloc(m->n);
        p->cyc_e32.alloc(m->n);
    }
    if (p->tuned32) {
        for (int k = 0; k < p->nlev; ++k) {
            Level &L = p->L[k];
            L.Ag32.G = p->tuned[k].ag32;
            L.PHg32.G = p->tuned[k].phg32;
            L.sgs_G32 = p->tuned[k].sgs32;
            L.cl_size = p->tuned[k].cl_size;
            L.cl_chunk = p->tuned[k].cl_chunk;
            L.sync32 = p->tuned[k].sync32;
        }
        rebuild_flag_plans(p, true, s);
    } else {
        if (p->autotune) autotune_levels(p, true, s);
        plan_sweeps(p, true, s);
    }
    p->mp_in.alloc(m->n);
    p->mp_out.alloc(m->n);
    Level &Lb = p->L[p->nlev - 1];
    if (p->coarse_df) coarse_inverse_df(Lb, s);
    p->coarse_b64.alloc(Lb.n);
    p->coarse_x64.alloc(Lb.n);
    GL_CUDA(cudaStreamSynchronize(s));
    p->has32 = true;
}

__global__ void k_negate(int64_t n, double2 *a) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = make_double2(-a[i].x, -a[i].y);
}

void precond_negate_coarsest(gl_prec_s *p, cudaStream_t s) {
    Level &L = p->L[p->nlev - 1];
    const int64_t nn = L.n * L.n;
    k_negate<<<grid_for(nn, 256), 256, 0, s>>>(nn, L.Ainv.get());
    GL_LAUNCH_CHECK();
    if (L.Ainv_df.get()) coarse_inverse_df(L, s);  // the FP32 V-cycle's copy follows
    GL_CUDA(cudaStreamSynchronize(s));
}

void rinf_reset(gl_prec_s *p, cudaStream_t s) {
    if (p && p->rinf) GL_CUDA(cudaMemsetAsync(p->rinf_dev.get(), 0, sizeof(RinfDev), s));
}

RinfDev rinf_read(gl_prec_s *p, cudaStream_t s) {
    RinfDev r{};
    if (p && p->rinf) {
        GL_CUDA(cudaMemcpyAsync(&r, p->rinf_dev.get(), sizeof(RinfDev), cudaMemcpyDeviceToHost, s));
        GL_CUDA(cudaStreamSynchronize(s));
    }
    return r;
}

double precond_cost(const gl_prec_s *p, int k) {
    if (k <= 0 || p->cost_fine <= 0) return 0.0;
    // R_k: k V-cycles and, between them, k - 1 finest-level residuals
    return ((double)k * p->cost_vcycle + (double)(k - 1) * p->cost_fine) / p->cost_fine;
}

}  // namespace gl

gl_prec_s::~gl_prec_s() {
    if (rinf_body) cudaStreamDestroy(rinf_body);
    if (rinf_eager) cudaStreamDestroy(rinf_eager);
    for (auto e : rinf_ev)
        if (e) cudaEventDestroy(e);
}
