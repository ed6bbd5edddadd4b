// gl_warmstart.cu -- learned initial guess for the Jacobian solve J(psi) x = b
// (Sec. 3, Eq. (16)); the paper has no learned part, the network is defined here.
//
//   x0 = ||b||_D * y(psi, b / ||b||_D) / K_ii,      ||b||_D^2 = sum_i |V_i| |b_i|^2
//
// y is a 4-layer, 64-channel graph network on the mesh.  Channels come in 32
// complex pairs; channel 63 is the constant 1 (it carries the biases).
//   h^0_i   = [Re b^_i, Im b^_i, Re psi_i, Im psi_i, |psi_i|^2, 0 ... 0, 1]
//   a^l_i   = [h^l_i ; (S h^l)_i],  (S u)_i = sum_k (-K-hat_ik / K-hat_ii) u_k  (per pair)
//   h^{l+1} = relu(W^l a^l), channel 63 reset to 1            (W^l: 64 x 128)
//   y_i     = U h^4_i                                          (U: 2 x 64)
// S = I - diag(K)^-1 K is the magnetic Jacobi operator: the edge weights and
// phases of Eq. (10) normalised per row.  Training minimises the squared relative
// true-Jacobian residual L = ||b^ - J x^||_D^2 of the guess (x^ = y / K_ii).
//
// GPU layout and precision:
//   * every vector is in the solve ordering of the mesh (red nodes first); the
//     aggregation reads the FP32 copy of K (sliced ELL) and K_ii;
//   * activations h^l are n x 64 BF16, node-major (128 B per node);
//   * the dense layers are tcgen05 MMAs (kind::f16, BF16 operands, FP32
//     accumulators in tensor memory), one 128-node tile per MMA group.  Operands
//     are staged in shared memory as K-major tiles of 8-row x 16-byte core
//     matrices without swizzle: leading-dimension offset 128 B (next core matrix
//     along K), stride-dimension offset 16 K bytes (next 8-row group);
//   * forward: one persistent kernel per layer builds [h, S h] for its tile
//     (gathering the neighbours' BF16 rows), issues 8 MMAs (K = 16 each) into a
//     128 x 64 FP32 accumulator, and applies relu (and the head on the last layer)
//     in the epilogue;
//   * backward: one persistent kernel per layer issues dA = dz W (M = 128 nodes,
//     N = 128, K = 64) and accumulates dW^T += a^T dz (M = 128 inputs, N = 64,
//     K = 128 nodes of the tile) in tensor memory across all of its tiles; the
//     adjoint aggregation S^T and the relu mask follow in a gather kernel;
//   * parameters are FP32 masters with Adam moments; BF16 images of each W in
//     the two shared-memory operand layouts are rebuilt after every update.
// Every reduction (loss, dW, dU, ||b||) sums per-block partials in a fixed order,
// so results are deterministic for a given launch configuration.
#include <cuda_bf16.h>

#include <cstring>

#include "gl_internal.cuh"
#include "gl_profile.cuh"

namespace gl {
namespace ws {

constexpr int CH = 64;               // channels
constexpr int CIN = 2 * CH;          // [h, S h]
constexpr int NL = 4;                // layers
constexpr int WSZ = CH * CIN;        // one W^l
constexpr int NPARAM = NL * WSZ + 2 * CH;
constexpr int TILE = 128;            // nodes per MMA tile (= M)
constexpr int THREADS = 128;         // one thread per node row of the tile
constexpr int FWD_SMEM = TILE * CIN * 2 + CH * CIN * 2;            // a tile + W image
constexpr int BWD_SMEM = TILE * CH * 2 + CIN * CH * 2 + CIN * TILE * 2 + CH * TILE * 2;
constexpr int DU_BLOCKS = 2 * NUM_SMS_HINT;
constexpr long long WAIT_CYCLES = 4000000000LL;   // about 2 s at the maximum SM clock

static_assert(NPARAM == GL_WS_NPARAM, "parameter count must match the header");

// ------------------------------------------------------------------ tcgen05 helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element offset (in 2-byte units) of (row r, column k) in an R x K K-major tile
// of 8 x 8 core matrices, K fastest between core matrices
__device__ __forceinline__ int cm_off(int r, int k, int K) {
    return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// shared-memory matrix descriptor: no swizzle, version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// wait on an mbarrier phase for at most WAIT_CYCLES; returns false if that ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    const long long t0 = clock64();
    while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity));
        if (!done && clock64() - t0 > WAIT_CYCLES) break;
    }
    return done != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// ------------------------------------------------------------------ BF16 row helpers
// 8 BF16 <-> 8 floats in one 16-byte word
__device__ __forceinline__ void unpack8(uint4 u, float *f) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float *f) {
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

// (S h)_p for one node: sum over its K row of K_pq h_q per complex pair, scaled by
// -1 / K_pp.  Rows of h are 64 BF16 (8 x 16 B).
__device__ __forceinline__ void aggregate_row(const SellView<float2> &K, const float *__restrict__ kdiag,
                                              const uint4 *__restrict__ H, int64_t p, float *acc) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = 0.f;
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    for (int k = 0; k < w; ++k) {
        int64_t q = beg + (int64_t)k * SELL_C + lane;
        float2 kv = K.val[q];
        if (kv.x == 0.f && kv.y == 0.f) continue;
        const uint4 *row = H + (int64_t)K.col[q] * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float f[8];
            unpack8(__ldg(row + j), f);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float re = f[2 * t], im = f[2 * t + 1];
                acc[8 * j + 2 * t] += kv.x * re - kv.y * im;
                acc[8 * j + 2 * t + 1] += kv.x * im + kv.y * re;
            }
        }
    }
    float sc = -1.f / kdiag[p];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] *= sc;
}

constexpr int WMAX = 8;   // sliced-ELL entries per row staged in shared memory

// accumulate K_pq h_q over one 16-byte chunk (four complex pairs) of h_q
__device__ __forceinline__ void cacc4(float *acc, float2 v, uint4 r) {
    float f[8];
    unpack8(r, f);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        acc[2 * t] += v.x * f[2 * t] - v.y * f[2 * t + 1];
        acc[2 * t + 1] += v.x * f[2 * t + 1] + v.y * f[2 * t];
    }
}

// (S h) for channels 8 j .. 8 j + 7 of two nodes rA, rB of the tile, with their
// sliced-ELL entries staged in shared memory (entries beyond WMAX, which the
// lattice meshes do not have, are read from global memory).  All neighbour
// chunks of both nodes are requested before any is used.
__device__ __forceinline__ void aggregate_pair(const SellView<float2> &K, const float *__restrict__ kdiag,
                                               const uint4 *__restrict__ H, const int32_t *sCol,
                                               const float2 *sVal, const int *sWid, int64_t base, int rA, int rB,
                                               int j, int64_t n, uint4 &outA, uint4 &outB) {
    float accA[8], accB[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) accA[i] = accB[i] = 0.f;
    const int wA = (base + rA < n) ? sWid[rA >> 5] : 0, wB = (base + rB < n) ? sWid[rB >> 5] : 0;
    uint4 ra[WMAX], rb[WMAX];
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        if (k < wA) ra[k] = __ldg(H + (int64_t)sCol[k * TILE + rA] * 8 + j);
        if (k < wB) rb[k] = __ldg(H + (int64_t)sCol[k * TILE + rB] * 8 + j);
    }
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        if (k < wA) cacc4(accA, sVal[k * TILE + rA], ra[k]);
        if (k < wB) cacc4(accB, sVal[k * TILE + rB], rb[k]);
    }
    // rows wider than WMAX (not produced by the lattice meshes)
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int r = h ? rB : rA;
        const int64_t p = base + r;
        if (p >= n) continue;
        const int64_t sl = p >> 5;
        const int64_t beg = K.sptr[sl];
        const int w = (int)((K.sptr[sl + 1] - beg) >> 5);
        for (int k = WMAX; k < w; ++k) {
            const int64_t e = beg + (int64_t)k * SELL_C + (p & 31);
            cacc4(h ? accB : accA, K.val[e], __ldg(H + (int64_t)K.col[e] * 8 + j));
        }
    }
    const float sa = base + rA < n ? -1.f / kdiag[base + rA] : 0.f;
    const float sb = base + rB < n ? -1.f / kdiag[base + rB] : 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        accA[i] *= sa;
        accB[i] *= sb;
    }
    outA = pack8(accA);
    outB = pack8(accB);
}

// ------------------------------------------------------------------ small kernels
// partials of sum |V_i| |b_i|^2
__global__ void k_bnorm_part(int64_t n, const double *__restrict__ vol, const double2 *__restrict__ b,
                             double *part) {
    __shared__ double sh[32];
    double a = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = b[i];
        a += vol[i] * (v.x * v.x + v.y * v.y);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
// bn[0] = ||b||_D, bn[1] = 1 / ||b||_D (0 if b = 0)
__global__ void k_bnorm_final(const double *part, int np, double *bn) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) {
        double r = sqrt(t);
        bn[0] = r;
        bn[1] = r > 0 ? 1.0 / r : 0.0;
    }
}

// ---- the hint: alpha = <J a, b>_R / <J a, J a>_R, r = b - alpha J a
// partials of <q, b>_R, <q, q>_R and ||a||_D^2 (q = J a)
__global__ void k_hint_part(int64_t n, const double *__restrict__ vol, const double2 *__restrict__ q,
                            const double2 *__restrict__ b, const double2 *__restrict__ a, double *part) {
    __shared__ double sh[32];
    double qb = 0, qq = 0, aa = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 qv = q[i], bv = b[i], av = a[i];
        const double w = vol[i];
        qb += w * (qv.x * bv.x + qv.y * bv.y);
        qq += w * (qv.x * qv.x + qv.y * qv.y);
        aa += w * (av.x * av.x + av.y * av.y);
    }
    const double t0 = block_sum(qb, sh);
    const double t1 = block_sum(qq, sh);
    const double t2 = block_sum(aa, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t0;
        part[RED_BLOCKS + blockIdx.x] = t1;
        part[2 * RED_BLOCKS + blockIdx.x] = t2;
    }
}
// hs[0] = alpha (0 when J a = 0), hs[1] = 1 / ||a||_D (0 when a = 0)
__global__ void k_hint_final(const double *part, double *hs) {
    __shared__ double sh[32];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) {
        s0 += part[i];
        s1 += part[RED_BLOCKS + i];
        s2 += part[2 * RED_BLOCKS + i];
    }
    const double qb = block_sum(s0, sh);
    const double qq = block_sum(s1, sh);
    const double aa = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        hs[0] = (aa > 0 && qq > 0) ? qb / qq : 0.0;
        hs[1] = aa > 0 ? 1.0 / sqrt(aa) : 0.0;
    }
}
// r = b - alpha q
__global__ void k_hint_resid(int64_t n, const double *__restrict__ hs, const double2 *__restrict__ b,
                             const double2 *__restrict__ q, double2 *__restrict__ r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double al = hs[0];
    r[i] = make_double2(b[i].x - al * q[i].x, b[i].y - al * q[i].y);
}
// x0 = alpha a
__global__ void k_hint_set(int64_t n, const double *__restrict__ hs, const double2 *__restrict__ a,
                           double2 *__restrict__ x0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double al = hs[0];
    x0[i] = make_double2(al * a[i].x, al * a[i].y);
}
// x0 += alpha a
__global__ void k_hint_add(int64_t n, const double *__restrict__ hs, const double2 *__restrict__ a,
                           double2 *__restrict__ x0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double al = hs[0];
    x0[i] = make_double2(x0[i].x + al * a[i].x, x0[i].y + al * a[i].y);
}

// h^0 rows: [Re r^, Im r^, Re psi, Im psi, |psi|^2, 0, Re a^, Im a^, 0 ..., 1]
// (the hint a^ = a / ||a||_D as the complex channel pair (6, 7), zero without one)
__global__ void k_features(int64_t n, const double2 *__restrict__ b, const double2 *__restrict__ psi,
                           const double *__restrict__ bn, const double2 *__restrict__ hint,
                           const double *__restrict__ hs, uint4 *__restrict__ H0) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double inv = bn[1];
    double2 bv = b[p], ps = psi[p];
    float f[8] = {(float)(bv.x * inv), (float)(bv.y * inv), (float)ps.x, (float)ps.y,
                  (float)(ps.x * ps.x + ps.y * ps.y), 0.f, 0.f, 0.f};
    if (hint) {
        const double ia = hs[1];
        f[6] = (float)(hint[p].x * ia);
        f[7] = (float)(hint[p].y * ia);
    }
    float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float last[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    uint4 *row = H0 + p * 8;
    row[0] = pack8(f);
#pragma unroll
    for (int j = 1; j < 7; ++j) row[j] = pack8(z);
    row[7] = pack8(last);
}

// ------------------------------------------------------------------ forward layer
enum { FWD_HIDDEN = 0, FWD_LAST_TRAIN = 1, FWD_LAST_PREDICT = 2 };

struct FwdArgs {
    int64_t n;
    int64_t ntiles;
    SellView<float2> K;
    const float *kdiag;
    const uint4 *Hin;        // n x 8 uint4
    uint4 *Hout;             // n x 8 uint4 (hidden layers, and h^4 when training)
    const uint4 *Wimg;       // 64 x 128 BF16 operand image (1024 uint4)
    const float *U;          // 2 x 64 head (last layer)
    float2 *xhat;            // training: x^ (FP32)
    double2 *x0;             // prediction: ||b|| x^ (FP64)
    const double *bn;
    int *err;
};

template <int MODE>
__global__ void __launch_bounds__(THREADS) k_fwd(FwdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smem);          // 128 x 128
    uint4 *sW = reinterpret_cast<uint4 *>(smem + TILE * CIN * 2);          // 64 x 128 image
    __shared__ int32_t sCol[WMAX * TILE];
    __shared__ float2 sVal[WMAX * TILE];
    __shared__ int sWid[TILE / SELL_C];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < CH * CIN / 8; i += THREADS) sW[i] = a.Wimg[i];
    if (warp == 0) tmem_alloc(&tslot, CH);
    if (tid == 0) mbar_init(&mbar);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const uint32_t idesc = idesc_bf16(TILE, CH);
    uint32_t phase = 0;
    bool failed = false;
    __shared__ float sU[2 * CH];
    if (MODE != FWD_HIDDEN) {
        sU[tid] = a.U[tid];
        __syncthreads();
    }
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t p = t * TILE + tid;
        // ---- stage the tile's sliced-ELL rows (thread tid: node tid of the tile)
        const int64_t base = t * TILE;
        {
            const int64_t sl = (base >> 5) + (tid >> 5);
            int w = 0;
            int64_t beg = 0;
            if (sl * SELL_C < a.n) {
                beg = a.K.sptr[sl];
                w = (int)((a.K.sptr[sl + 1] - beg) >> 5);
            }
            if ((tid & 31) == 0) sWid[tid >> 5] = w;
#pragma unroll
            for (int k = 0; k < WMAX; ++k) {
                if (k < w) {
                    const int64_t e = beg + (int64_t)k * SELL_C + (tid & 31);
                    sCol[k * TILE + tid] = a.K.col[e];
                    sVal[k * TILE + tid] = a.K.val[e];
                }
            }
        }
        __syncthreads();
        // ---- operand rows [h, S h] in BF16: eight threads per node, one 16-byte chunk each
        uint4 *rowA = reinterpret_cast<uint4 *>(sA);
        {
            const int j = tid & 7;
#pragma unroll 1
            for (int pass = 0; pass < TILE / 32; ++pass) {
                const int rA = pass * 32 + (tid >> 3), rB = rA + 16;
                uint4 hA = make_uint4(0, 0, 0, 0), hB = make_uint4(0, 0, 0, 0), sA4, sB4;
                if (base + rA < a.n) hA = __ldg(a.Hin + (base + rA) * 8 + j);
                if (base + rB < a.n) hB = __ldg(a.Hin + (base + rB) * 8 + j);
                aggregate_pair(a.K, a.kdiag, a.Hin, sCol, sVal, sWid, base, rA, rB, j, a.n, sA4, sB4);
                rowA[cm_off(rA, 8 * j, CIN) >> 3] = hA;
                rowA[cm_off(rA, CH + 8 * j, CIN) >> 3] = sA4;
                rowA[cm_off(rB, 8 * j, CIN) >> 3] = hB;
                rowA[cm_off(rB, CH + 8 * j, CIN) >> 3] = sB4;
            }
        }
        proxy_fence();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            uint32_t a0 = smem_u32(sA), b0 = smem_u32(sW);
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ++ks)
                mma_bf16(tmem, sdesc(a0 + ks * 256, 128, CIN * 16), sdesc(b0 + ks * 256, 128, CIN * 16), idesc,
                         ks > 0);
            mma_commit(&mbar);
        }
        const bool done = mbar_wait(&mbar, phase);
        if (__syncthreads_or(!done)) {
            failed = true;
            break;
        }
        phase ^= 1;
        tc_fence_after();
        // ---- epilogue: row tid of the 128 x 64 accumulator
        float h[CH];
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c = 0; c < CH; c += 16) tmem_ld16(lane_base + c, h + c);
        tc_fence_before();
        if (p < a.n) {
#pragma unroll
            for (int c = 0; c < CH; ++c) h[c] = fmaxf(h[c], 0.f);
            h[CH - 1] = 1.f;
            uint4 packed[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) packed[j] = pack8(h + 8 * j);
            if (MODE != FWD_LAST_PREDICT) {
                // stage the row in shared memory (chunks XOR-swizzled by row) for coalesced stores
                uint4 *stage = reinterpret_cast<uint4 *>(sA);
#pragma unroll
                for (int j = 0; j < 8; ++j) stage[tid * 8 + (j ^ (tid & 7))] = packed[j];
            }
            if (MODE != FWD_HIDDEN) {
                // head on the stored (BF16-rounded) h^4
                float y0 = 0.f, y1 = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float f[8];
                    unpack8(packed[j], f);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        y0 = fmaf(sU[8 * j + i], f[i], y0);
                        y1 = fmaf(sU[CH + 8 * j + i], f[i], y1);
                    }
                }
                float inv = 1.f / a.kdiag[p];
                if (MODE == FWD_LAST_TRAIN) {
                    a.xhat[p] = make_float2(y0 * inv, y1 * inv);
                } else {
                    double s = a.bn[0];
                    a.x0[p] = make_double2(s * (double)(y0 * inv), s * (double)(y1 * inv));
                }
            }
        }
        if (MODE != FWD_LAST_PREDICT) {
            __syncthreads();
            const uint4 *stage = reinterpret_cast<const uint4 *>(sA);
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int idx = it * THREADS + tid, r = idx >> 3, c = idx & 7;
                const int64_t node = t * TILE + r;
                if (node < a.n) a.Hout[node * 8 + c] = stage[r * 8 + (c ^ (r & 7))];
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, CH);
    if (failed && tid == 0) atomicExch(a.err, 1);
}

// ------------------------------------------------------------------ loss and its gradient in x^
// r^ = b^ - J x^ (FP32 arithmetic), loss partials sum |V| |r^|^2
__global__ void k_resid(int64_t n, SellView<float2> K, const float *__restrict__ kdiag,
                        const float *__restrict__ volp, const double2 *__restrict__ psi,
                        const double2 *__restrict__ b, const double *__restrict__ bn,
                        const float2 *__restrict__ xh, float2 *__restrict__ r, double *part) {
    __shared__ double sh[32];
    double a = 0;
    float inv = (float)bn[1];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = p >> 5;
        int lane = (int)(p & 31);
        int64_t beg = K.sptr[s];
        int w = (int)((K.sptr[s + 1] - beg) >> 5);
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < w; ++k) {
            int64_t q = beg + (int64_t)k * SELL_C + lane;
            cfma(acc, K.val[q], xh[K.col[q]]);
        }
        float2 ps = to32(psi[p]);
        float2 x = xh[p];
        float a2 = ps.x * ps.x + ps.y * ps.y;
        float d = kdiag[p] - 1.f + 2.f * a2;
        // J x = offdiag + (K_ii - 1 + 2|psi|^2) x + psi^2 conj(x)
        float2 p2 = make_float2(ps.x * ps.x - ps.y * ps.y, 2.f * ps.x * ps.y);
        float jx = acc.x + d * x.x + (p2.x * x.x + p2.y * x.y);
        float jy = acc.y + d * x.y + (p2.y * x.x - p2.x * x.y);
        double2 bv = b[p];
        float2 rr = make_float2((float)(bv.x * inv) - jx, (float)(bv.y * inv) - jy);
        r[p] = rr;
        a += (double)volp[p] * ((double)rr.x * rr.x + (double)rr.y * rr.y);
    }
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// loss[slot] += scale * sum(part)
__global__ void k_loss_acc(const double *part, int np, double scale, double *loss, int slot) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    double t = block_sum(a, sh);
    if (threadIdx.x == 0) loss[slot] += scale * t;
}

// dy = scale * (-2 |V| (J r^)) / K_ii   (Euclidean gradient of L in y)
__global__ void k_gout(int64_t n, SellView<float2> K, const float *__restrict__ kdiag, const float *__restrict__ volp,
                       const double2 *__restrict__ psi, const float2 *__restrict__ r, float scale,
                       float2 *__restrict__ dy) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < w; ++k) {
        int64_t q = beg + (int64_t)k * SELL_C + lane;
        cfma(acc, K.val[q], r[K.col[q]]);
    }
    float2 ps = to32(psi[p]);
    float2 x = r[p];
    float a2 = ps.x * ps.x + ps.y * ps.y;
    float d = kdiag[p] - 1.f + 2.f * a2;
    float2 p2 = make_float2(ps.x * ps.x - ps.y * ps.y, 2.f * ps.x * ps.y);
    float jx = acc.x + d * x.x + (p2.x * x.x + p2.y * x.y);
    float jy = acc.y + d * x.y + (p2.y * x.x - p2.x * x.y);
    float f = -2.f * scale * volp[p] / kdiag[p];
    dy[p] = make_float2(f * jx, f * jy);
}

// dU partials: block b, thread (o = tid / 64, c = tid % 64) sums dy_i[o] h4_i[c]
__global__ void __launch_bounds__(128) k_du_part(int64_t n, const float2 *__restrict__ dy,
                                                 const __nv_bfloat16 *__restrict__ H4, float *part) {
    int o = threadIdx.x >> 6, c = threadIdx.x & 63;
    float acc = 0.f;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        float2 g = dy[i];
        acc = fmaf(o ? g.y : g.x, __bfloat162float(H4[i * CH + c]), acc);
    }
    part[(int64_t)blockIdx.x * 128 + threadIdx.x] = acc;
}
__global__ void k_du_final(const float *part, int np, float *gU) {
    int t = threadIdx.x;
    float a = 0.f;
    for (int b = 0; b < np; ++b) a += part[(int64_t)b * 128 + t];
    gU[t] += a;
}

// ------------------------------------------------------------------ backward layer
struct BwdArgs {
    int64_t n;
    int64_t ntiles;
    SellView<float2> K;
    const float *kdiag;
    const float *volp;
    const uint4 *Hin;        // h^l (operand a^l is rebuilt)
    const uint4 *dZ;         // dz^l rows (BF16, masked) -- hidden layers
    const float2 *dy;        // head: dy
    const uint4 *H4;         // head: h^4 (mask)
    const float *U;          // head: U (2 x 64)
    const uint4 *Wbimg;      // 128 x 64 BF16 operand image of W^l (rows = inputs)
    float *dA;               // n x 128: [dA_self, dA_nbr / (K_ii |V_i|)]
    float *dWpart;           // grid x 128 x 64 (rows = inputs)
    int *err;
};

template <bool HEAD, bool NEED_DA>
__global__ void __launch_bounds__(THREADS) k_bwd(BwdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16 *sDz = reinterpret_cast<__nv_bfloat16 *>(smem);                   // 128 nodes x 64 (K-major)
    uint4 *sWb = reinterpret_cast<uint4 *>(smem + TILE * CH * 2);                     // 128 in x 64 out
    __nv_bfloat16 *sAt = reinterpret_cast<__nv_bfloat16 *>(smem + TILE * CH * 2 + CIN * CH * 2);  // 128 in x 128 nodes
    __nv_bfloat16 *sDzt = sAt + CIN * TILE;                                            // 64 out x 128 nodes
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (NEED_DA)
        for (int i = tid; i < CIN * CH / 8; i += THREADS) sWb[i] = a.Wbimg[i];
    if (warp == 0) tmem_alloc(&tslot, 256);
    if (tid == 0) mbar_init(&mbar);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const uint32_t tm_dA = tmem, tm_dW = tmem + 128;
    const uint32_t id_dA = idesc_bf16(TILE, CIN);   // M = 128 nodes, N = 128 inputs
    const uint32_t id_dW = idesc_bf16(CIN, CH);     // M = 128 inputs, N = 64 outputs
    uint32_t phase = 0;
    bool failed = false;
    int iter = 0;
    __shared__ float sU[2 * CH];
    if (HEAD) {
        sU[tid] = a.U[tid];
        __syncthreads();
    }
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++iter) {
        const int64_t p = t * TILE + tid;
        float dz[CH];
        float av[CH];
        uint4 *rowDz = reinterpret_cast<uint4 *>(sDz);
        if (p < a.n) {
            if (HEAD) {
                float2 g = a.dy[p];
                const uint4 *h4 = a.H4 + p * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float f[8];
                    unpack8(h4[j], f);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        int c = 8 * j + i;
                        float v = sU[c] * g.x + sU[CH + c] * g.y;
                        dz[c] = f[i] > 0.f ? v : 0.f;
                    }
                }
                dz[CH - 1] = 0.f;
                // round once to BF16 so both GEMMs see the same dz
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint4 u = pack8(dz + 8 * j);
                    unpack8(u, dz + 8 * j);
                    rowDz[cm_off(tid, 8 * j, CH) >> 3] = u;
                }
            } else {
                const uint4 *dp = a.dZ + p * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint4 u = dp[j];
                    unpack8(u, dz + 8 * j);
                    rowDz[cm_off(tid, 8 * j, CH) >> 3] = u;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < CH; ++c) dz[c] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) rowDz[cm_off(tid, 8 * j, CH) >> 3] = make_uint4(0, 0, 0, 0);
        }
        // transposed operands of dW^T += a^T dz: column tid (this node)
#pragma unroll
        for (int c = 0; c < CH; ++c) sDzt[cm_off(c, tid, TILE)] = __float2bfloat16_rn(dz[c]);
        if (p < a.n) {
            const uint4 *hp = a.Hin + p * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) unpack8(hp[j], av + 8 * j);
        } else {
#pragma unroll
            for (int c = 0; c < CH; ++c) av[c] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) sAt[cm_off(c, tid, TILE)] = __float2bfloat16_rn(av[c]);
        if (p < a.n) {
            aggregate_row(a.K, a.kdiag, a.Hin, p, av);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) sAt[cm_off(CH + c, tid, TILE)] = __float2bfloat16_rn(av[c]);
        proxy_fence();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            if (NEED_DA) {
                uint32_t a0 = smem_u32(sDz), b0 = smem_u32(sWb);
#pragma unroll
                for (int ks = 0; ks < CH / 16; ++ks)
                    mma_bf16(tm_dA, sdesc(a0 + ks * 256, 128, CH * 16), sdesc(b0 + ks * 256, 128, CH * 16), id_dA,
                             ks > 0);
            }
            uint32_t a1 = smem_u32(sAt), b1 = smem_u32(sDzt);
#pragma unroll
            for (int ks = 0; ks < TILE / 16; ++ks)
                mma_bf16(tm_dW, sdesc(a1 + ks * 256, 128, TILE * 16), sdesc(b1 + ks * 256, 128, TILE * 16), id_dW,
                         (ks > 0 || iter > 0) ? 1u : 0u);
            mma_commit(&mbar);
        }
        const bool done = mbar_wait(&mbar, phase);
        if (__syncthreads_or(!done)) {
            failed = true;
            break;
        }
        phase ^= 1;
        tc_fence_after();
        if (NEED_DA) {
            const uint32_t lane_base = tm_dA + ((uint32_t)(warp * 32) << 16);
            float v[16];
            float sn = 0.f;
            if (p < a.n) sn = 1.f / (a.kdiag[p] * a.volp[p]);
#pragma unroll
            for (int c = 0; c < CIN; c += 16) {
                tmem_ld16(lane_base + c, v);
                if (p < a.n) {
                    float4 *dst = reinterpret_cast<float4 *>(a.dA + p * CIN + c);
                    float f = c < CH ? 1.f : sn;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        dst[i] = make_float4(v[4 * i] * f, v[4 * i + 1] * f, v[4 * i + 2] * f, v[4 * i + 3] * f);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    // dW^T partial of this CTA: lane = input feature (tid), 64 output columns
    {
        tc_fence_after();
        float v[16];
        const uint32_t lane_base = tm_dW + ((uint32_t)(warp * 32) << 16);
        float *dst = a.dWpart + ((int64_t)blockIdx.x * CIN + tid) * CH;
#pragma unroll
        for (int c = 0; c < CH; c += 16) {
            tmem_ld16(lane_base + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[c + i] = (iter > 0 && !failed) ? v[i] : 0.f;
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 256);
    if (failed && tid == 0) atomicExch(a.err, 1);
}

// dz^{l-1}_k = (dA_self_k - |V_k| sum_i K_ki dA~_i) masked by h^l_k > 0 (channel 63 -> 0)
__global__ void __launch_bounds__(128) k_dh(int64_t n, SellView<float2> K, const float *__restrict__ volp,
                                            const float *__restrict__ dA, const uint4 *__restrict__ Hl,
                                            uint4 *__restrict__ dZ) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    float acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = 0.f;
    int64_t s = p >> 5;
    int lane = (int)(p & 31);
    int64_t beg = K.sptr[s];
    int w = (int)((K.sptr[s + 1] - beg) >> 5);
    for (int k = 0; k < w; ++k) {
        int64_t q = beg + (int64_t)k * SELL_C + lane;
        float2 kv = K.val[q];
        if (kv.x == 0.f && kv.y == 0.f) continue;
        const float4 *src = reinterpret_cast<const float4 *>(dA + (int64_t)K.col[q] * CIN + CH);
#pragma unroll
        for (int j = 0; j < CH / 4; ++j) {
            float4 u = __ldg(src + j);
            acc[4 * j] += kv.x * u.x - kv.y * u.y;
            acc[4 * j + 1] += kv.x * u.y + kv.y * u.x;
            acc[4 * j + 2] += kv.x * u.z - kv.y * u.w;
            acc[4 * j + 3] += kv.x * u.w + kv.y * u.z;
        }
    }
    float vk = -volp[p];
    const float4 *self = reinterpret_cast<const float4 *>(dA + p * CIN);
    const uint4 *hl = Hl + p * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float hf[8], o[8];
        unpack8(hl[j], hf);
        float4 s0 = self[2 * j], s1 = self[2 * j + 1];
        float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float g = sv[i] + vk * acc[8 * j + i];
            o[i] = hf[i] > 0.f ? g : 0.f;
        }
        if (j == 7) o[7] = 0.f;
        dZ[p * 8 + j] = pack8(o);
    }
}

// grad W^l (64 out x 128 in) += sum over CTAs of the partial dW^T (128 in x 64 out)
__global__ void k_dw_final(const float *part, int np, float *gW) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;   // over 64 x 128 in output layout
    if (idx >= WSZ) return;
    int o = idx / CIN, i = idx % CIN;
    float a = 0.f;
    for (int b = 0; b < np; ++b) a += part[((int64_t)b * CIN + i) * CH + o];
    gW[idx] += a;
}

// ------------------------------------------------------------------ zero-guess fallback
// per-block partials of sum |V| |b - J x|^2 and sum |V| |b|^2 (FP64 J)
__global__ void k_fallback_part(int64_t n, SellView<double2> K, const double *__restrict__ kdiag,
                                const double *__restrict__ volp, const double2 *__restrict__ psi,
                                const double2 *__restrict__ b, const double2 *__restrict__ x, double *part) {
    __shared__ double sh[32];
    double rr = 0, bb = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = p >> 5;
        int lane = (int)(p & 31);
        int64_t beg = K.sptr[s];
        int w = (int)((K.sptr[s + 1] - beg) >> 5);
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < w; ++k) {
            int64_t q = beg + (int64_t)k * SELL_C + lane;
            cfma(acc, K.val[q], x[K.col[q]]);
        }
        double2 ps = psi[p], xv = x[p], bv = b[p];
        double d = kdiag[p] - 1.0 + 2.0 * (ps.x * ps.x + ps.y * ps.y);
        double p2r = ps.x * ps.x - ps.y * ps.y, p2i = 2.0 * ps.x * ps.y;
        double jx = acc.x + d * xv.x + (p2r * xv.x + p2i * xv.y);
        double jy = acc.y + d * xv.y + (p2i * xv.x - p2r * xv.y);
        double rx = bv.x - jx, ry = bv.y - jy;
        rr += volp[p] * (rx * rx + ry * ry);
        bb += volp[p] * (bv.x * bv.x + bv.y * bv.y);
    }
    double t1 = block_sum(rr, sh);
    double t2 = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
}
// flag = 1 if the guess lowers the residual below ||b||_D (and is finite)
__global__ void k_fallback_decide(const double *part, int np, int *flag) {
    __shared__ double sh[32];
    double a = 0, c = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        a += part[2 * i];
        c += part[2 * i + 1];
    }
    double rr = block_sum(a, sh);
    double bb = block_sum(c, sh);
    if (threadIdx.x == 0) *flag = (rr < bb) ? 1 : 0;   // false for NaN
}
__global__ void k_fallback_apply(int64_t n, const int *flag, double2 *x) {
    if (*flag) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        x[p] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------ parameters
__global__ void k_adam(int np, float *th, const float *g, float *m, float *v, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 operand images of every W^l: forward (rows = 64 outputs, K = 128 inputs)
// and backward (rows = 128 inputs, K = 64 outputs)
__global__ void k_pack(const float *th, __nv_bfloat16 *Wf, __nv_bfloat16 *Wb) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NL * WSZ) return;
    int l = idx / WSZ, r = idx % WSZ;
    int o = r / CIN, i = r % CIN;
    __nv_bfloat16 v = __float2bfloat16_rn(th[idx]);
    Wf[(int64_t)l * WSZ + cm_off(o, i, CIN)] = v;
    Wb[(int64_t)l * WSZ + cm_off(i, o, CH)] = v;
}

}  // namespace ws
}  // namespace gl

using namespace gl;
using namespace gl::ws;

struct gl_warmstart_s {
    DBuf<float> theta, grad, m, v;
    DBuf<__nv_bfloat16> Wf, Wb;
    int64_t t = 0;           // Adam step count
    int64_t cap = 0;         // nodes the work buffers hold
    DBuf<__nv_bfloat16> H;   // 5 x cap x 64
    DBuf<__nv_bfloat16> dZ;  // cap x 64
    DBuf<float> dA;          // cap x 128
    DBuf<float2> xh, r, dy;
    DBuf<double> bn, part, loss;
    DBuf<float> dWpart, dUpart;
    DBuf<int> err;
    DBuf<int> used;          // zero-guess fallback decision of the last solve
    DBuf<double> fpart;      // its partials
    // the hint: J a, the residual r = b - alpha J a, the hint in the solve ordering,
    // partials and (alpha, 1 / ||a||_D)
    DBuf<double2> qa, rb, hp;
    DBuf<double> hpart, hsc;
    int fwd_grid = 0, bwd_grid = 0;
};

namespace {

template <typename F>
gl_status ws_guard(F &&f) {
    try {
        set_error("");
        return f();
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return GL_ERR_OOM;
    }
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

void ws_pack(gl_warmstart_s *w, cudaStream_t s) {
    k_pack<<<grid_for(NL * WSZ, 256), 256, 0, s>>>(w->theta.get(), w->Wf.get(), w->Wb.get());
    GL_LAUNCH_CHECK();
}

void ws_reserve(gl_warmstart_s *w, int64_t n) {
    if (n <= w->cap) return;
    w->H.alloc((size_t)5 * n * CH);
    w->dZ.alloc((size_t)n * CH);
    w->dA.alloc((size_t)n * CIN);
    w->xh.alloc(n);
    w->r.alloc(n);
    w->dy.alloc(n);
    w->qa.alloc(n);
    w->rb.alloc(n);
    w->hp.alloc(n);
    w->cap = n;
}

void ws_setup_kernels(gl_warmstart_s *w) {
    if (w->fwd_grid) return;
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM));
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_LAST_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM));
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_LAST_PREDICT>, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM));
    // ask for the largest shared-memory carveout, or only one CTA fits an SM
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_HIDDEN>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_LAST_TRAIN>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    GL_CUDA(cudaFuncSetAttribute(k_fwd<FWD_LAST_PREDICT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    GL_CUDA(cudaFuncSetAttribute(k_bwd<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int dev = 0, nsm = 0, smem_sm = 0;
    GL_CUDA(cudaGetDevice(&dev));
    GL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GL_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // CTAs per SM from the kernels' own register and shared-memory use (the
    // occupancy query reports 0 for these kernels); tensor memory holds 512
    // columns per SM: the forward kernel takes 64 and the backward 256.  The
    // CTAs of one launch never wait on each other, so an estimate that is too
    // high only queues CTAs.
    auto per_sm = [&](const void *fn, int dyn, int cap) {
        cudaFuncAttributes fa;
        GL_CUDA(cudaFuncGetAttributes(&fa, fn));
        int regs = ((fa.numRegs + 7) / 8) * 8 * THREADS;
        int by_regs = regs > 0 ? 65536 / regs : cap;
        int by_smem = smem_sm / (dyn + (int)fa.sharedSizeBytes + 1024);
        return std::max(1, std::min(cap, std::min(by_regs, by_smem)));
    };
    int f = std::min(per_sm((const void *)k_fwd<FWD_HIDDEN>, FWD_SMEM, 8),
                     std::min(per_sm((const void *)k_fwd<FWD_LAST_TRAIN>, FWD_SMEM, 8),
                              per_sm((const void *)k_fwd<FWD_LAST_PREDICT>, FWD_SMEM, 8)));
    int b = std::min(per_sm((const void *)k_bwd<true, true>, BWD_SMEM, 2),
                     std::min(per_sm((const void *)k_bwd<false, true>, BWD_SMEM, 2),
                              per_sm((const void *)k_bwd<false, false>, BWD_SMEM, 2)));
    w->fwd_grid = f * nsm;
    w->bwd_grid = b * nsm;
    w->part.alloc(RED_BLOCKS);
    w->bn.alloc(2);
    w->dWpart.alloc((size_t)w->bwd_grid * CIN * CH);
    w->dUpart.alloc((size_t)DU_BLOCKS * 128);
    w->err.alloc(1);
    GL_CUDA(cudaMemset(w->err.get(), 0, sizeof(int)));
    w->used.alloc(1);
    w->fpart.alloc(2 * RED_BLOCKS);
    w->hpart.alloc(3 * RED_BLOCKS);
    w->hsc.alloc(2);
}

// with a hint (solve ordering): alpha and 1 / ||a||_D into hsc, and the residual
// b - alpha J a the network works on; returns the right-hand side to use
const double2 *ws_hint(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p,
                       const double2 *hint_p, cudaStream_t s) {
    if (!hint_p) return b_p;
    const int64_t n = m->n;
    jacobian_apply_p(m, psi_p, hint_p, w->qa.get(), s);
    note_launch(3);
    k_hint_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->volp.get(), w->qa.get(), b_p, hint_p, w->hpart.get());
    k_hint_final<<<1, 1024, 0, s>>>(w->hpart.get(), w->hsc.get());
    k_hint_resid<<<grid_for(n, 256), 256, 0, s>>>(n, w->hsc.get(), b_p, w->qa.get(), w->rb.get());
    GL_LAUNCH_CHECK();
    return w->rb.get();
}

__nv_bfloat16 *Hbuf(gl_warmstart_s *w, int l) { return w->H.get() + (size_t)l * w->cap * CH; }

// forward pass in the solve ordering; train: keep h^1..h^4 and x^, else write x0.
// b_p is the network's right-hand side (the residual the hint leaves, when there
// is one: see ws_hint); hint_p (nullable) fills the hint channels
void ws_forward(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, bool train, double2 *x0_p,
                cudaStream_t s, const double2 *hint_p = nullptr) {
    const int64_t n = m->n;
    k_bnorm_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->volp.get(), b_p, w->part.get());
    k_bnorm_final<<<1, 1024, 0, s>>>(w->part.get(), RED_BLOCKS, w->bn.get());
    k_features<<<grid_for(n, 256), 256, 0, s>>>(n, b_p, psi_p, w->bn.get(), hint_p, w->hsc.get(),
                                                reinterpret_cast<uint4 *>(Hbuf(w, 0)));
    GL_LAUNCH_CHECK();
    note_launch(3);
    const int64_t ntiles = (n + TILE - 1) / TILE;
    const int grid = (int)std::min<int64_t>(ntiles, w->fwd_grid);
    // algorithmic bytes of one layer: each node's h row read once (neighbour rows
    // are re-reads of the same array), its K row (value + column) and K_ii, and
    // the written h row (the last layer of a prediction writes x0 instead)
    const double k_bytes = (double)m->K32.nnz_stored * (sizeof(float2) + 4) + (double)n * 4;
    for (int l = 0; l < NL; ++l) {
        const bool last_pred = (l == NL - 1) && !train;
        ProfScope ps("wsf", (double)n * (CH * 2 + (last_pred ? 16 : CH * 2)) + k_bytes, s);
        FwdArgs a{};
        a.n = n;
        a.ntiles = ntiles;
        a.K = m->K32.view();
        a.kdiag = m->kdiag32.get();
        // prediction ping-pongs between buffers 0 and 1
        int in = train ? l : (l & 1), out = train ? l + 1 : ((l + 1) & 1);
        a.Hin = reinterpret_cast<const uint4 *>(Hbuf(w, in));
        a.Hout = reinterpret_cast<uint4 *>(Hbuf(w, out));
        a.Wimg = reinterpret_cast<const uint4 *>(w->Wf.get() + (size_t)l * WSZ);
        a.U = w->theta.get() + NL * WSZ;
        a.xhat = w->xh.get();
        a.x0 = x0_p;
        a.bn = w->bn.get();
        a.err = w->err.get();
        if (l < NL - 1)
            k_fwd<FWD_HIDDEN><<<grid, THREADS, FWD_SMEM, s>>>(a);
        else if (train)
            k_fwd<FWD_LAST_TRAIN><<<grid, THREADS, FWD_SMEM, s>>>(a);
        else
            k_fwd<FWD_LAST_PREDICT><<<grid, THREADS, FWD_SMEM, s>>>(a);
        GL_LAUNCH_CHECK();
    }
}

// loss (added to loss[slot] with weight `scale`) and gradient (added to grad with
// weight `scale`) of one sample; requires ws_forward(train = true) just before
void ws_backward(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, double scale,
                 double *loss, int slot, cudaStream_t s) {
    const int64_t n = m->n;
    note_launch(5);
    k_resid<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->K32.view(), m->kdiag32.get(), m->volp32.get(), psi_p, b_p,
                                               w->bn.get(), w->xh.get(), w->r.get(), w->part.get());
    k_loss_acc<<<1, 1024, 0, s>>>(w->part.get(), RED_BLOCKS, scale, loss, slot);
    k_gout<<<grid_for(n, 256), 256, 0, s>>>(n, m->K32.view(), m->kdiag32.get(), m->volp32.get(), psi_p, w->r.get(),
                                            (float)scale, w->dy.get());
    float *gU = w->grad.get() + NL * WSZ;
    k_du_part<<<DU_BLOCKS, 128, 0, s>>>(n, w->dy.get(), Hbuf(w, NL), w->dUpart.get());
    k_du_final<<<1, 128, 0, s>>>(w->dUpart.get(), DU_BLOCKS, gU);
    GL_LAUNCH_CHECK();
    const int64_t ntiles = (n + TILE - 1) / TILE;
    const int grid = (int)std::min<int64_t>(ntiles, w->bwd_grid);
    const double k_bytes = (double)m->K32.nnz_stored * (sizeof(float2) + 4) + (double)n * 8;
    for (int l = NL - 1; l >= 0; --l) {
        // algorithmic bytes: h^l and dz rows read, K row, dA rows written
        note_launch(l > 0 ? 2 : 1);
        BwdArgs a{};
        a.n = n;
        a.ntiles = ntiles;
        a.K = m->K32.view();
        a.kdiag = m->kdiag32.get();
        a.volp = m->volp32.get();
        a.Hin = reinterpret_cast<const uint4 *>(Hbuf(w, l));
        a.dZ = reinterpret_cast<const uint4 *>(w->dZ.get());
        a.dy = w->dy.get();
        a.H4 = reinterpret_cast<const uint4 *>(Hbuf(w, NL));
        a.U = w->theta.get() + NL * WSZ;
        a.Wbimg = reinterpret_cast<const uint4 *>(w->Wb.get() + (size_t)l * WSZ);
        a.dA = w->dA.get();
        a.dWpart = w->dWpart.get();
        a.err = w->err.get();
        {
            // algorithmic bytes: h^l and dz rows read, K row, dA rows written
            ProfScope ps("wsb", (double)n * (CH * 2 + CH * 2 + (l > 0 ? CIN * 4 : 0)) + k_bytes, s);
            if (l == NL - 1)
                k_bwd<true, true><<<grid, THREADS, BWD_SMEM, s>>>(a);
            else if (l > 0)
                k_bwd<false, true><<<grid, THREADS, BWD_SMEM, s>>>(a);
            else
                k_bwd<false, false><<<grid, THREADS, BWD_SMEM, s>>>(a);
        }
        GL_LAUNCH_CHECK();
        k_dw_final<<<grid_for(WSZ, 256), 256, 0, s>>>(w->dWpart.get(), grid, w->grad.get() + (size_t)l * WSZ);
        GL_LAUNCH_CHECK();
        if (l > 0) {
            k_dh<<<grid_for(n, 128), 128, 0, s>>>(n, m->K32.view(), m->volp32.get(), w->dA.get(),
                                                  reinterpret_cast<const uint4 *>(Hbuf(w, l)),
                                                  reinterpret_cast<uint4 *>(w->dZ.get()));
            GL_LAUNCH_CHECK();
        }
    }
}

void check_err(gl_warmstart_s *w, cudaStream_t s) {
    int e = 0;
    GL_CUDA(cudaMemcpyAsync(&e, w->err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    if (e) {
        GL_CUDA(cudaMemsetAsync(w->err.get(), 0, sizeof(int), s));
        throw Error{GL_ERR_TIMEOUT, "warm-start network: a tensor-core completion wait ran out"};
    }
}

void ensure_mesh_scratch(gl_mesh_s *m) {
    if (m->t0.n != (size_t)m->n) {
        m->t0.alloc(m->n);
        m->t1.alloc(m->n);
        m->t2.alloc(m->n);
    }
}

}  // namespace

namespace gl {

// x0_p = network guess for b_p (solve ordering; hint_p nullable, solve ordering)
void warmstart_predict_p(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, double2 *x0_p,
                         cudaStream_t s, const double2 *hint_p) {
    mesh_ensure_fp32(m, s);
    ws_setup_kernels(w);
    ws_reserve(w, m->n);
    const double2 *r_p = ws_hint(w, m, psi_p, b_p, hint_p, s);
    ws_forward(w, m, psi_p, r_p, false, x0_p, s, hint_p);
    if (hint_p) {
        note_launch();
        k_hint_add<<<grid_for(m->n, 256), 256, 0, s>>>(m->n, w->hsc.get(), hint_p, x0_p);
        GL_LAUNCH_CHECK();
    }
}

void warmstart_apply_p(gl_warmstart_s *w, gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, double2 *x_p,
                       cudaStream_t s, const double2 *hint_nat) {
    const double2 *hint_p = nullptr;
    if (hint_nat) {
        ws_reserve(w, m->n);
        permute_in(m->n, m->perm.get(), hint_nat, w->hp.get(), s);
        hint_p = w->hp.get();
    }
    warmstart_predict_p(w, m, psi_p, b_p, x_p, s, hint_p);
    note_launch(3);
    k_fallback_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->n, m->K.view(), m->kdiag.get(), m->volp.get(), psi_p, b_p,
                                                       x_p, w->fpart.get());
    k_fallback_decide<<<1, 1024, 0, s>>>(w->fpart.get(), RED_BLOCKS, w->used.get());
    k_fallback_apply<<<grid_for(m->n, 256, 4 * NUM_SMS_HINT), 256, 0, s>>>(m->n, w->used.get(), x_p);
    GL_LAUNCH_CHECK();
}

// the hint's minimal-residual multiple alone (no network): x_p = alpha a with
// alpha = <J a, b>_R / <J a, J a>_R, which is never a worse guess than zero
void hint_guess_p(gl_mesh_s *m, const double2 *psi_p, const double2 *b_p, const double2 *hint_nat, double2 *x_p,
                  cudaStream_t s) {
    struct HintWork {
        DBuf<double2> a, q;
        DBuf<double> part, hs;
    };
    static thread_local HintWork H;
    const int64_t n = m->n;
    if (H.a.n != (size_t)n) {
        H.a.alloc(n);
        H.q.alloc(n);
    }
    if (!H.part.get()) {
        H.part.alloc(3 * RED_BLOCKS);
        H.hs.alloc(2);
    }
    permute_in(n, m->perm.get(), hint_nat, H.a.get(), s);
    jacobian_apply_p(m, psi_p, H.a.get(), H.q.get(), s);
    note_launch(3);
    k_hint_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m->volp.get(), H.q.get(), b_p, H.a.get(), H.part.get());
    k_hint_final<<<1, 1024, 0, s>>>(H.part.get(), H.hs.get());
    k_hint_set<<<grid_for(n, 256), 256, 0, s>>>(n, H.hs.get(), H.a.get(), x_p);
    GL_LAUNCH_CHECK();
}

int warmstart_used(gl_warmstart_s *w, cudaStream_t s) {
    check_err(w, s);
    int u = 0;
    GL_CUDA(cudaMemcpyAsync(&u, w->used.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return u;
}

}  // namespace gl

extern "C" {

gl_status gl_warmstart_create(const float *params, gl_warmstart *out) {
    return ws_guard([&] {
        GL_REQUIRE(out, GL_ERR_ARG, "out must not be NULL");
        auto *w = new gl_warmstart_s();
        try {
            w->theta.alloc(NPARAM);
            w->grad.alloc(NPARAM);
            w->m.alloc(NPARAM);
            w->v.alloc(NPARAM);
            w->Wf.alloc((size_t)NL * WSZ);
            w->Wb.alloc((size_t)NL * WSZ);
            w->loss.alloc(1);
            if (params)
                GL_CUDA(cudaMemcpy(w->theta.get(), params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
            else
                GL_CUDA(cudaMemset(w->theta.get(), 0, NPARAM * sizeof(float)));
            GL_CUDA(cudaMemset(w->grad.get(), 0, NPARAM * sizeof(float)));
            GL_CUDA(cudaMemset(w->m.get(), 0, NPARAM * sizeof(float)));
            GL_CUDA(cudaMemset(w->v.get(), 0, NPARAM * sizeof(float)));
            ws_pack(w, 0);
            GL_CUDA(cudaDeviceSynchronize());
        } catch (...) {
            delete w;
            throw;
        }
        *out = w;
        return GL_OK;
    });
}

gl_status gl_warmstart_destroy(gl_warmstart w) {
    return ws_guard([&] {
        if (w) {
            cudaDeviceSynchronize();
            delete w;
        }
        return GL_OK;
    });
}

gl_status gl_warmstart_get_params(gl_warmstart w, float *params) {
    return ws_guard([&] {
        GL_REQUIRE(w && params, GL_ERR_ARG, "NULL argument");
        GL_CUDA(cudaMemcpy(params, w->theta.get(), NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_warmstart_set_params(gl_warmstart w, const float *params) {
    return ws_guard([&] {
        GL_REQUIRE(w && params, GL_ERR_ARG, "NULL argument");
        GL_CUDA(cudaMemcpy(w->theta.get(), params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
        GL_CUDA(cudaMemset(w->m.get(), 0, NPARAM * sizeof(float)));
        GL_CUDA(cudaMemset(w->v.get(), 0, NPARAM * sizeof(float)));
        w->t = 0;
        ws_pack(w, 0);
        GL_CUDA(cudaDeviceSynchronize());
        return GL_OK;
    });
}

gl_status gl_warmstart_predict(gl_warmstart w, gl_mesh m, const void *psi, const void *b, const void *hint, void *x0,
                               void *stream) {
    return ws_guard([&] {
        GL_REQUIRE(w && m && psi && b && x0, GL_ERR_ARG, "NULL argument");
        cudaStream_t s = as_stream(stream);
        ensure_mesh_scratch(m);
        permute_in(m->n, m->perm.get(), (const double2 *)psi, m->t0.get(), s);
        permute_in(m->n, m->perm.get(), (const double2 *)b, m->t1.get(), s);
        const double2 *hp = nullptr;
        if (hint) {
            ws_setup_kernels(w);
            ws_reserve(w, m->n);
            permute_in(m->n, m->perm.get(), (const double2 *)hint, w->hp.get(), s);
            hp = w->hp.get();
        }
        warmstart_predict_p(w, m, m->t0.get(), m->t1.get(), m->t2.get(), s, hp);
        permute_out(m->n, m->perm.get(), m->t2.get(), (double2 *)x0, s);
        check_err(w, s);
        return GL_OK;
    });
}

gl_status gl_warmstart_grad(gl_warmstart w, gl_mesh m, const void *psi, const void *b, const void *hint,
                            float *grad_host, double *loss_out, void *stream) {
    return ws_guard([&] {
        GL_REQUIRE(w && m && psi && b, GL_ERR_ARG, "NULL argument");
        cudaStream_t s = as_stream(stream);
        ensure_mesh_scratch(m);
        mesh_ensure_fp32(m, s);
        ws_setup_kernels(w);
        ws_reserve(w, m->n);
        permute_in(m->n, m->perm.get(), (const double2 *)psi, m->t0.get(), s);
        permute_in(m->n, m->perm.get(), (const double2 *)b, m->t1.get(), s);
        const double2 *hp = nullptr;
        if (hint) {
            permute_in(m->n, m->perm.get(), (const double2 *)hint, w->hp.get(), s);
            hp = w->hp.get();
        }
        GL_CUDA(cudaMemsetAsync(w->grad.get(), 0, NPARAM * sizeof(float), s));
        GL_CUDA(cudaMemsetAsync(w->loss.get(), 0, sizeof(double), s));
        const double2 *r_p = ws_hint(w, m, m->t0.get(), m->t1.get(), hp, s);
        ws_forward(w, m, m->t0.get(), r_p, true, nullptr, s, hp);
        ws_backward(w, m, m->t0.get(), r_p, 1.0, w->loss.get(), 0, s);
        check_err(w, s);
        if (grad_host) GL_CUDA(cudaMemcpy(grad_host, w->grad.get(), NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
        if (loss_out) GL_CUDA(cudaMemcpy(loss_out, w->loss.get(), sizeof(double), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_warmstart_train(gl_warmstart w, int count, const gl_mesh *meshes, const void *const *psi,
                             const void *const *b, const void *const *hints, int steps, int batch, float lr,
                             double *loss_out, void *stream) {
    return ws_guard([&] {
        GL_REQUIRE(w && meshes && psi && b, GL_ERR_ARG, "NULL argument");
        GL_REQUIRE(count > 0 && steps >= 0 && batch > 0 && lr > 0, GL_ERR_ARG, "bad count, steps, batch or lr");
        cudaStream_t s = as_stream(stream);
        ws_setup_kernels(w);
        for (int j = 0; j < count; ++j) {
            GL_REQUIRE(meshes[j] && psi[j] && b[j], GL_ERR_ARG, "NULL sample");
            ensure_mesh_scratch(meshes[j]);
            mesh_ensure_fp32(meshes[j], s);
            ws_reserve(w, meshes[j]->n);
        }
        DBuf<double> losses(std::max(steps, 1));
        GL_CUDA(cudaMemsetAsync(losses.get(), 0, losses.bytes(), s));
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        for (int st = 0; st < steps; ++st) {
            GL_CUDA(cudaMemsetAsync(w->grad.get(), 0, NPARAM * sizeof(float), s));
            for (int j = 0; j < batch; ++j) {
                int k = (int)(((int64_t)st * batch + j) % count);
                gl_mesh_s *m = meshes[k];
                permute_in(m->n, m->perm.get(), (const double2 *)psi[k], m->t0.get(), s);
                permute_in(m->n, m->perm.get(), (const double2 *)b[k], m->t1.get(), s);
                const double2 *hp = nullptr;
                if (hints && hints[k]) {
                    permute_in(m->n, m->perm.get(), (const double2 *)hints[k], w->hp.get(), s);
                    hp = w->hp.get();
                }
                const double2 *r_p = ws_hint(w, m, m->t0.get(), m->t1.get(), hp, s);
                ws_forward(w, m, m->t0.get(), r_p, true, nullptr, s, hp);
                ws_backward(w, m, m->t0.get(), r_p, 1.0 / batch, losses.get(), st, s);
            }
            w->t += 1;
            float c1 = 1.f - powf(b1, (float)w->t), c2 = 1.f - powf(b2, (float)w->t);
            k_adam<<<grid_for(NPARAM, 256), 256, 0, s>>>(NPARAM, w->theta.get(), w->grad.get(), w->m.get(),
                                                         w->v.get(), lr, b1, b2, c1, c2, eps);
            GL_LAUNCH_CHECK();
            ws_pack(w, s);
            if ((st & 15) == 15) check_err(w, s);
        }
        check_err(w, s);
        if (loss_out && steps > 0)
            GL_CUDA(cudaMemcpy(loss_out, losses.get(), steps * sizeof(double), cudaMemcpyDeviceToHost));
        return GL_OK;
    });
}

gl_status gl_warmstart_adam_step(gl_warmstart w, const float *grad_host, float lr) {
    return ws_guard([&] {
        GL_REQUIRE(w && grad_host && lr > 0, GL_ERR_ARG, "bad argument");
        GL_CUDA(cudaMemcpy(w->grad.get(), grad_host, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
        w->t += 1;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        float c1 = 1.f - powf(b1, (float)w->t), c2 = 1.f - powf(b2, (float)w->t);
        k_adam<<<grid_for(NPARAM, 256), 256>>>(NPARAM, w->theta.get(), w->grad.get(), w->m.get(), w->v.get(), lr, b1,
                                               b2, c1, c2, eps);
        GL_LAUNCH_CHECK();
        ws_pack(w, 0);
        GL_CUDA(cudaDeviceSynchronize());
        return GL_OK;
    });
}

}  // extern "C"
