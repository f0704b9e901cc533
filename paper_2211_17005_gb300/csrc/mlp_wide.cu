// Neural regression of Sec. 2 at hidden width 128: the NN+ network of eq. (e:nnp)
// with two hidden ReLU layers of 128 units on the F <= 32 standardised factors,
// trained at each date by Algorithm 1 (BaseAlg) inside Algorithm 2 (backward
// learning), for samples large enough that one Adam batch covers many 128-path
// tiles (2^20 paths in 32 batches: 256 tiles per step).
//
// Kernels of one date, in order on one stream:
//   wide_train_kernel   one epoch of Adam steps on a cooperative grid (one CTA per
//                       SM, at most one tile per CTA and round)
//   wide_sweep_kernel   the refit's Gram matrix: a full-sample forward pass in the
//                       trainer's layout (one CTA per SM)
//   wide_fwd_kernel     full-sample forward passes: the epoch loss with the
//                       best-parameter choice, or the predictions (two tiles of a
//                       CTA in a pipeline, one CTA per SM)
//   mlp_refit_kernel    (shared) Gram sum, FP64 Cholesky, new (w3, b3)
//
// Every CTA owns one 128-row tile slot worked by its two warpgroups; warpgroup h
// takes hidden columns [64 h, 64 h + 64) in every epilogue. Per tile:
//   GEMM1  D = X W1^T                      (K = 32 padded inputs, N = 128)
//   GEMM2  D = H1 W2^T                     (K = 128, N = 128)
//   GEMM3  D = dH2 W2                      (K = 128; the W2 image read MN-major)
//   GEMMW  DW2 (+)= dH2^T [H1 | 1]          (M = 128, N = 144, K = the 128 paths)
//          DW1 (+)= dH1^T [X | 1]           (M = 128, N = 48)
// with the per-path rows A = [dH2 | dH1] (256 wide) and B = [H1 | 1 | X | 1]
// (192 wide) in K-major core matrices, read MN-major by GEMMW. BF16 operands in
// shared memory, FP32 accumulators in tensor memory (D at columns [0, 128), DW2 at
// [128, 272), DW1 at [320, 368)); biases, ReLU, the output layer and the loss in
// FP32 on the CUDA cores.
//
// One Adam step on the grid: every CTA writes its FP32 gradient partial to global
// memory (column order q); after a grid barrier CTA c owns slice c of the
// parameter vector: it sums the slice over all CTAs' partials (fixed order, every
// load of a thread in flight at once), applies Adam (moments and FP32 master values
// in global memory) and writes the new FP32 values and their BF16 images; after a
// second grid barrier every CTA fetches the images and the FP32 vectors by bulk
// copies. The grid barrier is one arrival counter with bounded waits (a wait that
// gives up sets the status word; every other wait then ends at once).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <climits>
#include <atomic>
#include <mutex>
#include <string>

#include "cva_internal.h"
#include "mlp_common.cuh"
#include "umma.cuh"

namespace cva {

namespace {

constexpr int kWThreads = 256;
constexpr uint32_t kGridPolls = 1u << 22;   // default limit of a grid-barrier wait (polls 32 ns apart)

struct WL {
    static constexpr int U = 128;
    static constexpr int NP = 35 * U + U * U + 2;
    static constexpr int NPpad = (NP + 63) / 64 * 64;
    static constexpr int oW1 = 0, ob1 = kIn * U, oW2 = ob1 + U, ob2 = oW2 + U * U, ow3 = ob2 + U, ob3 = ow3 + U,
                         omu = ob3 + 1;
    static constexpr int Z = U + 2;
    static constexpr int wA = 2 * U, wB = U + 64;                 // row widths (elements)
    static constexpr int cOne1 = U, cX = U + 16, cOne2 = U + 48;  // columns of B
    // shared memory (bytes)
    static constexpr int sA = 0;
    static constexpr int sB = sA + kRows * wA * 2;
    static constexpr int sW1 = sB + kRows * wB * 2;               // W1 image [U][32], K-major
    static constexpr int sW2 = sW1 + U * kIn * 2;                 // W2 image [U][U], K-major
    static constexpr int sVec = sW2 + U * U * 2;                  // b1 | b2 | w3 | b3, mu (FP32)
    static constexpr int sStage = sVec + 512 * 4;                 // [kIn + 1][128] FP32 inputs, target
    static constexpr int sStats = sStage + (kIn + 1) * kRows * 4; // mean[32], 1/std[32]
    static constexpr int sGsl = sStats + 2 * kIn * 4;             // [8 warps][66] output-layer gradient sums
    static constexpr int sOut = sGsl + 8 * 66 * 4;                // [2][128] half outputs
    static constexpr int sRed = sOut + 2 * kRows * 4;             // [256] float4 owner sums
    static constexpr int bytes = sRed + kWThreads * 16;
    static constexpr int img_elems = U * kIn + U * U;             // BF16 images of W1 | W2
    static constexpr uint32_t tmem_cols = 512;
    static constexpr uint32_t cD = 0, cW2 = 128, cW1 = 320;
    static constexpr bool kGram = true;   // the layout holds the Gram pass's A buffer
    // vector offsets inside sVec
    static constexpr int vb1 = 0, vb2 = U, vw3 = 2 * U, vb3 = 3 * U, vmu = 3 * U + 1;

    // W1 and W2 in column order (q) for the partials and the master copy; global
    // parameters keep the row order (p)
    __host__ __device__ static int p_of(int q)
    {
        if (q < ob1) return oW1 + (q % U) * kIn + q / U;
        if (q >= oW2 && q < ob2) {
            const int t = q - oW2;
            return oW2 + (t % U) * U + t / U;
        }
        return q;
    }
};
static_assert(WL::sStage % 128 == 0, "TMA destination must be 128-byte aligned");
static_assert(WL::bytes <= 227 * 1024, "shared memory");

// Pipelined forward layout of the loss and prediction passes: two B buffers and two
// TMEM accumulators, so that the first GEMM of a CTA's next tile runs while the
// output layer of its current tile is evaluated, and kStages staging buffers, so that
// the inputs of the next kStages tiles are in flight (one CTA per SM).
struct WLP : WL {
    static constexpr int kStages = 4;
    static constexpr int stage_bytes = (kIn + 1) * kRows * 4;
    static constexpr int sA = -1;
    static constexpr int sB = 0;
    static constexpr int sB1 = sB + kRows * wB * 2;               // the second B buffer
    static constexpr int sW1 = sB1 + kRows * wB * 2;
    static constexpr int sW2 = sW1 + U * kIn * 2;
    static constexpr int sVec = sW2 + U * U * 2;
    static constexpr int sStage = sVec + 512 * 4;                // [kStages][kIn + 1][128] FP32 inputs, target
    static constexpr int sStats = sStage + kStages * stage_bytes;
    static constexpr int sGsl = sStats + 2 * kIn * 4;
    static constexpr int sOut = sGsl + 8 * 66 * 4;
    static constexpr int bytes = sOut + 2 * kRows * 4;
    static constexpr uint32_t tmem_cols = 256;                   // D of tile k at 128 (k & 1)
};
static_assert(WLP::sStage % 128 == 0 && WLP::stage_bytes % 128 == 0 && WLP::sB1 % 1024 == 0,
              "TMA destinations and operand alignment");
static_assert(WLP::bytes <= 227 * 1024, "shared memory");

// byte offset of element c of row r in a BF16 row buffer of width w (K-major core
// matrices of 8 rows x 16 bytes)
__host__ __device__ constexpr uint32_t wrow_off(uint32_t r, uint32_t c, uint32_t w)
{
    return (r >> 3) * (w / 8u) * 128u + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

struct WTrainArgs {
    const float *targ;             // [M] targets (features through the tensor map)
    int F;
    uint32_t M;
    int tiles_per_batch, n_steps, step0, pos;
    float lr, beta1, beta2, eps;
    const float *init;             // [NP] row order: parameters at the start of the launch
    float *params;                 // [NP] row order: parameters at its end
    float *snap;                   // [NP] row order: a second copy of them (nullable)
    float *best;                   // step0 == 0: receives init ...
    double *best_loss;             // ... and +inf
    float *adam_m, *adam_v;        // [NPpad] q order; step0 == 0: start at zero
    float *gq;                     // [NPpad] q order: FP32 master parameters
    uint16_t *gimg;                // [img_elems] BF16 images of W1 | W2 (shared-memory layout)
    float *gpart;                  // [grid][NPpad] q order: gradient partials
    unsigned *flags;               // [1] grid barrier: arrivals over the launch (zero at launch)
    uint32_t grid_polls;           // polls after which a grid-barrier wait gives up
    const float *stats;            // mean[32], 1/std[32]
    float *grad_out;               // [NP] row order: gradient of the first step (nullable)
    int *err;
};

struct WSweepArgs {
    const float *targ;
    int F;
    uint32_t M;
    int mode;                      // 0 loss, 1 Gram of the refit, 2 predictions
    const float *theta;            // [NP] row order
    const float *stats;
    double *part;                  // per-CTA partials
    unsigned *count;               // last-CTA ticket (mode 0)
    double *best_loss;
    float *best;
    float *loss_out;               // [epochs] (nullable)
    int epoch;
    float *pred;                   // mode 2
    int *err;
};

// make this thread's generic-proxy global writes visible to later bulk (async
// proxy) reads of them, and order its async-proxy reads before later writes
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Grid barrier of generation gen: bar[0] counts arrivals over the launch (one per
// CTA and barrier; zero at launch), so generation gen is complete once it reaches
// gen * nblocks. After a block barrier, thread 0 of every CTA fences and arrives
// with one atomic (the release: fence, then the relaxed increment); the others of
// the generation poll the counter itself with relaxed loads and fence once they see
// it complete (the acquire). There is no second word for the last arrival to
// publish, so a barrier takes one round trip through L2 fewer. Bounded: a wait that gives up
// (or sees the status word set) sets the status word and returns false; all
// threads of the CTA get the same answer. Every thread's global writes before the
// barrier are visible to every thread of the grid after it.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, unsigned &gen, int *err,
                                             uint32_t max_polls)
{
    __syncthreads();
    gen += 1u;
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned target = gen * nblocks;
        const unsigned t = atomicAdd(bar, 1u);
        if (t + 1u != target) {
            uint32_t it = 0;
            for (;;) {
                unsigned v;
                asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
                if ((int)(v - target) >= 0) break;
                if (++it > max_polls || *(volatile int *)err) {
                    ok = 0;
                    atomicExch(err, 3);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

template <class L>
struct WNetT {
    unsigned char *smem;
    uint32_t tmem = 0;
    uint64_t *mbar, *sbar;
    uint32_t phase = 0, sphase = 0;
    bool pending = false;
    int tid, warp, lane, row, half;
    float *vec, *stage;
    const float *mean, *istd;

    __device__ WNetT(unsigned char *s, uint64_t *mbars) : smem(s)
    {
        tid = threadIdx.x;
        warp = tid >> 5;
        lane = tid & 31;
        row = tid & 127;
        half = tid >> 7;
        mbar = mbars;
        sbar = mbars + 1;
        vec = reinterpret_cast<float *>(smem + L::sVec);
        stage = reinterpret_cast<float *>(smem + L::sStage);
        mean = reinterpret_cast<const float *>(smem + L::sStats);
        istd = mean + kIn;
    }

    __device__ uint32_t saddr(int off) const { return umma::smem_u32(smem + off); }
    __device__ uint32_t taddr(uint32_t col) const { return tmem + ((uint32_t)((warp & 3) * 32) << 16) + col; }

    // one tensor-core step of the CTA: operands written -> issue (thread 0) ->
    // completion; side() runs in every thread after the barrier while the tensor
    // core works
    template <class Issue, class Side>
    __device__ bool mma(Issue issue, bool pre_ok, Side side)
    {
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            issue();
            umma::commit(mbar);
        }
        side();
        const bool done = umma::mbar_wait(mbar, phase, kMbarPolls);
        phase ^= 1u;
        umma::fence_after_sync();
        return __syncthreads_and(done && pre_ok) != 0;
    }
    template <class Issue>
    __device__ bool mma(Issue issue)
    {
        return mma(issue, true, [] {});
    }

    // D = A B^T: A = K columns of a row buffer (width w, from column c0, K-major),
    // B = a K-major image [N][K]
    __device__ void gemm_rows(uint32_t d, int a_off, uint32_t w, int c0, int b_off, int K, int N) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, (uint32_t)N);
        const uint32_t a0 = saddr(a_off) + (uint32_t)(c0 / 8) * 128u, b0 = saddr(b_off);
        const uint32_t asbo = (w / 8u) * 128u, bsbo = (uint32_t)(K / 8) * 128u;
        for (int kk = 0; kk < K / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(a0 + kk * 256u, 128u, asbo), umma::smem_desc(b0 + kk * 256u, 128u, bsbo),
                           id, kk > 0 ? 1u : 0u);
    }

    // D = dH2 W2: A = the dH2 columns of A (K = U), B = the W2 image read MN-major
    __device__ void gemm_w2t(uint32_t d) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, L::U) | umma::kMnMajorB;
        const uint32_t a0 = saddr(L::sA), b0 = saddr(L::sW2), lbo = (L::U / 8) * 128u;
        const uint32_t asbo = (L::wA / 8u) * 128u;
        for (int kk = 0; kk < L::U / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(a0 + kk * 256u, 128u, asbo),
                           umma::smem_desc(b0 + kk * 2u * lbo, lbo, 128u), id, kk > 0 ? 1u : 0u);
    }

    // D (+)= X^T Y over the tile's 128 rows: X = 128 columns of a row buffer from
    // column xc (width xw), Y = N columns of a row buffer from column yc (width yw),
    // both read MN-major
    __device__ void gemm_paths(uint32_t d, int x_off, uint32_t xw, int xc, int y_off, uint32_t yw, int yc, int N,
                               bool acc) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, (uint32_t)N) | umma::kMnMajorA | umma::kMnMajorB;
        const uint32_t x0 = saddr(x_off) + (uint32_t)(xc / 8) * 128u, y0 = saddr(y_off) + (uint32_t)(yc / 8) * 128u;
        const uint32_t xl = (xw / 8u) * 128u, yl = (yw / 8u) * 128u;
        for (int kk = 0; kk < kRows / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(x0 + kk * 2u * xl, xl, 128u), umma::smem_desc(y0 + kk * 2u * yl, yl, 128u),
                           id, (acc || kk > 0) ? 1u : 0u);
    }

    // ---- inputs ----
    // request the tile of paths [path0, path0 + 128): F feature rows (one TMA box)
    // and the target row; called by every thread once all are done reading the
    // staging area
    __device__ void prefetch(const CUtensorMap *tm, const float *targ, int F, uint32_t path0)
    {
        if (tid == 32) {
            umma::mbar_arrive_expect_tx(sbar, (uint32_t)(F + 1) * kRows * 4u);
            umma::tma_load_2d(umma::smem_u32(stage), tm, (int32_t)path0, 0, sbar);
            umma::bulk_g2s(umma::smem_u32(stage + kIn * kRows), targ + path0, kRows * 4u, sbar);
        }
        pending = true;
    }

    // wait for the staged tile; this thread's 16 standardised inputs into the X
    // columns of B; y receives the target
    __device__ bool stage_x(float &y)
    {
        const bool ok = umma::mbar_wait(sbar, sphase, kMbarPolls);
        sphase ^= 1u;
        pending = false;
        const float4 *mv = reinterpret_cast<const float4 *>(mean), *iv = reinterpret_cast<const float4 *>(istd);
        float x[16];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int f0 = 16 * half + 4 * g;
            const float4 m = mv[f0 / 4], r = iv[f0 / 4];
            x[4 * g + 0] = (stage[(f0 + 0) * kRows + row] - m.x) * r.x;
            x[4 * g + 1] = (stage[(f0 + 1) * kRows + row] - m.y) * r.y;
            x[4 * g + 2] = (stage[(f0 + 2) * kRows + row] - m.z) * r.z;
            x[4 * g + 3] = (stage[(f0 + 3) * kRows + row] - m.w) * r.w;
        }
        unsigned char *b = smem + L::sB;
        *reinterpret_cast<uint4 *>(b + wrow_off(row, L::cX + 16 * half, L::wB)) = pack8(x);
        *reinterpret_cast<uint4 *>(b + wrow_off(row, L::cX + 16 * half + 8, L::wB)) = pack8(x + 8);
        y = stage[kIn * kRows + row];
        return ok;
    }

    // ---- epilogues: thread = (row, half), 64 hidden columns each ----
    // H1 = relu(D + b1) into B; the mask of h1 > 0 in m1
    __device__ void epi1(uint32_t (&m1)[2]) const
    {
        unsigned char *b = smem + L::sB;
        const float4 *b1 = reinterpret_cast<const float4 *>(vec + L::vb1 + 64 * half);
        float v[64];
        umma::tmem_ld64(taddr(L::cD + 64u * half), v);
        m1[0] = m1[1] = 0u;
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float4 c = b1[g];
            v[4 * g + 0] = fmaxf(v[4 * g + 0] + c.x, 0.f);
            v[4 * g + 1] = fmaxf(v[4 * g + 1] + c.y, 0.f);
            v[4 * g + 2] = fmaxf(v[4 * g + 2] + c.z, 0.f);
            v[4 * g + 3] = fmaxf(v[4 * g + 3] + c.w, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 64; ++i) m1[i / 32] |= (v[i] > 0.f ? 1u : 0u) << (i % 32);
#pragma unroll
        for (int g = 0; g < 8; ++g) *reinterpret_cast<uint4 *>(b + wrow_off(row, 64 * half + 8 * g, L::wB)) = pack8(v + 8 * g);
    }

    // h2 = relu(D + b2) of this thread's 64 columns in place; returns their share of
    // w3 . h2 (four partial sums)
    __device__ float layer2(float (&v)[64]) const
    {
        const float4 *b2 = reinterpret_cast<const float4 *>(vec + L::vb2 + 64 * half),
                     *w3 = reinterpret_cast<const float4 *>(vec + L::vw3 + 64 * half);
        umma::tmem_ld64(taddr(L::cD + 64u * half), v);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float4 c = b2[g], w = w3[g];
            v[4 * g + 0] = fmaxf(v[4 * g + 0] + c.x, 0.f);
            v[4 * g + 1] = fmaxf(v[4 * g + 1] + c.y, 0.f);
            v[4 * g + 2] = fmaxf(v[4 * g + 2] + c.z, 0.f);
            v[4 * g + 3] = fmaxf(v[4 * g + 3] + c.w, 0.f);
            acc[0] = fmaf(v[4 * g + 0], w.x, acc[0]);
            acc[1] = fmaf(v[4 * g + 1], w.y, acc[1]);
            acc[2] = fmaf(v[4 * g + 2], w.z, acc[2]);
            acc[3] = fmaf(v[4 * g + 3], w.w, acc[3]);
        }
        return (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }

    // zeta = w3 . h2 + b3 of this thread's row: the two halves' shares added in order
    __device__ float zeta(float share) const
    {
        float *so = reinterpret_cast<float *>(smem + L::sOut);
        so[half * kRows + row] = share;
        __syncthreads();
        const float z = (so[row] + so[kRows + row]) + vec[L::vb3];
        __syncthreads();
        return z;
    }

    // output, loss derivative and the output-layer backward of this thread's row:
    // dH2 = dout w3 (h2 > 0) into A; column sums of h2 dout over the warp's rows
    // (dw3) and, in the first warpgroup, of dout (db3) and dpred (dmu)
    __device__ void out_back2(int pos, float y, float inv_batch, float *gsl) const
    {
        unsigned char *a = smem + L::sA;
        const float4 *w3 = reinterpret_cast<const float4 *>(vec + L::vw3 + 64 * half);
        float v[64];
        const float out = zeta(layer2(v));
        const float pred = (pos ? fmaxf(out, 0.f) : out) + vec[L::vmu];
        const float dpred = 2.f * (pred - y) * inv_batch;
        const float dout = pos ? (out > 0.f ? dpred : 0.f) : dpred;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float4 w0 = w3[2 * g], w1 = w3[2 * g + 1];
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float d[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) d[i] = v[8 * g + i] > 0.f ? dout * wv[i] : 0.f;
            *reinterpret_cast<uint4 *>(a + wrow_off(row, 64 * half + 8 * g, L::wA)) = pack8(d);
        }
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] *= dout;
        const float2 cs = column_sums64(v, lane);
        gsl[2 * lane] += cs.x;
        gsl[2 * lane + 1] += cs.y;
        if (half == 0) {
            const float s3 = warp_sum(dout), smu = warp_sum(dpred);
            if (lane == 0) {
                gsl[64] += s3;
                gsl[65] += smu;
            }
        }
    }

    // dH1 = D (h1 > 0) into A
    __device__ void back1(const uint32_t (&m1)[2]) const
    {
        unsigned char *a = smem + L::sA;
        float v[64];
        umma::tmem_ld64(taddr(L::cD + 64u * half), v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = ((m1[i / 32] >> (i % 32)) & 1u) ? v[i] : 0.f;
#pragma unroll
        for (int g = 0; g < 8; ++g)
            *reinterpret_cast<uint4 *>(a + wrow_off(row, L::U + 64 * half + 8 * g, L::wA)) = pack8(v + 8 * g);
    }

    // first two layers of the staged tile; D holds the second-layer pre-activation
    template <class Side>
    __device__ bool forward12(uint32_t (&m1)[2], bool in_ok, Side side)
    {
        if (!mma([&] { gemm_rows(L::cD, L::sB, L::wB, L::cX, L::sW1, kIn, L::U); }, in_ok, side)) return false;
        epi1(m1);
        return mma([&] { gemm_rows(L::cD, L::sB, L::wB, 0, L::sW2, L::U, L::U); });
    }

    // constant columns of B: ones after H1 (first warpgroup) and after X (second)
    __device__ void init_constants()
    {
        const uint4 one = make_uint4((uint32_t)bf16_bits(1.f), 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
        unsigned char *b = smem + L::sB;
        const int c = half ? L::cOne2 : L::cOne1;
        *reinterpret_cast<uint4 *>(b + wrow_off(row, c, L::wB)) = one;
        *reinterpret_cast<uint4 *>(b + wrow_off(row, c + 8, L::wB)) = zero;
    }
};
using WNet = WNetT<WL>;

// common start: TMEM, mbarriers, standardisation, zero staging rows >= F, the
// constant columns of B, optionally a zeroed A
template <class L>
__device__ void wide_setup(WNetT<L> &n, uint32_t *s_tmem, uint64_t *s_mbar, const float *stats, int F, bool zero_a)
{
    if (n.warp == 0) {
        umma::tmem_alloc(s_tmem, L::tmem_cols);
        umma::tmem_relinquish();
    }
    if (n.tid == 0) {
        umma::mbar_init(&s_mbar[0], 1);
        umma::mbar_init(&s_mbar[1], 1);
        umma::fence_mbar_init();
    }
    float *st = reinterpret_cast<float *>(n.smem + L::sStats);
    if (n.tid < 2 * kIn) st[n.tid] = __ldg(stats + n.tid);
    for (int i = n.tid; i < (kIn + 1) * kRows; i += kWThreads) {
        const int f = i / kRows;
        if (f >= F && f < kIn) n.stage[i] = 0.f;
    }
    float *gsl = reinterpret_cast<float *>(n.smem + L::sGsl);
    for (int i = n.tid; i < 8 * 66; i += kWThreads) gsl[i] = 0.f;
    if constexpr (L::sA >= 0) if (zero_a) {
        uint4 *a = reinterpret_cast<uint4 *>(n.smem + L::sA);
        for (int i = n.tid; i < kRows * L::wA * 2 / 16; i += kWThreads) a[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    n.init_constants();
}

// images and FP32 vectors of the parameters theta (global, row order)
template <class L>
__device__ void wide_load_params(WNetT<L> &n, const float *theta)
{
    for (int i = n.tid; i < L::U * (kIn / 8); i += kWThreads) {   // W1: row o, 8 inputs from k
        const int o = i / (kIn / 8), k = (i % (kIn / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(theta + L::oW1 + o * kIn + k + j);
        *reinterpret_cast<uint4 *>(n.smem + L::sW1 + umma::kmajor_offset(o, k, kIn)) = pack8(v);
    }
    for (int i = n.tid; i < L::U * (L::U / 8); i += kWThreads) {  // W2: row o, 8 inputs from k
        const int o = i / (L::U / 8), k = (i % (L::U / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(theta + L::oW2 + o * L::U + k + j);
        *reinterpret_cast<uint4 *>(n.smem + L::sW2 + umma::kmajor_offset(o, k, L::U)) = pack8(v);
    }
    for (int i = n.tid; i < L::U; i += kWThreads) {
        n.vec[L::vb1 + i] = __ldg(theta + L::ob1 + i);
        n.vec[L::vb2 + i] = __ldg(theta + L::ob2 + i);
        n.vec[L::vw3 + i] = __ldg(theta + L::ow3 + i);
    }
    if (n.tid == 0) {
        n.vec[L::vb3] = __ldg(theta + L::ob3);
        n.vec[L::vmu] = __ldg(theta + L::omu);
    }
}

template <class L>
__device__ void wide_finish_setup(WNetT<L> &n, uint32_t *s_tmem)
{
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    n.tmem = *s_tmem;
}

template <class L>
__device__ void wide_teardown(WNetT<L> &n)
{
    if (n.pending) (void)umma::mbar_wait(n.sbar, n.sphase, kMbarPolls);
    umma::fence_before_sync();
    __syncthreads();
    if (n.warp == 0) umma::tmem_dealloc(n.tmem, L::tmem_cols);
}

// One epoch (or its first n_steps batches) of Adam on a cooperative grid. Batch b
// covers paths [b P, (b + 1) P), P = tiles_per_batch * 128; in each step the
// grid's CTAs take the batch's tiles round-robin.
__global__ void __launch_bounds__(kWThreads, 1) wide_train_kernel(WTrainArgs a, const __grid_constant__ CUtensorMap tm)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[3];   // tensor core, input staging, parameter reload
    WNet n(smem, s_mbar);
    const int G = (int)gridDim.x, cta = (int)blockIdx.x;
    // owned slice [lo, hi) of the padded parameter vector (multiples of 4 entries)
    const int S = ((WL::NPpad + 4 * G - 1) / (4 * G)) * 4;
    const int lo = min(WL::NPpad, cta * S), hi = min(WL::NPpad, lo + S);

    wide_setup(n, &s_tmem, s_mbar, a.stats, a.F, false);
    if (n.tid == 0) {
        umma::mbar_init(&s_mbar[2], 1);
        umma::fence_mbar_init();
    }
    wide_load_params(n, a.init);
    for (int q = lo + n.tid; q < hi; q += kWThreads) {
        a.gq[q] = q < WL::NP ? __ldg(a.init + WL::p_of(q)) : 0.f;
        if (a.step0 == 0) a.adam_m[q] = a.adam_v[q] = 0.f;
    }
    if (a.step0 == 0 && cta == 0) {   // start of a date: the starting parameters are the best so far
        for (int p = n.tid; p < WL::NP; p += kWThreads) a.best[p] = __ldg(a.init + p);
        if (n.tid == 0) *a.best_loss = 1e300;
    }
    wide_finish_setup(n, &s_tmem);

    const uint32_t per_batch = (uint32_t)a.tiles_per_batch * kRows;
    const float inv_batch = 1.f / (float)per_batch;
    const int my_rounds = cta < a.tiles_per_batch ? (a.tiles_per_batch - 1 - cta) / G + 1 : 0;
    auto path_of = [&](int st, int rd) { return (uint32_t)st * per_batch + (uint32_t)(rd * G + cta) * kRows; };
    float *gsl = reinterpret_cast<float *>(smem + WL::sGsl);
    float *my_gsl = gsl + n.warp * 66;
    float4 *red = reinterpret_cast<float4 *>(smem + WL::sRed);
    uint64_t *rbar = &s_mbar[2];
    uint32_t rphase = 0;
    bool rpending = false;
    unsigned gen = 0;
    bool ok = true;

    if (my_rounds > 0) n.prefetch(&tm, a.targ, a.F, path_of(0, 0));
    for (int st = 0; st < a.n_steps; ++st) {
        for (int rd = 0; rd < my_rounds && ok; ++rd) {
            const bool last = rd + 1 == my_rounds;
            const bool has_next = !last || st + 1 < a.n_steps;
            const uint32_t next = last ? path_of(st + 1, 0) : path_of(st, rd + 1);
            float y;
            const bool in_ok = n.stage_x(y);
            uint32_t m1[2];
            ok = n.forward12(m1, in_ok, [&] {
                if (has_next) n.prefetch(&tm, a.targ, a.F, next);
            });
            if (ok) {
                n.out_back2(a.pos, y, inv_batch, my_gsl);
                ok = n.mma([&] { n.gemm_w2t(WL::cD); });
            }
            if (ok) {
                n.back1(m1);
                const bool acc = rd > 0;
                ok = n.mma([&] {
                    n.gemm_paths(WL::cW2, WL::sA, WL::wA, 0, WL::sB, WL::wB, 0, WL::U + 16, acc);
                    n.gemm_paths(WL::cW1, WL::sA, WL::wA, WL::U, WL::sB, WL::wB, WL::cX, kIn + 16, acc);
                });
            }
            if (!ok && n.tid == 0) atomicExch(a.err, 2);
        }
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // this CTA's partial (zero when it had no tile) to global memory, q order
        float *P = a.gpart + (size_t)cta * WL::NPpad;
        {
            const uint32_t lanes = (uint32_t)((n.warp & 3) * 32) << 16;
            const int r = (n.warp & 3) * 32 + n.lane;
            const bool have = my_rounds > 0;
            // DW2 | db2 (9 chunks of 16 columns): chunks [0, 5) in the first half, [5, 9) in
            // the second; DW1 | db1 (3 chunks): [0, 1) and [1, 3). Every load is issued
            // before the one wait (the unused chunks read allocated, unused columns).
            const int k0 = n.half ? 5 : 0, k1 = n.half ? 9 : 5, j0 = n.half ? 1 : 0, j1 = n.half ? 3 : 1;
            float v2[5][16], v1[2][16];
#pragma unroll
            for (int k = 0; k < 5; ++k) umma::tmem_ld16(n.tmem + lanes + WL::cW2 + 16u * (uint32_t)(k0 + k), v2[k]);
#pragma unroll
            for (int k = 0; k < 2; ++k) umma::tmem_ld16(n.tmem + lanes + WL::cW1 + 16u * (uint32_t)(j0 + k), v1[k]);
            umma::tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 5; ++k)
#pragma unroll
                for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(v2[k][i]));
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(v1[k][i]));
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k0 + k < k1) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * (k0 + k) + i;
                        const float g = have ? v2[k][i] : 0.f;
                        if (c < WL::U) P[WL::oW2 + c * WL::U + r] = g;
                        else if (c == WL::U) P[WL::ob2 + r] = g;
                    }
                }
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (j0 + k < j1) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * (j0 + k) + i;
                        const float g = have ? v1[k][i] : 0.f;
                        if (c < kIn) P[WL::oW1 + c * WL::U + r] = g;
                        else if (c == kIn) P[WL::ob1 + r] = g;
                    }
                }
            if (n.tid < WL::U + 2) {   // w3 from the warps of the column's half; b3, mu from the first half
                const int j = n.tid;
                const int h = j < WL::U ? j >> 6 : 0, c = j < WL::U ? (j & 63) : j - WL::U + 64;
                float s = 0.f;
                for (int w = 4 * h; w < 4 * h + 4; ++w) s += gsl[w * 66 + c];
                P[j < WL::U ? WL::ow3 + j : (j == WL::U ? WL::ob3 : WL::omu)] = s;
            }
            __syncthreads();
            for (int i = n.tid; i < 8 * 66; i += kWThreads) gsl[i] = 0.f;
        }
        fence_proxy_async_global();   // the last reload's bulk reads come before this step's writes
        if (!grid_barrier(a.flags, (unsigned)G, gen, a.err, a.grid_polls)) ok = false;

        // the owned slice: partials summed over the grid (nsub fixed interleaved
        // ranges of CTAs per group of four parameters, added in range order), Adam,
        // new FP32 values and their BF16 images
        {
            const int step = a.step0 + st + 1;
            const float inv_bc1 = 1.f / (1.f - powf(a.beta1, (float)step)),
                        inv_bc2 = 1.f / (1.f - powf(a.beta2, (float)step));
            const int NG = (hi - lo) / 4;
            const int nsub = NG >= kWThreads ? 1 : (NG > 0 ? kWThreads / NG : 1);
            const int Pg = kWThreads / nsub;
            for (int g0 = 0; g0 < NG; g0 += Pg) {
                const int gi = g0 + n.tid % Pg, j = n.tid / Pg;
                const bool upd = j == 0 && gi < NG;   // this thread updates the group
                float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f), v4 = m4, t4 = m4;
                if (upd) {   // Adam state of the group, requested together with the partials
                    m4 = *reinterpret_cast<const float4 *>(a.adam_m + lo + 4 * gi);
                    v4 = *reinterpret_cast<const float4 *>(a.adam_v + lo + 4 * gi);
                    t4 = *reinterpret_cast<const float4 *>(a.gq + lo + 4 * gi);
                }
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gi < NG && j < nsub)
                    for (int c0 = j; c0 < G; c0 += 32 * nsub) {   // 32 loads in flight, added in CTA order
                        float4 v[32];
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const int c = c0 + u * nsub;
                            v[u] = c < G ? __ldcg(reinterpret_cast<const float4 *>(a.gpart + (size_t)c * WL::NPpad + lo + 4 * gi))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            acc.x += v[u].x;
                            acc.y += v[u].y;
                            acc.z += v[u].z;
                            acc.w += v[u].w;
                        }
                    }
                red[n.tid] = acc;
                __syncthreads();
                if (upd) {
                    float4 g = red[n.tid];
                    for (int jj = 1; jj < nsub; ++jj) {
                        const float4 v = red[jj * Pg + n.tid];
                        g.x += v.x;
                        g.y += v.y;
                        g.z += v.z;
                        g.w += v.w;
                    }
                    const float gv[4] = {g.x, g.y, g.z, g.w};
                    float mv[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w},
                          tv[4] = {t4.x, t4.y, t4.z, t4.w};
                    for (int e = 0; e < 4; ++e) {
                        const int q = lo + 4 * gi + e;
                        if (step == 1 && a.grad_out && q < WL::NP) a.grad_out[WL::p_of(q)] = gv[e];
                        float t = 0.f;   // padding stays zero
                        if (q < WL::NP && !(q < WL::ob1 && q / WL::U >= a.F)) {
                            mv[e] = a.beta1 * mv[e] + (1.f - a.beta1) * gv[e];
                            vv[e] = a.beta2 * vv[e] + (1.f - a.beta2) * gv[e] * gv[e];
                            t = tv[e] - adam_delta(mv[e], vv[e], inv_bc1, inv_bc2, a.lr, a.eps);
                        }
                        tv[e] = t;
                        if (q < WL::ob1) {
                            const int o = q % WL::U, f = q / WL::U;
                            a.gimg[umma::kmajor_offset(o, f, kIn) / 2] = bf16_bits(t);
                        } else if (q >= WL::oW2 && q < WL::ob2) {
                            const int o = (q - WL::oW2) % WL::U, k = (q - WL::oW2) / WL::U;
                            a.gimg[(WL::U * kIn * 2 + umma::kmajor_offset(o, k, WL::U)) / 2] = bf16_bits(t);
                        }
                    }
                    *reinterpret_cast<float4 *>(a.adam_m + lo + 4 * gi) = make_float4(mv[0], mv[1], mv[2], mv[3]);
                    *reinterpret_cast<float4 *>(a.adam_v + lo + 4 * gi) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                    *reinterpret_cast<float4 *>(a.gq + lo + 4 * gi) = make_float4(tv[0], tv[1], tv[2], tv[3]);
                }
                __syncthreads();
            }
        }
        fence_proxy_async_global();   // the new slice is read by bulk copies
        if (!grid_barrier(a.flags, (unsigned)G, gen, a.err, a.grid_polls)) ok = false;

        // every CTA: the new images (W1 | W2, stored in the shared-memory layout) and the
        // FP32 vectors b1 and b2 | w3 | b3 | mu (one padding word after them) by three
        // bulk copies completing on the reload barrier (none is issued while an earlier
        // one may still be in flight: after a wait that gave up the launch is failing)
        if (!rpending) {
            if (n.tid == 0) {
                fence_proxy_async_global();
                constexpr uint32_t img_bytes = WL::img_elems * 2u, b1_bytes = WL::U * 4u,
                                   rest_bytes = (2 * WL::U + 4) * 4u;
                static_assert(WL::sW2 == WL::sW1 + WL::U * kIn * 2 && img_bytes % 16 == 0, "images are one copy");
                static_assert((WL::ob1 * 4) % 16 == 0 && (WL::ob2 * 4) % 16 == 0 && rest_bytes % 16 == 0,
                              "bulk copy alignment");
                static_assert(WL::vb2 + 2 * WL::U + 4 <= 512 && WL::ob2 + 2 * WL::U + 4 <= WL::NPpad,
                              "vector copy bounds");
                static_assert(WL::vw3 == WL::vb2 + (WL::ow3 - WL::ob2) && WL::vb3 == WL::vb2 + (WL::ob3 - WL::ob2) &&
                                  WL::vmu == WL::vb2 + (WL::omu - WL::ob2),
                              "b2 | w3 | b3 | mu keep their order");
                umma::mbar_arrive_expect_tx(rbar, img_bytes + b1_bytes + rest_bytes);
                umma::bulk_g2s(n.saddr(WL::sW1), a.gimg, img_bytes, rbar);
                umma::bulk_g2s(n.saddr(WL::sVec + WL::vb1 * 4), a.gq + WL::ob1, b1_bytes, rbar);
                umma::bulk_g2s(n.saddr(WL::sVec + WL::vb2 * 4), a.gq + WL::ob2, rest_bytes, rbar);
            }
            const bool got = umma::mbar_wait(rbar, rphase, kMbarPolls);
            rphase ^= 1u;
            rpending = __syncthreads_and(got) == 0;
            if (rpending) {
                ok = false;
                if (n.tid == 0) atomicExch(a.err, 2);
            }
        }
    }
    for (int q = lo + n.tid; q < hi; q += kWThreads)
        if (q < WL::NP) {
            const float t = a.gq[q];
            a.params[WL::p_of(q)] = t;
            if (a.snap) a.snap[WL::p_of(q)] = t;
        }
    if (rpending) (void)umma::mbar_wait(rbar, rphase ^ 1u, kMbarPolls);   // no copy outlives the CTA
    wide_teardown(n);
}

// Full-sample passes with fixed parameters, output ReLU on: the loss (mode 0), the
// refit's Gram matrix of Z = [h2 | 1 | y - mu] (mode 1), the predictions (mode 2).
template <class L, int MinBlocks>
__global__ void __launch_bounds__(kWThreads, MinBlocks) wide_sweep_kernel(WSweepArgs a,
                                                                         const __grid_constant__ CUtensorMap tm)
{
    constexpr int Z = L::Z;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ double s_red[8][3];
    __shared__ int s_flag[2];
    WNetT<L> n(smem, s_mbar);
    wide_setup(n, &s_tmem, s_mbar, a.stats, a.F, a.mode == 1);
    wide_load_params(n, a.theta);
    wide_finish_setup(n, &s_tmem);

    const uint32_t tiles = a.M / kRows, stride = gridDim.x;
    uint32_t t = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    bool ok = true, first = true;
    if (t < tiles) n.prefetch(&tm, a.targ, a.F, t * kRows);
    for (; t < tiles && ok; t += stride) {
        const uint32_t nt = t + stride;
        float y;
        const bool in_ok = n.stage_x(y);
        uint32_t m1[2];
        ok = n.forward12(m1, in_ok, [&] {
            if (nt < tiles) n.prefetch(&tm, a.targ, a.F, nt * kRows);
        });
        if (!ok) break;
        float v[64];
        const float share = n.layer2(v);
        if (a.mode != 1) {
            const float pred = fmaxf(n.zeta(share), 0.f) + n.vec[L::vmu];
            if (n.half == 0) {
                if (a.mode == 2) {
                    if (a.pred) a.pred[t * kRows + n.row] = pred;
                } else {
                    acc[0] += (double)((pred - y) * (pred - y));
                }
            }
        } else if constexpr (L::kGram) {
            // row of Z into A: [h2 | 1 | y - mu | 0 ...]; the corner sums (1, y - mu,
            // (y - mu)^2 with y - mu rounded as the tensor core sees it) in FP64
            unsigned char *ar = smem + L::sA;
#pragma unroll
            for (int g = 0; g < 8; ++g)
                *reinterpret_cast<uint4 *>(ar + wrow_off(n.row, 64 * n.half + 8 * g, L::wA)) = pack8(v + 8 * g);
            if (n.half == 1) {
                const float d = y - n.vec[L::vmu];
                *reinterpret_cast<uint4 *>(ar + wrow_off(n.row, L::U, L::wA)) = make_uint4(pack2(1.f, d), 0u, 0u, 0u);
                const double db = (double)__bfloat162float(__float2bfloat16_rn(d));
                acc[0] += 1.0;
                acc[1] += db;
                acc[2] += db * db;
            }
            // G (+)= Z^T Z: M = the 128 h2 columns, N = the first 144 columns of the rows
            ok = n.mma([&] { n.gemm_paths(L::cW2, L::sA, L::wA, 0, L::sA, L::wA, 0, L::U + 16, !first); });
        }
        if (!ok && n.tid == 0) atomicExch(a.err, 2);
        first = false;
    }
    if (!ok && n.tid == 0) atomicExch(a.err, 2);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    // block sums of acc[0..2]
    for (int k = 0; k < 3; ++k) {
        double s = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (n.lane == 0) s_red[n.warp][k] = s;
    }
    __syncthreads();
    if (a.mode == 0) {
        if (n.tid == 0) {
            double b = 0.0;
            for (int w = 0; w < 8; ++w) b += s_red[w][0];
            a.part[blockIdx.x] = b;
            __threadfence();
            s_flag[0] = atomicAdd(a.count, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_flag[0]) {   // the last CTA: total loss, best parameters so far
            __threadfence();
            if (n.tid == 0) {
                double tot = 0.0;
                for (uint32_t b = 0; b < gridDim.x; ++b) tot += __ldcg(a.part + b);
                tot /= (double)a.M;
                if (a.loss_out) a.loss_out[a.epoch - 1] = (float)tot;
                s_flag[1] = tot < *a.best_loss;
                if (s_flag[1]) *a.best_loss = tot;
                *a.count = 0u;
            }
            __syncthreads();
            if (s_flag[1])
                for (int p = n.tid; p < L::NP; p += kWThreads) a.best[p] = __ldg(a.theta + p);
        }
    } else if constexpr (L::kGram) {   // mode 1: this CTA's Gram as FP64, [Z][Z]
        double *P = a.part + (size_t)blockIdx.x * Z * Z;
        const bool have = blockIdx.x < tiles;
        const uint32_t lanes = (uint32_t)((n.warp & 3) * 32) << 16;
        const int r = (n.warp & 3) * 32 + n.lane;
        const int k0 = n.half ? 5 : 0, k1 = n.half ? 9 : 5;
        for (int k = k0; k < k1; ++k) {
            float v[16];
            umma::tmem_ld16(n.tmem + lanes + L::cW2 + 16u * k, v);
            umma::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = 16 * k + i;
                if (c < Z) {
                    const double g = have ? (double)v[i] : 0.0;
                    P[r * Z + c] = g;
                    if (c >= L::U) P[c * Z + r] = g;   // rows U, U + 1 by symmetry
                }
            }
        }
        if (n.tid == 0) {
            double c0 = 0.0, c1 = 0.0, c2 = 0.0;
            for (int w = 4; w < 8; ++w) {
                c0 += s_red[w][0];
                c1 += s_red[w][1];
                c2 += s_red[w][2];
            }
            P[L::U * Z + L::U] = c0;
            P[L::U * Z + L::U + 1] = P[(L::U + 1) * Z + L::U] = c1;
            P[(L::U + 1) * Z + L::U + 1] = c2;
        }
    }
    wide_teardown(n);
}

// Loss (mode 0) and prediction (mode 2) passes: the forward pass of the trainer's
// tiles (both warpgroups on one tile, 64 hidden columns each) in a two-stage
// pipeline over the CTA's tiles k = 0, 1, ...:
//   stage tile k into B[k & 1] and issue D[k & 1] = X W1^T;
//   wait for tile k - 1's second GEMM, evaluate its output layer and loss;
//   wait for tile k's first GEMM, H1 = relu(D + b1) into B[k & 1], issue
//   D[k & 1] = H1 W2^T.
// Every row's arithmetic is the trainer's forward pass, and a CTA adds its rows'
// losses in tile order, so the result does not depend on the pipeline.
__global__ void __launch_bounds__(kWThreads, 1) wide_fwd_kernel(WSweepArgs a, const __grid_constant__ CUtensorMap tm)
{
    using L = WLP;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[3];   // first GEMM, (unused staging), second GEMM
    __shared__ __align__(8) uint64_t s_sbar[L::kStages];   // staging buffer s complete
    __shared__ double s_red[8];
    __shared__ int s_flag[2];
    WNetT<L> n(smem, s_mbar);
    wide_setup(n, &s_tmem, s_mbar, a.stats, a.F, false);
    if (n.tid == 0) {
        umma::mbar_init(&s_mbar[2], 1);
        for (int q = 0; q < L::kStages; ++q) umma::mbar_init(&s_sbar[q], 1);
        umma::fence_mbar_init();
    }
    // rows f >= F of every staging buffer stay zero (the copies fill rows < F)
    for (int i = n.tid; i < L::kStages * (kIn + 1) * kRows; i += kWThreads) {
        const int f = (i / kRows) % (kIn + 1);
        if (f >= a.F && f < kIn) n.stage[i] = 0.f;
    }
    wide_load_params(n, a.theta);
    wide_finish_setup(n, &s_tmem);
    uint64_t *bar1 = &s_mbar[0], *bar2 = &s_mbar[2];
    uint32_t ph1 = 0, ph2 = 0;

    // tensor-core issue by thread 0 once every thread's operands are written
    auto issue = [&](uint64_t *bar, auto f) {
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (n.tid == 0) {
            f();
            umma::commit(bar);
        }
    };
    auto wait = [&](uint64_t *bar, uint32_t &ph) {
        const bool d = umma::mbar_wait(bar, ph, kMbarPolls);
        ph ^= 1u;
        umma::fence_after_sync();
        return d;
    };
    // the inputs of the CTA's tile j (paths path0 ...) into staging buffer j % kStages
    // (one thread issues; called once no thread reads that buffer any more)
    auto request = [&](uint32_t j, uint32_t path0) {
        if (n.tid == 32) {
            uint64_t *sb = &s_sbar[j % L::kStages];
            const uint32_t dst = n.saddr(L::sStage + (int)(j % L::kStages) * L::stage_bytes);
            umma::mbar_arrive_expect_tx(sb, (uint32_t)(a.F + 1) * kRows * 4u);
            umma::tma_load_2d(dst, &tm, (int32_t)path0, 0, sb);
            umma::bulk_g2s(dst + kIn * kRows * 4u, a.targ + path0, kRows * 4u, sb);
        }
    };
    // wait for tile j's inputs; this thread's 16 standardised inputs into the X columns
    // of B[b]; y receives the target
    auto stage_into = [&](uint32_t j, int b, float &y) {
        const bool got = umma::mbar_wait(&s_sbar[j % L::kStages], (j / L::kStages) & 1u, kMbarPolls);
        const float *stg = reinterpret_cast<const float *>(smem + L::sStage + (int)(j % L::kStages) * L::stage_bytes);
        const float4 *mv = reinterpret_cast<const float4 *>(n.mean), *iv = reinterpret_cast<const float4 *>(n.istd);
        float x[16];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int f0 = 16 * n.half + 4 * g;
            const float4 m = mv[f0 / 4], r = iv[f0 / 4];
            x[4 * g + 0] = (stg[(f0 + 0) * kRows + n.row] - m.x) * r.x;
            x[4 * g + 1] = (stg[(f0 + 1) * kRows + n.row] - m.y) * r.y;
            x[4 * g + 2] = (stg[(f0 + 2) * kRows + n.row] - m.z) * r.z;
            x[4 * g + 3] = (stg[(f0 + 3) * kRows + n.row] - m.w) * r.w;
        }
        unsigned char *bp = smem + (b ? L::sB1 : L::sB);
        *reinterpret_cast<uint4 *>(bp + wrow_off(n.row, L::cX + 16 * n.half, L::wB)) = pack8(x);
        *reinterpret_cast<uint4 *>(bp + wrow_off(n.row, L::cX + 16 * n.half + 8, L::wB)) = pack8(x + 8);
        y = stg[kIn * kRows + n.row];
        return got;
    };
    // H1 = relu(D[b] + b1) of this thread's 64 columns into B[b]
    auto epi1_into = [&](int b) {
        unsigned char *bp = smem + (b ? L::sB1 : L::sB);
        const float4 *b1 = reinterpret_cast<const float4 *>(n.vec + L::vb1 + 64 * n.half);
        float v[64];
        umma::tmem_ld64(n.taddr(128u * (uint32_t)b + 64u * (uint32_t)n.half), v);
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float4 c = b1[g];
            v[4 * g + 0] = fmaxf(v[4 * g + 0] + c.x, 0.f);
            v[4 * g + 1] = fmaxf(v[4 * g + 1] + c.y, 0.f);
            v[4 * g + 2] = fmaxf(v[4 * g + 2] + c.z, 0.f);
            v[4 * g + 3] = fmaxf(v[4 * g + 3] + c.w, 0.f);
        }
#pragma unroll
        for (int g = 0; g < 8; ++g)
            *reinterpret_cast<uint4 *>(bp + wrow_off(n.row, 64 * n.half + 8 * g, L::wB)) = pack8(v + 8 * g);
    };
    // this thread's share of w3 . relu(D[b] + b2) (four partial sums, the order of layer2)
    auto share_of = [&](int b) {
        const float4 *b2 = reinterpret_cast<const float4 *>(n.vec + L::vb2 + 64 * n.half),
                     *w3 = reinterpret_cast<const float4 *>(n.vec + L::vw3 + 64 * n.half);
        float v[64];
        umma::tmem_ld64(n.taddr(128u * (uint32_t)b + 64u * (uint32_t)n.half), v);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float4 c = b2[g], w = w3[g];
            v[4 * g + 0] = fmaxf(v[4 * g + 0] + c.x, 0.f);
            v[4 * g + 1] = fmaxf(v[4 * g + 1] + c.y, 0.f);
            v[4 * g + 2] = fmaxf(v[4 * g + 2] + c.z, 0.f);
            v[4 * g + 3] = fmaxf(v[4 * g + 3] + c.w, 0.f);
            acc[0] = fmaf(v[4 * g + 0], w.x, acc[0]);
            acc[1] = fmaf(v[4 * g + 1], w.y, acc[1]);
            acc[2] = fmaf(v[4 * g + 2], w.z, acc[2]);
            acc[3] = fmaf(v[4 * g + 3], w.w, acc[3]);
        }
        return (acc[0] + acc[1]) + (acc[2] + acc[3]);
    };

    const uint32_t tiles = a.M / kRows, stride = gridDim.x;
    const uint32_t K = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / stride + 1 : 0;   // this CTA's tiles
    double acc = 0.0;
    bool ok = true, pend2 = false;   // pend2: a second GEMM issued and not yet waited for
    float y_prev = 0.f, y = 0.f;
    uint32_t requested = 0, consumed = 0;   // tiles whose inputs were requested / read
    for (; requested < K && requested < (uint32_t)L::kStages; ++requested)
        request(requested, (blockIdx.x + requested * stride) * kRows);
    for (uint32_t k = 0; k <= K; ++k) {
        const int b = (int)(k & 1u);
        const uint32_t t = blockIdx.x + k * stride;
        if (k < K) {
            ok = stage_into(k, b, y) && ok;
            ++consumed;
            issue(bar1, [&] { n.gemm_rows(128u * (uint32_t)b, b ? L::sB1 : L::sB, L::wB, L::cX, L::sW1, kIn, L::U); });
            if (requested < K) {   // every thread is past buffer k % kStages: tile k + kStages into it
                request(requested, (blockIdx.x + requested * stride) * kRows);
                ++requested;
            }
        }
        if (k > 0) {   // the output layer of tile k - 1
            ok = wait(bar2, ph2) && ok;
            pend2 = false;
            const float pred = fmaxf(n.zeta(share_of(b ^ 1)), 0.f) + n.vec[L::vmu];
            if (n.half == 0) {
                if (a.mode == 2) {
                    if (a.pred) a.pred[(t - stride) * kRows + n.row] = pred;
                } else {
                    acc += (double)((pred - y_prev) * (pred - y_prev));
                }
            }
        }
        if (k < K) {
            ok = wait(bar1, ph1) && ok;
            epi1_into(b);
            issue(bar2, [&] { n.gemm_rows(128u * (uint32_t)b, b ? L::sB1 : L::sB, L::wB, 0, L::sW2, L::U, L::U); });
            pend2 = true;
        }
        y_prev = y;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
    }
    if (pend2) (void)wait(bar2, ph2);   // a loop left early: no tensor-core work outlives the CTA
    for (uint32_t j = consumed; j < requested; ++j)   // nor any input copy
        (void)umma::mbar_wait(&s_sbar[j % L::kStages], (j / L::kStages) & 1u, kMbarPolls);
    if (!ok && n.tid == 0) atomicExch(a.err, 2);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    if (a.mode == 0) {
        double sred = acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sred += __shfl_xor_sync(0xffffffffu, sred, o);
        if (n.lane == 0) s_red[n.warp] = sred;
        __syncthreads();
        if (n.tid == 0) {
            double bsum = 0.0;
            for (int w = 0; w < 8; ++w) bsum += s_red[w];
            a.part[blockIdx.x] = bsum;
            __threadfence();
            s_flag[0] = atomicAdd(a.count, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_flag[0]) {   // the last CTA: total loss, best parameters so far
            __threadfence();
            if (n.tid == 0) {
                double tot = 0.0;
                for (uint32_t bb = 0; bb < gridDim.x; ++bb) tot += __ldcg(a.part + bb);
                tot /= (double)a.M;
                if (a.loss_out) a.loss_out[a.epoch - 1] = (float)tot;
                s_flag[1] = tot < *a.best_loss;
                if (s_flag[1]) *a.best_loss = tot;
                *a.count = 0u;
            }
            __syncthreads();
            if (s_flag[1])
                for (int p = n.tid; p < L::NP; p += kWThreads) a.best[p] = __ldg(a.theta + p);
        }
    }
    wide_teardown(n);
}

// ---- host side ----
struct WideWork {
    void *buf = nullptr;
    size_t cap = 0;
    bool attrs = false;
    // the full-sample loss passes of epochs 1..E-1 and the predictions run on this
    // low-priority stream, on the SMs the trainer's grid leaves free
    cudaStream_t side = nullptr;
    cudaEvent_t ev_train = nullptr, ev_side = nullptr;
};
std::mutex g_wide_mu;
std::atomic<uint32_t> g_grid_polls{kGridPolls};
WideWork g_wide[64];


// grid of the trainer: at most one CTA per SM, about two tiles per CTA and round
int wide_grid(int tiles_per_batch, int sms)
{
    int G = tiles_per_batch >= 2 ? (tiles_per_batch + 1) / 2 : 1;
    return G > sms ? sms : G;
}
}  // namespace

void mlp_wide_set_grid_polls(uint32_t polls) { g_grid_polls.store(polls == UINT32_MAX ? kGridPolls : polls); }

cva_status mlp_wide_plan(int tiles_per_batch, int32_t out[4])
{
    int dev = 0, sms = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = wide_grid(tiles_per_batch, sms);
    out[0] = G;
    out[1] = 0;
    out[2] = tiles_per_batch;
    out[3] = (tiles_per_batch + G - 1) / G;
    return CVA_OK;
}

cva_status mlp_wide_fit_dates(const float *feat0, size_t feat_stride, const float *targ0, size_t targ_stride,
                              int n_dates, int F, uint64_t M, int n_batches, int epochs, float lr, int max_steps,
                              float *params_dev, float *pred0, float *grad_out_dev, float *loss_out_dev,
                              unsigned *count, int *err, cudaStream_t st)
{
    constexpr int Z = WL::Z;
    const int tiles_per_batch = (int)(M / n_batches / kRows);
    int dev = 0, sms = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_wide_mu);
    WideWork &w = g_wide[dev];
    if (!w.attrs) {
        CVA_CUDA_TRY(cudaFuncSetAttribute(wide_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WL::bytes));
        CVA_CUDA_TRY(cudaFuncSetAttribute(wide_sweep_kernel<WL, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          WL::bytes));
        CVA_CUDA_TRY(cudaFuncSetAttribute(wide_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WLP::bytes));
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_refit_kernel<WL::U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)refit_smem_bytes(WL::U)));
        int least = 0, greatest = 0;
        CVA_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CVA_CUDA_TRY(cudaStreamCreateWithPriority(&w.side, cudaStreamNonBlocking, least));
        CVA_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_train, cudaEventDisableTiming));
        CVA_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_side, cudaEventDisableTiming));
        w.attrs = true;
    }
    int per_sm = 0;
    CVA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wide_train_kernel, kWThreads, WL::bytes));
    if (per_sm < 1) return fail(CVA_ENOTSUP, "mlp: the width-128 trainer does not fit on an SM");
    const int G = wide_grid(tiles_per_batch, sms);
    const uint64_t tiles = M / kRows;
    const int sweep_grid = (int)(tiles < (uint64_t)sms ? tiles : (uint64_t)sms);
    // passes that overlap the training take the SMs its grid leaves (the trainer's CTA
    // fills an SM, and so does a pass's); with fewer than 8 of them every pass stays on
    // st with the whole GPU
    const bool overlap = sms - G >= 8;
    const int side_grid = overlap ? (int)(tiles < (uint64_t)(sms - G) ? tiles : (uint64_t)(sms - G)) : sweep_grid;
    const int fwd_grid = sweep_grid;
    const cudaStream_t sst = overlap ? w.side : st;

    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_vec = al((size_t)WL::NPpad * 4), b_img = al((size_t)WL::img_elems * 2),
                 b_stats = al((size_t)n_dates * 2 * kIn * 4), b_snaps = al((size_t)epochs * WL::NPpad * 4),
                 b_part = al((size_t)G * WL::NPpad * 4), b_flags = al(4), b_bl = al(8),
                 b_G = al(refit_g_bytes(WL::U)), b_pl = al((size_t)(fwd_grid > sweep_grid ? fwd_grid : sweep_grid) * 8),
                 b_pg = al((size_t)sweep_grid * Z * Z * 8);
    const size_t need = 5 * b_vec + b_img + b_stats + b_snaps + b_part + b_flags + 2 * b_bl + b_G + b_pl + b_pg;
    if (w.cap < need) {
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        CVA_CUDA_TRY(cudaStreamSynchronize(w.side));
        if (w.buf) cudaFree(w.buf);
        w.buf = nullptr;
        w.cap = 0;
        if (cudaMalloc(&w.buf, need) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: workspace (width 128)");
        w.cap = need;
    }
    char *p = static_cast<char *>(w.buf);
    auto take = [&](size_t b) {
        char *r = p;
        p += b;
        return r;
    };
    float *adam_m = reinterpret_cast<float *>(take(b_vec)), *adam_v = reinterpret_cast<float *>(take(b_vec));
    float *gq = reinterpret_cast<float *>(take(b_vec));
    float *best[2] = {reinterpret_cast<float *>(take(b_vec)), reinterpret_cast<float *>(take(b_vec))};
    uint16_t *gimg = reinterpret_cast<uint16_t *>(take(b_img));
    float *stats = reinterpret_cast<float *>(take(b_stats));
    float *snaps = reinterpret_cast<float *>(take(b_snaps));
    float *gpart = reinterpret_cast<float *>(take(b_part));
    unsigned *flags = reinterpret_cast<unsigned *>(take(b_flags));
    double *best_loss[2] = {reinterpret_cast<double *>(take(b_bl)), reinterpret_cast<double *>(take(b_bl))};
    double *Gm = reinterpret_cast<double *>(take(b_G));
    double *part_loss = reinterpret_cast<double *>(take(b_pl));
    double *part_gram = reinterpret_cast<double *>(take(b_pg));

    mlp_stats_kernel<<<dim3(kIn, (unsigned)n_dates), 256, 0, st>>>(feat0, F, (uint32_t)M, feat_stride, stats);
    CVA_CUDA_TRY(cudaGetLastError());

    WTrainArgs ta = {};
    ta.F = F;
    ta.M = (uint32_t)M;
    ta.tiles_per_batch = tiles_per_batch;
    ta.lr = lr;
    ta.beta1 = 0.9f;
    ta.beta2 = 0.999f;
    ta.eps = 1e-8f;
    ta.params = params_dev;
    ta.adam_m = adam_m;
    ta.adam_v = adam_v;
    ta.gq = gq;
    ta.gimg = gimg;
    ta.gpart = gpart;
    ta.flags = flags;
    ta.grid_polls = g_grid_polls.load();
    ta.grad_out = grad_out_dev;
    ta.err = err;

    WSweepArgs sw = {};
    sw.F = F;
    sw.M = (uint32_t)M;
    sw.count = count + 1;
    sw.part = part_loss;
    sw.loss_out = loss_out_dev;
    sw.err = err;

    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kWThreads);
    cfg.dynamicSmemBytes = WL::bytes;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;

    int steps_left = max_steps > 0 ? max_steps : INT_MAX;
    for (int d = n_dates - 1; d >= 0; --d) {
        const int par = d & 1;
        const float *feat = feat0 + (size_t)d * feat_stride, *targ = targ0 + (size_t)d * targ_stride;
        CUtensorMap tm;
        cva_status r = features_map(&tm, feat, F, M);
        if (r != CVA_OK) return r;
        ta.targ = sw.targ = targ;
        ta.stats = sw.stats = stats + (size_t)d * 2 * kIn;
        ta.best = sw.best = best[par];
        ta.best_loss = sw.best_loss = best_loss[par];
        for (int e = 1; e <= epochs; ++e) {
            float *snap = snaps + (size_t)(e - 1) * WL::NPpad;
            ta.init = (e == 1 && d < n_dates - 1) ? best[par ^ 1] : params_dev;   // Algorithm 2's warm start
            ta.snap = snap;
            ta.n_steps = n_batches < steps_left ? n_batches : steps_left;
            ta.step0 = (e - 1) * n_batches;
            ta.pos = (epochs / 2 >= 1 && e > epochs / 2) ? 1 : 0;
            CVA_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            const bool timed = mlp_timing_pair(dev, &t0, &t1);
            if (timed) CVA_CUDA_TRY(cudaEventRecord(t0, st));
            CVA_CUDA_TRY(cudaLaunchKernelEx(&cfg, wide_train_kernel, ta, tm));
            if (timed) CVA_CUDA_TRY(cudaEventRecord(t1, st));
            steps_left -= ta.n_steps;
            if (max_steps > 0 && steps_left <= 0) {
                if (overlap) {   // passes already requested finish before the caller's stream moves on
                    CVA_CUDA_TRY(cudaEventRecord(w.ev_side, sst));
                    CVA_CUDA_TRY(cudaStreamWaitEvent(st, w.ev_side, 0));
                }
                return CVA_OK;
            }
            if (e == epochs / 2) {
                WSweepArgs g = sw;
                g.mode = 1;
                g.theta = params_dev;
                g.part = part_gram;
                g.loss_out = nullptr;
                wide_sweep_kernel<WL, 1><<<sweep_grid, kWThreads, WL::bytes, st>>>(g, tm);
                CVA_CUDA_TRY(cudaGetLastError());
                mlp_refit_kernel<WL::U><<<Z, 256, refit_smem_bytes(WL::U), st>>>(part_gram, sweep_grid, Gm, count + 2,
                                                                                 params_dev, snap);
                CVA_CUDA_TRY(cudaGetLastError());
            }
            // the epoch's loss from its snapshot: beside the next epoch's training on the
            // free SMs, the last epoch's with the whole GPU (the next date waits for it)
            sw.mode = 0;
            sw.theta = snap;
            sw.epoch = e;
            if (overlap) {
                CVA_CUDA_TRY(cudaEventRecord(w.ev_train, st));
                CVA_CUDA_TRY(cudaStreamWaitEvent(sst, w.ev_train, 0));
            }
            wide_fwd_kernel<<<e == epochs ? fwd_grid : side_grid, kWThreads, WLP::bytes, sst>>>(sw, tm);
            CVA_CUDA_TRY(cudaGetLastError());
        }
        // the best parameters are known once the last loss pass ran: the next date (st)
        // starts from them; the predictions (side) overlap its training
        if (overlap) {
            CVA_CUDA_TRY(cudaEventRecord(w.ev_side, sst));
            CVA_CUDA_TRY(cudaStreamWaitEvent(st, w.ev_side, 0));
        }
        if (pred0) {
            WSweepArgs pv = sw;
            pv.mode = 2;
            pv.theta = best[par];
            pv.pred = pred0 + (size_t)d * M;
            wide_fwd_kernel<<<side_grid, kWThreads, WLP::bytes, sst>>>(pv, tm);
            CVA_CUDA_TRY(cudaGetLastError());
        }
        if (d == 0)
            CVA_CUDA_TRY(cudaMemcpyAsync(params_dev, best[par], WL::NP * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    if (overlap) {   // the caller's stream sees every pass
        CVA_CUDA_TRY(cudaEventRecord(w.ev_side, sst));
        CVA_CUDA_TRY(cudaStreamWaitEvent(st, w.ev_side, 0));
    }
    return CVA_OK;
}

}  // namespace cva
