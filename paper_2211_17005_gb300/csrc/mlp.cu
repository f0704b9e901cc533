// Neural regression of Sec. 2 on tcgen05 tensor cores: the NN+ network of eq.
// (e:nnp) (two hidden ReLU layers of width U, output zeta^+ + mu) trained at one
// pricing date by Algorithm 1 (BaseAlg):
//   * mini-batch Adam over contiguous path ranges, output ReLU off for the first
//     floor(E/2) epochs;
//   * at epoch floor(E/2) the last layer (w3, b3) is refitted in closed form by
//     least squares on the last hidden layer (normal equations in FP64);
//   * after every epoch the full-sample loss (output ReLU on) decides whether the
//     parameters are the best so far.
// Algorithm 2 (backward learning) runs this once per date, from the last date
// down, each date starting from the previous date's best parameters.
//
// Kernels of one date, in order on the caller's stream:
//   mlp_stats_kernel   input standardisation (FP64 sums), Adam state reset
//   mlp_train_kernel   one epoch of Adam steps on ONE thread-block cluster
//   mlp_sweep_kernel   full-sample forward passes on all SMs: the epoch loss and
//                      the best-parameter choice, the Gram matrix of the refit, or
//                      the predictions
//   mlp_refit_kernel   sum of the Gram partials, FP64 Cholesky, new (w3, b3)
//
// Every CTA runs two warpgroups, each owning one 128-row tile slot. Per tile:
//   GEMM1  D = X W1^T                    (K = 32 padded inputs)
//   GEMM2  D = H1 W2^T                   (K = U)
//   GEMM3  D = dH2 W2                    (K = U; the W2 image read MN-major)
//   GEMMW  DW (+)= [dH2 | dH1]^T [H1 | 1 | X | 1]   (K = the tile's 128 paths;
//          both operands read MN-major from per-path rows)
// so that every operand is written as 16-byte pieces of its path's row. BF16
// operands in shared memory, FP32 accumulators in tensor memory; biases, ReLU,
// the output layer and the loss in FP32 on the CUDA cores. A tile's inputs (one
// 128-path row per feature, one 2-D TMA box of the feature array, and the 512
// bytes of targets, one bulk copy) are requested one tile ahead by a single
// thread while the tensor core runs the tile's first GEMM, and complete on the
// slot's staging mbarrier.
//
// One Adam step inside the cluster: each CTA writes its FP32 gradient partial
// into its own shared memory; after a cluster barrier CTA c sums slice c of the
// parameter vector over all CTAs' partials (distributed shared memory, 16-byte
// accesses, fixed CTA order), applies Adam to the slice and stores the new values
// into every CTA's copy of the parameters; a second cluster barrier publishes them.
//
// Consecutive train launches of a date use programmatic dependent launch: a
// running train kernel lets the next one become resident (on its own cluster of
// SMs) and that one waits, in hardware, for its predecessor to complete before
// it reads anything. The next epoch's cluster is thus placed before the loss pass
// of the side stream can take the SMs it needs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <climits>
#include <atomic>
#include <mutex>
#include <vector>
#include <string>

#include "cva_internal.h"
#include "mlp_common.cuh"
#include "umma.cuh"

namespace cva {

namespace {

constexpr int kThreads = 256;     // two warpgroups, one tile slot each
constexpr int kMaxCluster = 16;

// byte offset of element c of row r in a 128-element-wide BF16 row buffer stored
// as K-major core matrices (8 rows x 16 bytes): 16 core matrices per 8-row group
__host__ __device__ constexpr uint32_t row_off(uint32_t r, uint32_t c)
{
    return (r >> 3) * 2048u + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

template <int U>
struct Layout {
    static_assert(U == 64, "the operand rows [dH2 | dH1] and [H1 | 1 | X | 1] are 128 wide for U = 64");
    static constexpr int NP = 35 * U + U * U + 2;     // parameters
    static constexpr int NPpad = (NP + 63) / 64 * 64;
    static constexpr int oW1 = 0, ob1 = kIn * U, oW2 = ob1 + U, ob2 = oW2 + U * U, ow3 = ob2 + U,
                         ob3 = ow3 + U, omu = ob3 + 1;
    static constexpr int Z = U + 2;                   // refit: [h2 | 1] unknowns and the target column
    // columns of the row buffers: B = [H1 | 1 0.. | X | 1 0..], A = [dH2 | dH1]
    static constexpr int cOne1 = U, cX = U + 16, cOne2 = U + 48, cDH1 = U;
    // shared memory (bytes)
    static constexpr int sSlot = 65536;                         // slot s: A at s * sSlot, B at + 32768
    static constexpr int sW1 = 2 * sSlot;                       // W1 image [U][32], K-major
    static constexpr int sW2 = sW1 + U * kIn * 2;               // W2 image [U][U], K-major
    static constexpr int sTh = sW2 + U * U * 2;                 // parameters, FP32, column order
    static constexpr int sStage = sTh + NPpad * 4;              // [2][kIn + 1][128] FP32 inputs, target
    static constexpr int sVec = sStage + 2 * (kIn + 1) * kRows * 4;   // mean[32], istd[32]
    static constexpr int sGsl = sVec + 2 * kIn * 4;             // [8 warps][U + 2] output-layer gradients
    static constexpr int sRecv = sGsl + 8 * (U + 2) * 4;        // train: [CL][NPpad / CL] partial slices received
    static constexpr int bytes_train = sRecv + NPpad * 4;
    static constexpr int bytes_sweep = sRecv;
    static constexpr uint32_t tmem_cols = 512;   // D of slot s at [64 s, 64 s + U), DW at [128 + 128 s, +128)

    // The shared copy of the parameters and the gradient partials keep W1 and W2
    // column by column (q order), so that the owner of a slice and the writers of
    // the partials touch consecutive words; global memory keeps the row order (p).
    __host__ __device__ static int q_of(int p)
    {
        if (p < ob1) return oW1 + (p % kIn) * U + p / kIn;
        if (p >= oW2 && p < ob2) {
            const int t = p - oW2;
            return oW2 + (t % U) * U + t / U;
        }
        return p;
    }
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

struct TrainArgs {
    const float *feat, *targ;      // [F][M] state at the date, [M] targets
    int F;
    uint32_t M;
    int tiles_per_batch, n_steps, step0, pos;   // batches 0..n_steps-1; Adam steps step0+1..; output ReLU
    float lr, beta1, beta2, eps;
    const float *init;             // [NP] row order: parameters at the start of the launch
    float *params;                 // [NP] row order: parameters at its end (may equal init)
    float *snap;                   // [NP] row order: a second copy of them (nullable)
    float *best;                   // step0 == 0: receives init (the date's best so far) ...
    double *best_loss;             // ... and +inf
    float *adam_m, *adam_v;        // [NPpad] column order; step0 == 0: the moments start at zero
    const float *stats;            // mean[32], 1/std[32]
    float *grad_out;               // [NP] row order: gradient of the date's first step (nullable)
    int *err;
};

struct SweepArgs {
    const float *feat, *targ;
    int F;
    uint32_t M;
    int mode;                      // 0 loss, 1 Gram of the refit, 2 predictions
    const float *theta;            // [NP] parameters of the pass, row order
    const float *stats;
    double *part;                  // per-CTA partials
    unsigned *count;               // last-CTA ticket (mode 0)
    double *best_loss;             // mode 0
    float *best;                   // mode 0: receives theta when its loss is the lowest so far
    float *loss_out;               // mode 0: [epochs] (nullable)
    int epoch;
    float *pred;                   // mode 2 (nullable)
    float *params_out;             // mode 2: receives theta (nullable)
    int *err;
};

template <int U>
struct Net {
    using L = Layout<U>;
    unsigned char *smem;
    uint32_t tmem = 0;
    uint64_t *mbar, *sbar;         // tensor-core completion, input staging (this slot's)
    uint32_t phase = 0, sphase = 0;
    bool pending = false;          // a staging copy was issued and not yet consumed
    int tid, warp, lane, slot, row;
    const float *th, *mean, *istd;
    float *stage;

    __device__ Net(unsigned char *s, uint64_t *mbars) : smem(s)
    {
        tid = threadIdx.x;
        warp = tid >> 5;
        lane = tid & 31;
        slot = tid >> 7;
        row = tid & 127;
        mbar = mbars + slot;
        sbar = mbars + 2 + slot;
        th = reinterpret_cast<const float *>(smem + L::sTh);
        mean = reinterpret_cast<const float *>(smem + L::sVec);
        istd = mean + kIn;
        stage = reinterpret_cast<float *>(smem + L::sStage) + slot * (kIn + 1) * kRows;
    }

    __device__ int offA() const { return slot * L::sSlot; }
    __device__ int offB() const { return slot * L::sSlot + 32768; }
    __device__ uint32_t dcol() const { return 64u * (uint32_t)slot; }
    __device__ uint32_t wcol() const { return 128u + 128u * (uint32_t)slot; }
    __device__ uint32_t saddr(int off) const { return umma::smem_u32(smem + off); }
    __device__ uint32_t taddr(uint32_t col) const { return tmem + ((uint32_t)((warp & 3) * 32) << 16) + col; }
    __device__ void ld16(uint32_t col, float (&v)[16]) const { umma::tmem_ld16(taddr(col), v); }

    // the 128 threads of this slot
    __device__ void wg_sync() const { asm volatile("bar.sync %0, 128;" ::"r"(1 + slot) : "memory"); }
    __device__ bool wg_all(bool p) const
    {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(r)
            : "r"((uint32_t)p), "r"(1 + slot)
            : "memory");
        return r != 0;
    }

    // one tensor-core step of this slot: operands written -> issue (row 0) ->
    // completion; the result is the same for the whole slot
    // side() runs in every thread of the slot after the slot barrier, while the
    // tensor core works (it may request the next tile's inputs)
    template <class Issue, class Side>
    __device__ bool mma(Issue issue, bool pre_ok, Side side)
    {
        umma::fence_proxy_async();
        umma::fence_before_sync();
        wg_sync();
        umma::fence_after_sync();
        if (row == 0) {
            issue();
            umma::commit(mbar);
        }
        side();
        const bool done = umma::mbar_wait(mbar, phase, kMbarPolls);
        phase ^= 1u;
        umma::fence_after_sync();
        return wg_all(done && pre_ok);
    }
    template <class Issue>
    __device__ bool mma(Issue issue)
    {
        return mma(issue, true, [] {});
    }

    // D = A B^T: A = K columns of the rows from column c0 (K-major), B = a K-major image [N][K]
    __device__ void gemm_rows(uint32_t d, int a_off, int c0, int b_off, int K, int N, bool acc) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, (uint32_t)N);
        const uint32_t a0 = saddr(a_off) + (uint32_t)(c0 / 8) * 128u, b0 = saddr(b_off);
        const uint32_t bsbo = (uint32_t)(K / 8) * 128u;
        for (int kk = 0; kk < K / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(a0 + kk * 256u, 128u, 2048u),
                           umma::smem_desc(b0 + kk * 256u, 128u, bsbo), id, (acc || kk > 0) ? 1u : 0u);
    }

    // D = A W2 (B[n][k] = W2[k][n]): the W2 image read MN-major
    __device__ void gemm_rows_w2t(uint32_t d, int a_off) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, U) | umma::kMnMajorB;
        const uint32_t a0 = saddr(a_off), b0 = saddr(L::sW2), lbo = (U / 8) * 128u;
        for (int kk = 0; kk < U / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(a0 + kk * 256u, 128u, 2048u),
                           umma::smem_desc(b0 + kk * 2u * lbo, lbo, 128u), id, kk > 0 ? 1u : 0u);
    }

    // D (+)= A^T B over the tile's 128 rows: the 128 columns of A's rows and the
    // first N columns of B's rows, both read MN-major
    __device__ void gemm_paths(uint32_t d, int a_off, int b_off, int N, bool acc) const
    {
        const uint32_t id = umma::idesc_bf16_f32(kRows, (uint32_t)N) | umma::kMnMajorA | umma::kMnMajorB;
        const uint32_t a0 = saddr(a_off), b0 = saddr(b_off);
        for (int kk = 0; kk < kRows / 16; ++kk)
            umma::mma_bf16(tmem + d, umma::smem_desc(a0 + kk * 4096u, 2048u, 128u),
                           umma::smem_desc(b0 + kk * 4096u, 2048u, 128u), id, (acc || kk > 0) ? 1u : 0u);
    }

    // ---- inputs ----
    // stage the tile of paths [path0, path0 + 128): the F feature rows (one box of
    // the tensor map at (path0, 0)) and the target row, completing on this slot's
    // staging barrier. Called by every thread of the slot once all of them are done
    // reading the staging area; one thread issues the copies.
    __device__ void prefetch(const CUtensorMap *tm, const float *targ, int F, uint32_t path0)
    {
        if (row == 32) {
            umma::mbar_arrive_expect_tx(sbar, (uint32_t)(F + 1) * kRows * 4u);
            umma::tma_load_2d(umma::smem_u32(stage), tm, (int32_t)path0, 0, sbar);
            umma::bulk_g2s(umma::smem_u32(stage + kIn * kRows), targ + path0, kRows * 4u, sbar);
        }
        pending = true;
    }

    // wait for the staged tile; standardised inputs of this thread's row into the X
    // columns of B (rows f >= F of the staging area hold zeros, as do their mean and
    // 1/std); y receives the target. False if the bounded wait gave up.
    __device__ bool stage_x(float &y)
    {
        const bool ok = umma::mbar_wait(sbar, sphase, kMbarPolls);
        sphase ^= 1u;
        pending = false;
        const float4 *mv = reinterpret_cast<const float4 *>(mean), *iv = reinterpret_cast<const float4 *>(istd);
        float x[kIn];
#pragma unroll
        for (int g = 0; g < kIn / 4; ++g) {
            const float4 m = mv[g], r = iv[g];
            x[4 * g + 0] = (stage[(4 * g + 0) * kRows + row] - m.x) * r.x;
            x[4 * g + 1] = (stage[(4 * g + 1) * kRows + row] - m.y) * r.y;
            x[4 * g + 2] = (stage[(4 * g + 2) * kRows + row] - m.z) * r.z;
            x[4 * g + 3] = (stage[(4 * g + 3) * kRows + row] - m.w) * r.w;
        }
        unsigned char *b = smem + offB();
#pragma unroll
        for (int g = 0; g < kIn / 8; ++g) *reinterpret_cast<uint4 *>(b + row_off(row, L::cX + 8 * g)) = pack8(x + 8 * g);
        y = stage[kIn * kRows + row];
        return ok;
    }

    // constant columns of B (ones after H1 and after X, zeros beside them), both slots
    __device__ void init_constants()
    {
        const uint4 one = make_uint4((uint32_t)bf16_bits(1.f), 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
        unsigned char *b = smem + offB();
        *reinterpret_cast<uint4 *>(b + row_off(row, L::cOne1)) = one;
        *reinterpret_cast<uint4 *>(b + row_off(row, L::cOne1 + 8)) = zero;
        *reinterpret_cast<uint4 *>(b + row_off(row, L::cOne2)) = one;
        *reinterpret_cast<uint4 *>(b + row_off(row, L::cOne2 + 8)) = zero;
    }

    // BF16 images of W1 and W2 from the shared parameters (all 256 threads)
    __device__ void build_images()
    {
        const int o = tid & (U - 1), g = tid / U;   // 4 column groups of 8
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = th[L::oW1 + (8 * g + k) * U + o];
        *reinterpret_cast<uint4 *>(smem + L::sW1 + umma::kmajor_offset(o, 8 * g, kIn)) = pack8(v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gg = g + 4 * h;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = th[L::oW2 + (8 * gg + k) * U + o];
            *reinterpret_cast<uint4 *>(smem + L::sW2 + umma::kmajor_offset(o, 8 * gg, U)) = pack8(v);
        }
    }

    // ---- epilogues (thread = row of the tile) ----
    // H1 = relu(D + b1) into B; the mask of h1 > 0 in m1
    __device__ void epi1(uint32_t (&m1)[U / 32]) const
    {
        unsigned char *b = smem + offB();
        const float4 *b1 = reinterpret_cast<const float4 *>(th + L::ob1);
        float v[64];
        umma::tmem_ld64(taddr(dcol()), v);
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
        for (int g = 0; g < 8; ++g) *reinterpret_cast<uint4 *>(b + row_off(row, 8 * g)) = pack8(v + 8 * g);
    }

    // second hidden layer of this thread's row from its accumulator: h2 = relu(D + b2)
    // in place, and zeta = w3 . h2 + b3 (four partial sums)
    __device__ float layer2(float (&v)[64]) const
    {
        const float4 *b2 = reinterpret_cast<const float4 *>(th + L::ob2), *w3 = reinterpret_cast<const float4 *>(th + L::ow3);
        umma::tmem_ld64(taddr(dcol()), v);
        float acc[4] = {th[L::ob3], 0.f, 0.f, 0.f};
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

    // output of this thread's row: zeta (+ relu if pos) + mu
    __device__ float output(int pos, float &outv) const
    {
        float v[64];
        const float out = layer2(v);
        outv = out;
        return (pos ? fmaxf(out, 0.f) : out) + th[L::omu];
    }

    // output, loss derivative and the output-layer backward of this thread's row:
    // dH2 = dout w3 (h2 > 0) into A; the column sums of h2 dout (dw3), of dout (db3)
    // and of dpred (dmu) over the warp's rows into this warp's slots gsl
    __device__ void out_back2(int pos, float y, float inv_batch, float *gsl) const
    {
        unsigned char *a = smem + offA();
        const float4 *w3 = reinterpret_cast<const float4 *>(th + L::ow3);
        float v[64];
        const float out = layer2(v);
        const float pred = (pos ? fmaxf(out, 0.f) : out) + th[L::omu];
        const float dpred = 2.f * (pred - y) * inv_batch;
        const float dout = pos ? (out > 0.f ? dpred : 0.f) : dpred;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float4 w0 = w3[2 * g], w1 = w3[2 * g + 1];
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float d[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) d[i] = v[8 * g + i] > 0.f ? dout * wv[i] : 0.f;
            *reinterpret_cast<uint4 *>(a + row_off(row, 8 * g)) = pack8(d);
        }
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] *= dout;
        const float2 cs = column_sums64(v, lane);
        gsl[2 * lane] += cs.x;
        gsl[2 * lane + 1] += cs.y;
        const float s3 = warp_sum(dout), smu = warp_sum(dpred);
        if (lane == 0) {
            gsl[U] += s3;
            gsl[U + 1] += smu;
        }
    }

    // dH1 = D (h1 > 0) into A
    __device__ void back1(const uint32_t (&m1)[U / 32]) const
    {
        unsigned char *a = smem + offA();
        float v[64];
        umma::tmem_ld64(taddr(dcol()), v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = ((m1[i / 32] >> (i % 32)) & 1u) ? v[i] : 0.f;
#pragma unroll
        for (int g = 0; g < 8; ++g) *reinterpret_cast<uint4 *>(a + row_off(row, L::cDH1 + 8 * g)) = pack8(v + 8 * g);
    }

    // first two layers of the staged tile (staging status in_ok); D holds the second-layer
    // pre-activation after it. side() runs during the first GEMM, when every thread of
    // the slot is past the staging area (the next tile's copies may be requested).
    template <class Side>
    __device__ bool forward12(uint32_t (&m1)[U / 32], bool in_ok, Side side)
    {
        if (!mma([&] { gemm_rows(dcol(), offB(), L::cX, L::sW1, kIn, U, false); }, in_ok, side)) return false;
        epi1(m1);
        return mma([&] { gemm_rows(dcol(), offB(), 0, L::sW2, U, U, false); });
    }

    // forward + backward of one tile whose inputs stage_x has placed (target y, staging
    // status in_ok); weight gradients accumulate in this slot's DW
    __device__ bool train_tile(const TrainArgs &a, const CUtensorMap *tm, float y, bool in_ok, bool first,
                               float inv_batch, bool has_next, uint32_t next_path, float *gsl)
    {
        uint32_t m1[U / 32];
        if (!forward12(m1, in_ok, [&] {
                if (has_next) prefetch(tm, a.targ, a.F, next_path);
            }))
            return false;
        out_back2(a.pos, y, inv_batch, gsl);
        if (!mma([&] { gemm_rows_w2t(dcol(), offA()); })) return false;
        back1(m1);
        return mma([&] { gemm_paths(wcol(), offA(), offB(), kRows, !first); });
    }

    // this CTA's gradient partial (both slots' DW + the output-layer slots) into P, q order
    __device__ void write_partial(float *P, float *gsl, bool h0, bool h1) const
    {
        const int q4 = warp & 3, wg = warp >> 2;
        const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
        // every TMEM load of the thread is issued before the one wait; a chunk past the
        // thread's range reads allocated columns whose values are not used
        if (q4 < 2) {   // rows o < U: dW2[o][:] at columns [0, U), db2[o] at column U
            const int o = q4 * 32 + lane;
            const int k0 = wg ? 3 : 0, k1 = wg ? 5 : 3;
            float v0[3][16], v1[3][16];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                umma::tmem_ld16(tmem + lanes + 128u + 16u * (uint32_t)(k0 + j), v0[j]);
                umma::tmem_ld16(tmem + lanes + 256u + 16u * (uint32_t)(k0 + j), v1[j]);
            }
            umma::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(v0[j][i]), "+f"(v1[j][i]));
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (k0 + j < k1) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int col = 16 * (k0 + j) + i;
                        const float g = (h0 ? v0[j][i] : 0.f) + (h1 ? v1[j][i] : 0.f);
                        if (col < U) P[L::oW2 + col * U + o] = g;
                        else if (col == U) P[L::ob2 + o] = g;
                    }
                }
        } else {        // rows U + i: dW1[i][:] at columns [cX, cX + 32), db1[i] at column cOne2
            const int i0 = (q4 - 2) * 32 + lane;
            const int k0 = wg ? 7 : 5, k1 = wg ? 8 : 7;
            float v0[2][16], v1[2][16];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                umma::tmem_ld16(tmem + lanes + 128u + 16u * (uint32_t)(k0 + j), v0[j]);
                umma::tmem_ld16(tmem + lanes + 256u + 16u * (uint32_t)(k0 + j), v1[j]);
            }
            umma::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(v0[j][i]), "+f"(v1[j][i]));
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (k0 + j < k1) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int f = 16 * (k0 + j) + i - L::cX;
                        const float g = (h0 ? v0[j][i] : 0.f) + (h1 ? v1[j][i] : 0.f);
                        if (f < kIn) P[L::oW1 + f * U + i0] = g;
                        else if (f == kIn) P[L::ob1 + i0] = g;
                    }
                }
        }
        if (tid < U + 2) {
            float s = 0.f;
            for (int w = 0; w < 8; ++w) s += gsl[w * (U + 2) + tid];
            P[tid < U ? L::ow3 + tid : (tid == U ? L::ob3 : L::omu)] = s;
        }
        __syncthreads();
        for (int i = tid; i < 8 * (U + 2); i += kThreads) gsl[i] = 0.f;
    }
};

// common start of the train and sweep kernels: TMEM, mbarriers, parameters (q
// order), standardisation, constant operand columns, weight images
template <int U>
__device__ void net_setup(Net<U> &n, uint32_t *s_tmem, uint64_t *s_mbar, const float *params, const float *stats,
                          int F, bool zero_a)
{
    using L = Layout<U>;
    if (n.warp == 0) {
        umma::tmem_alloc(s_tmem, L::tmem_cols);
        umma::tmem_relinquish();
    }
    if (n.tid == 0) {
        for (int i = 0; i < 4; ++i) umma::mbar_init(&s_mbar[i], 1);
        umma::fence_mbar_init();
    }
    float *th = reinterpret_cast<float *>(n.smem + L::sTh);
    for (int q = n.tid; q < L::NPpad; q += kThreads) th[q] = q < L::NP ? __ldg(params + L::p_of(q)) : 0.f;
    float *vec = reinterpret_cast<float *>(n.smem + L::sVec);
    if (n.tid < 2 * kIn) vec[n.tid] = __ldg(stats + n.tid);
    float *gsl = reinterpret_cast<float *>(n.smem + L::sGsl);
    for (int i = n.tid; i < 8 * (U + 2); i += kThreads) gsl[i] = 0.f;
    // staging rows of the padded inputs stay zero (the copies fill rows < F)
    float *stg = reinterpret_cast<float *>(n.smem + L::sStage);
    for (int i = n.tid; i < 2 * (kIn + 1) * kRows; i += kThreads) {
        const int f = (i / kRows) % (kIn + 1);
        if (f >= F && f < kIn) stg[i] = 0.f;
    }
    if (zero_a) {
        uint4 *a = reinterpret_cast<uint4 *>(n.smem + n.offA());
        for (int i = n.row; i < 32768 / 16; i += kRows) a[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    n.init_constants();
    __syncthreads();
    n.build_images();
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    n.tmem = *s_tmem;
}

template <int U>
__device__ void net_teardown(Net<U> &n)
{
    if (n.pending) (void)umma::mbar_wait(n.sbar, n.sphase, kMbarPolls);   // no copy outlives the CTA
    umma::fence_before_sync();
    __syncthreads();
    if (n.warp == 0) umma::tmem_dealloc(n.tmem, Layout<U>::tmem_cols);
}

// One epoch (or its first n_steps batches) of Adam on one cluster of CL >= 4 CTAs.
// Batch b covers paths [b * P, (b + 1) * P), P = tiles_per_batch * 128; in each
// step the cluster's 2 CL slots take the batch's tiles round-robin.
//
// The exchange of one Adam step moves data only by bulk copies between the CTAs'
// shared memories, each completing on the receiver's mbarrier (no cluster-wide
// barrier inside the step loop):
//   1. every CTA writes its gradient partial (column order q) and copies slice c
//      of it into CTA c's receive buffer, at row = its own rank;
//   2. CTA c waits for the CL slices of its own slice, sums them in CTA order,
//      applies Adam (moments in global memory, requested before the wait) and
//      writes the new values into its own copy of the parameters;
//   3. CTA c copies that slice into every other CTA's copy of the parameters;
//      every CTA waits for the other CL - 1 slices before its next step.
// A CTA's next partial reaches an owner only after that CTA received the owner's
// new slice, which the owner sent after summing the previous partials: the
// receive buffer, the partial and the parameter slices are never overwritten
// while still being read.
template <int U>
__global__ void __launch_bounds__(kThreads, 1) mlp_train_kernel(TrainArgs a, const __grid_constant__ CUtensorMap tm)
{
    using L = Layout<U>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];
    __shared__ __align__(8) uint64_t s_xbar[2];   // exchange: partial slices received, parameter slices received
    Net<U> n(smem, s_mbar);
    const uint32_t rank = umma::cluster_rank(), CL = umma::cluster_size();
    float *th = reinterpret_cast<float *>(smem + L::sTh);
    float *part = reinterpret_cast<float *>(smem);   // slot 0's A rows, free between steps
    float *gsl = reinterpret_cast<float *>(smem + L::sGsl);
    const float *recv = reinterpret_cast<const float *>(smem + L::sRecv);
    // owned slice [lo, hi) of the padded parameter vector: a multiple of 4 entries
    const int S = L::NPpad / (int)CL, lo = (int)rank * S, hi = lo + S;
    const uint32_t slice_bytes = (uint32_t)S * 4u;

    // the previous kernel of the stream has completed and its writes are visible;
    // from here on the next train launch may become resident
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (n.tid == 0) {
        umma::mbar_init(&s_xbar[0], 1);
        umma::mbar_init(&s_xbar[1], 1);
    }
    net_setup<U>(n, &s_tmem, s_mbar, a.init, a.stats, a.F, false);   // fences the barrier initialisation
    if (a.step0 == 0 && rank == 0) {   // start of a date: the starting parameters are the best so far
        for (int p = n.tid; p < L::NP; p += kThreads) a.best[p] = __ldg(a.init + p);
        if (n.tid == 0) *a.best_loss = 1e300;
    }
    umma::cluster_sync();   // every CTA's exchange barriers exist before any copy targets them

    const uint32_t per_batch = (uint32_t)a.tiles_per_batch * kRows;
    const float inv_batch = 1.f / (float)per_batch;
    const int span = 2 * (int)CL, my = 2 * (int)rank + n.slot;
    const int my_rounds = my < a.tiles_per_batch ? (a.tiles_per_batch - 1 - my) / span + 1 : 0;
    auto path_of = [&](int st, int rd) { return (uint32_t)st * per_batch + (uint32_t)(rd * span + my) * kRows; };
    const bool h0 = 2 * (int)rank < a.tiles_per_batch, h1 = 2 * (int)rank + 1 < a.tiles_per_batch;
    float *my_gsl = gsl + n.warp * (U + 2);
    const uint32_t part_s = umma::smem_u32(part), th_s = umma::smem_u32(th), recv_s = umma::smem_u32(recv);
    const uint32_t xbar_part = umma::smem_u32(&s_xbar[0]), xbar_par = umma::smem_u32(&s_xbar[1]);
    uint32_t ph_part = 0, ph_par = 0;

    // bias corrections 1 - beta^t of Adam, as running powers of beta
    float b1t = powf(a.beta1, (float)a.step0), b2t = powf(a.beta2, (float)a.step0);
    bool ok = true, staged = false, in_ok_next = true;
    float y_next = 0.f;
    if (my_rounds > 0) n.prefetch(&tm, a.targ, a.F, path_of(0, 0));
    for (int st = 0; st < a.n_steps; ++st) {
        for (int rd = 0; rd < my_rounds && ok; ++rd) {
            const bool last = rd + 1 == my_rounds;
            const bool has_next = !last || st + 1 < a.n_steps;
            const uint32_t next = last ? path_of(st + 1, 0) : path_of(st, rd + 1);
            float y = y_next;
            bool in_ok = in_ok_next;
            if (!staged) in_ok = n.stage_x(y);   // else placed during the previous exchange
            staged = false;
            ok = n.train_tile(a, &tm, y, in_ok, rd == 0, inv_batch, has_next, next, my_gsl);
            if (!ok && n.row == 0) atomicExch(a.err, 2);
        }
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        n.write_partial(part, gsl, h0, h1);
        umma::fence_proxy_async();   // the partial is read by the bulk copies (async proxy)
        __syncthreads();
        if (n.tid < (int)CL)   // slice c of this CTA's partial -> CTA c's receive buffer, row `rank`
            umma::bulk_s2c(umma::map_rank(recv_s + rank * slice_bytes, (uint32_t)n.tid),
                           part_s + (uint32_t)n.tid * slice_bytes, slice_bytes,
                           umma::map_rank(xbar_part, (uint32_t)n.tid));

        // the next step's first tile: its inputs into the X columns of B (free since the
        // weight-gradient GEMM completed) while the exchange runs
        if (ok && my_rounds > 0 && st + 1 < a.n_steps) {
            in_ok_next = n.stage_x(y_next);
            staged = true;
        }

        // the owned slice: Adam moments requested before the wait for the partials
        const int step = a.step0 + st + 1;
        const bool fresh = a.step0 == 0 && st == 0;   // the moments of a date start at zero
        b1t *= a.beta1;
        b2t *= a.beta2;
        const float inv_bc1 = 1.f / (1.f - b1t), inv_bc2 = 1.f / (1.f - b2t);
        const int q_first = lo + 4 * n.tid;
        float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f), v4 = m4;
        if (q_first < hi && !fresh) {
            m4 = __ldcg(reinterpret_cast<const float4 *>(a.adam_m + q_first));
            v4 = __ldcg(reinterpret_cast<const float4 *>(a.adam_v + q_first));
        }
        if (n.tid == 0) umma::mbar_arrive_expect_tx(&s_xbar[0], (uint32_t)L::NPpad * 4u);
        if (!umma::mbar_wait(&s_xbar[0], ph_part, kMbarPolls)) {
            ok = false;
            atomicExch(a.err, 4);
        }
        ph_part ^= 1u;
        auto adam = [&](int q, float g, float &m, float &v) -> float {
            if (step == 1 && a.grad_out && q < L::NP) a.grad_out[L::p_of(q)] = g;
            if (q >= L::NP || (q < L::ob1 && q / U >= a.F)) return 0.f;   // padding stays zero
            m = a.beta1 * m + (1.f - a.beta1) * g;
            v = a.beta2 * v + (1.f - a.beta2) * g * g;
            return th[q] - adam_delta(m, v, inv_bc1, inv_bc2, a.lr, a.eps);
        };
        for (int q0 = q_first; q0 < hi; q0 += 4 * kThreads) {
            if (q0 != q_first && !fresh) {
                m4 = __ldcg(reinterpret_cast<const float4 *>(a.adam_m + q0));
                v4 = __ldcg(reinterpret_cast<const float4 *>(a.adam_v + q0));
            } else if (q0 != q_first) {
                m4 = v4 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float4 *rv = reinterpret_cast<const float4 *>(recv + (q0 - lo));
            float4 pv[kMaxCluster];
#pragma unroll
            for (int c = 0; c < kMaxCluster; ++c)   // all loads in flight
                pv[c] = (uint32_t)c < CL ? rv[c * (S / 4)] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < kMaxCluster; ++c) {   // fixed CTA order
                g.x += pv[c].x;
                g.y += pv[c].y;
                g.z += pv[c].z;
                g.w += pv[c].w;
            }
            const float4 t = make_float4(adam(q0, g.x, m4.x, v4.x), adam(q0 + 1, g.y, m4.y, v4.y),
                                         adam(q0 + 2, g.z, m4.z, v4.z), adam(q0 + 3, g.w, m4.w, v4.w));
            *reinterpret_cast<float4 *>(th + q0) = t;
            __stcg(reinterpret_cast<float4 *>(a.adam_m + q0), m4);
            __stcg(reinterpret_cast<float4 *>(a.adam_v + q0), v4);
        }
        umma::fence_proxy_async();   // the new slice is read by the bulk copies
        __syncthreads();
        if (n.tid < (int)CL && n.tid != (int)rank)   // the new slice -> every other CTA's parameters
            umma::bulk_s2c(umma::map_rank(th_s + (uint32_t)lo * 4u, (uint32_t)n.tid), th_s + (uint32_t)lo * 4u,
                           slice_bytes, umma::map_rank(xbar_par, (uint32_t)n.tid));
        if (n.tid == 0) umma::mbar_arrive_expect_tx(&s_xbar[1], (CL - 1u) * slice_bytes);
        if (!umma::mbar_wait(&s_xbar[1], ph_par, kMbarPolls)) {
            ok = false;
            atomicExch(a.err, 4);
        }
        ph_par ^= 1u;
        n.build_images();
        umma::fence_proxy_async();
        __syncthreads();
    }
    for (int q = lo + n.tid; q < hi; q += kThreads) {
        if (q < L::NP) {
            a.params[L::p_of(q)] = th[q];
            if (a.snap) a.snap[L::p_of(q)] = th[q];
        }
    }
    umma::cluster_sync();   // no CTA leaves while another may address its shared memory
    net_teardown<U>(n);
}

// Full-sample passes with fixed parameters, output ReLU on: the loss (mode 0), the
// refit's Gram matrix of Z = [h2 | 1 | y - mu] (mode 1), the predictions (mode 2).
template <int U>
__global__ void __launch_bounds__(kThreads, 1) mlp_sweep_kernel(SweepArgs a, const __grid_constant__ CUtensorMap tm)
{
    using L = Layout<U>;
    constexpr int Z = L::Z;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];
    __shared__ double s_red[8];
    __shared__ int s_flag[2];
    Net<U> n(smem, s_mbar);
    net_setup<U>(n, &s_tmem, s_mbar, a.theta, a.stats, a.F, a.mode == 1);

    const uint32_t tiles = a.M / kRows, stride = 2u * gridDim.x;
    uint32_t t = 2u * blockIdx.x + (uint32_t)n.slot;
    double acc = 0.0;
    bool ok = true, first = true;
    if (t < tiles) n.prefetch(&tm, a.targ, a.F, t * kRows);
    for (; t < tiles && ok; t += stride) {
        const uint32_t nt = t + stride;
        float y;
        const bool in_ok = n.stage_x(y);
        uint32_t m1[U / 32];
        ok = n.forward12(m1, in_ok, [&] {
            if (nt < tiles) n.prefetch(&tm, a.targ, a.F, nt * kRows);
        });
        if (ok && a.mode != 1) {
            float out;
            const float pred = n.output(1, out);
            if (a.mode == 2) {
                if (a.pred) a.pred[t * kRows + n.row] = pred;
            } else {
                acc += (double)((pred - y) * (pred - y));
            }
        } else if (ok) {
            // row of Z into A: [relu(D + b2) | 1 | y - mu | 0 ...]
            unsigned char *ar = smem + n.offA();
            float v[64];
            (void)n.layer2(v);
#pragma unroll
            for (int g = 0; g < 8; ++g) *reinterpret_cast<uint4 *>(ar + row_off(n.row, 8 * g)) = pack8(v + 8 * g);
            *reinterpret_cast<uint4 *>(ar + row_off(n.row, U)) =
                make_uint4(pack2(1.f, y - n.th[L::omu]), 0u, 0u, 0u);
            // G (+)= Z^T Z: M = the 128 columns of the rows (Z in the first U + 2), N = U + 16
            ok = n.mma([&] { n.gemm_paths(n.wcol(), n.offA(), n.offA(), U + 16, !first); });
        }
        if (!ok && n.row == 0) atomicExch(a.err, 2);
        first = false;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    if (a.mode == 0) {
        double s = acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (n.lane == 0) s_red[n.warp] = s;
        __syncthreads();
        if (n.tid == 0) {
            double b = 0.0;
            for (int w = 0; w < 8; ++w) b += s_red[w];
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
                for (int p = n.tid; p < L::NP; p += kThreads) a.best[p] = __ldg(a.theta + p);
        }
    } else if (a.mode == 1) {   // this CTA's Gram (both slots) as FP64, rows/columns [0, Z)
        const int q4 = n.warp & 3, wg = n.warp >> 2, R = q4 * 32 + n.lane;
        const bool h0 = 2u * blockIdx.x < tiles, h1 = 2u * blockIdx.x + 1u < tiles;
        double *P = a.part + (size_t)blockIdx.x * Z * Z;
        if (q4 < 3) {
            const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
            const int k0 = wg ? 3 : 0, k1 = wg ? 5 : 3;
            for (int k = k0; k < k1; ++k) {
                float v0[16], v1[16];
                umma::tmem_ld16(n.tmem + lanes + 128u + 16u * k, v0);
                umma::tmem_ld16(n.tmem + lanes + 256u + 16u * k, v1);
                umma::tmem_wait_ld();
                if (R < Z)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * k + i;
                        if (c < Z) P[R * Z + c] = (h0 ? (double)v0[i] : 0.0) + (h1 ? (double)v1[i] : 0.0);
                    }
            }
        }
    } else if (blockIdx.x == 0 && a.params_out) {
        for (int p = n.tid; p < L::NP; p += kThreads) a.params_out[p] = __ldg(a.theta + p);
    }
    net_teardown<U>(n);
}

// ---- host side ----
// Per-device state: the workspace, counters and status word, and two internal
// streams. Training runs on the high-priority one; the full-sample loss of each
// epoch and the predictions run on the low-priority one, beside the next epoch's
// training (the train kernel occupies one cluster; the passes use the other SMs).
struct MlpWork {
    void *buf = nullptr;
    size_t cap = 0;          // bytes
    unsigned *count = nullptr;
    int *err = nullptr;
    bool attrs = false;
    int max_cluster = 0;     // 16 when a 16-CTA cluster of the train kernel fits, else 8
    cudaStream_t main = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_train = nullptr, ev_side = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> tev;   // timing events, a pair around each train launch
    size_t tev_used = 0;
};
std::mutex g_mlp_mu;
MlpWork g_mlp[64];

// kernel timing of the train launches (cva_mlp_kernel_timing); totals under g_mlp_mu
std::atomic<bool> g_mlp_timing{false};
double g_train_ms = 0.0;
uint64_t g_train_launches = 0;

// the next pair of timing events of a device (created on first use), false when
// timing is off or an event cannot be created; the caller holds g_mlp_mu
bool timing_pair_locked(MlpWork &w, cudaEvent_t &a, cudaEvent_t &b)
{
    if (!g_mlp_timing.load()) return false;
    while (w.tev.size() < w.tev_used + 2) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        w.tev.push_back(e);
    }
    a = w.tev[w.tev_used];
    b = w.tev[w.tev_used + 1];
    w.tev_used += 2;
    return true;
}

struct MlpPlan {
    float *adam, *best[2], *stats, *snaps;
    double *best_loss[2], *part_loss, *part_gram, *G;
    int sweep_grid, cluster;
};

// kernel attributes, the largest cluster the train kernel can run on, the internal
// streams and events of a device (once per device; the caller holds g_mlp_mu)
cva_status mlp_attrs(MlpWork &w)
{
    using L = Layout<64>;
    if (!w.attrs) {
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          L::bytes_train));
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel<64>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_sweep_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          L::bytes_sweep));
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_refit_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)refit_smem_bytes(64)));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = L::bytes_train;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n16 = 0;
        if (cudaOccupancyMaxActiveClusters(&n16, mlp_train_kernel<64>, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            n16 = 0;
        }
        w.max_cluster = n16 >= 1 ? 16 : 8;
        int least = 0, greatest = 0;
        CVA_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CVA_CUDA_TRY(cudaStreamCreateWithPriority(&w.main, cudaStreamNonBlocking, greatest));
        CVA_CUDA_TRY(cudaStreamCreateWithPriority(&w.side, cudaStreamNonBlocking, least));
        for (cudaEvent_t *e : {&w.ev_fork, &w.ev_train, &w.ev_side, &w.ev_join})
            CVA_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        w.attrs = true;
    }
    return CVA_OK;
}

// cluster of the train kernel for a batch of tiles_per_batch tiles: the smallest
// power of two >= 4 whose two tile slots per CTA cover the batch in one round, at
// most the largest cluster that fits
int mlp_cluster(const MlpWork &w, int tiles_per_batch)
{
    int cl = 4;
    while (cl < w.max_cluster && 2 * cl < tiles_per_batch) cl *= 2;
    return cl;
}

cva_status mlp_prepare(int dev, int sms, uint64_t M, int tiles_per_batch, int n_dates, int epochs, cudaStream_t st,
                       MlpWork *&wout, MlpPlan &pl)
{
    using L = Layout<64>;
    MlpWork &w = g_mlp[dev];
    cva_status ar = mlp_attrs(w);
    if (ar != CVA_OK) return ar;
    const uint64_t tiles = M / kRows;
    const int rounds = (int)((tiles + 2 * (uint64_t)sms - 1) / (2 * (uint64_t)sms));
    pl.sweep_grid = (int)((tiles + 2 * (uint64_t)rounds - 1) / (2 * (uint64_t)rounds));
    pl.cluster = mlp_cluster(w, tiles_per_batch);
    constexpr int Z = L::Z;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_adam = al(2 * (size_t)L::NPpad * 4), b_best = al((size_t)L::NPpad * 4),
                 b_stats = al((size_t)n_dates * 2 * kIn * 4), b_snaps = al((size_t)epochs * L::NPpad * 4), b_bl = al(8),
                 b_G = al(refit_g_bytes(64)), b_pl = al((size_t)pl.sweep_grid * 8),
                 b_pg = al((size_t)pl.sweep_grid * Z * Z * 8);
    const size_t need = b_adam + 2 * b_best + b_stats + b_snaps + 2 * b_bl + b_G + b_pl + b_pg;
    if (w.cap < need) {
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        CVA_CUDA_TRY(cudaStreamSynchronize(w.main));
        CVA_CUDA_TRY(cudaStreamSynchronize(w.side));
        if (w.buf) cudaFree(w.buf);
        w.buf = nullptr;
        w.cap = 0;
        if (cudaMalloc(&w.buf, need) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: workspace");
        w.cap = need;
    }
    if (!w.count) {
        if (cudaMalloc(&w.count, 4 * sizeof(unsigned)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: counters");
        if (cudaMalloc(&w.err, sizeof(int)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: status");
    }
    char *p = static_cast<char *>(w.buf);
    auto take = [&](size_t b) {
        char *r = p;
        p += b;
        return r;
    };
    pl.adam = reinterpret_cast<float *>(take(b_adam));
    pl.best[0] = reinterpret_cast<float *>(take(b_best));
    pl.best[1] = reinterpret_cast<float *>(take(b_best));
    pl.stats = reinterpret_cast<float *>(take(b_stats));
    pl.snaps = reinterpret_cast<float *>(take(b_snaps));
    pl.best_loss[0] = reinterpret_cast<double *>(take(b_bl));
    pl.best_loss[1] = reinterpret_cast<double *>(take(b_bl));
    pl.G = reinterpret_cast<double *>(take(b_G));
    pl.part_loss = reinterpret_cast<double *>(take(b_pl));
    pl.part_gram = reinterpret_cast<double *>(take(b_pg));
    wout = &w;
    return CVA_OK;
}

// validation shared by every entry
cva_status mlp_check_args(int F, uint64_t M, int U, int n_batches, int epochs)
{
    if (U != 64 && U != 128) return fail(CVA_ENOTSUP, "mlp: hidden widths 64 and 128 are compiled");
    if (F < 1 || F > kIn) return fail(CVA_EINVAL, "mlp: need 1 <= F <= 32 inputs");
    if (n_batches < 1 || epochs < 1) return fail(CVA_EINVAL, "mlp: need batches >= 1, epochs >= 1");
    if (M == 0 || M % ((uint64_t)n_batches * kRows) != 0 || M > 0x7fffffffull)
        return fail(CVA_EINVAL, "mlp: M must be a positive multiple of 128 * batches");
    return CVA_OK;
}

}  // namespace

int mlp_num_params(int U) { return 35 * U + U * U + 2; }

cva_status mlp_plan(uint64_t M, int U, int n_batches, int32_t out[4])
{
    cva_status r = mlp_check_args(1, M, U, n_batches, 1);
    if (r != CVA_OK) return r;
    const int tiles_per_batch = (int)(M / n_batches / kRows);
    if (U == 128) return mlp_wide_plan(tiles_per_batch, out);
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    MlpWork &w = g_mlp[dev];
    r = mlp_attrs(w);
    if (r != CVA_OK) return r;
    const int cl = mlp_cluster(w, tiles_per_batch);
    out[0] = cl;
    out[1] = cl;
    out[2] = tiles_per_batch;
    out[3] = (tiles_per_batch + 2 * cl - 1) / (2 * cl);
    return CVA_OK;
}

bool mlp_timing_pair(int dev, cudaEvent_t *a, cudaEvent_t *b)
{
    if (dev < 0 || dev >= 64 || !g_mlp_timing.load()) return false;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    return timing_pair_locked(g_mlp[dev], *a, *b);
}

void mlp_kernel_timing(bool on, double *ms, uint64_t *launches)
{
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    if (ms) *ms = g_train_ms;
    if (launches) *launches = g_train_launches;
    g_train_ms = 0.0;
    g_train_launches = 0;
    g_mlp_timing.store(on);
}

cva_status mlp_begin(cudaStream_t st)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    MlpWork &w = g_mlp[dev];
    w.tev_used = 0;
    if (!w.count) {
        if (cudaMalloc(&w.count, 4 * sizeof(unsigned)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: counters");
        if (cudaMalloc(&w.err, sizeof(int)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: status");
    }
    CVA_CUDA_TRY(cudaMemsetAsync(w.count, 0, 4 * sizeof(unsigned), st));
    CVA_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    return CVA_OK;
}

cva_status mlp_finish(cudaStream_t st)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    int *err = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mlp_mu);
        err = g_mlp[dev].err;
    }
    int herr = 0;
    if (err) CVA_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CVA_CUDA_TRY(cudaStreamSynchronize(st));
    {   // every timed train launch has ended: add its duration
        std::lock_guard<std::mutex> lk(g_mlp_mu);
        MlpWork &w = g_mlp[dev];
        for (size_t i = 0; i + 1 < w.tev_used; i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, w.tev[i], w.tev[i + 1]) == cudaSuccess) {
                g_train_ms += ms;
                ++g_train_launches;
            } else {
                (void)cudaGetLastError();
            }
        }
        w.tev_used = 0;
    }
    if (herr != 0) return fail(CVA_ETIMEOUT, "mlp: a bounded device wait gave up (status " + std::to_string(herr) + ")");
    return CVA_OK;
}

// Algorithm 2 over dates n_dates-1 .. 0 of date-major arrays (Algorithm 1 when
// n_dates = 1). Per date, on the internal streams (forked from and joined back
// to st):
//   main: E train launches (one per epoch; epoch E/2 followed by the Gram pass
//         and the closed-form refit), the date's last loss pass gating the next
//         date, whose first launch starts from the best parameters;
//   side: the full-sample loss of every epoch (deciding the best parameters, in
//         epoch order) and the predictions of the best network.
// Each epoch's parameters are snapshotted for its loss pass; the best parameters
// and best loss alternate between two buffers by date parity, so that a date's
// prediction pass can overlap the next date's training.
cva_status mlp_fit_dates(const float *feat0, size_t feat_stride, const float *targ0, size_t targ_stride, int n_dates,
                         int F, uint64_t M, int U, int n_batches, int epochs, float lr, int max_steps,
                         float *params_dev, float *pred0, float *grad_out_dev, float *loss_out_dev, cudaStream_t st)
{
    cva_status r = mlp_check_args(F, M, U, n_batches, epochs);
    if (r != CVA_OK) return r;
    if (n_dates < 1) return fail(CVA_EINVAL, "mlp: no dates");
    if ((reinterpret_cast<uintptr_t>(feat0) | reinterpret_cast<uintptr_t>(targ0)) & 15u)
        return fail(CVA_EINVAL, "mlp: features and targets must be 16-byte aligned (TMA and bulk copies)");
    if (U == 128) {   // the grid-wide trainer (mlp_wide.cu), on st
        int dev = 0;
        CVA_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
        unsigned *count = nullptr;
        int *err = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_mlp_mu);
            count = g_mlp[dev].count;
            err = g_mlp[dev].err;
        }
        if (!count || !err) return fail(CVA_EINVAL, "mlp: mlp_begin was not called");
        return mlp_wide_fit_dates(feat0, feat_stride, targ0, targ_stride, n_dates, F, M, n_batches, epochs, lr,
                                  max_steps, params_dev, pred0, grad_out_dev, loss_out_dev, count, err, st);
    }
    using L = Layout<64>;
    constexpr int Z = L::Z;
    const int tiles_per_batch = (int)(M / n_batches / kRows);
    int dev = 0, sms = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    MlpWork *w = nullptr;
    MlpPlan pl;
    r = mlp_prepare(dev, sms, M, tiles_per_batch, n_dates, epochs, st, w, pl);
    if (r != CVA_OK) return r;
    const cudaStream_t mst = w->main, sst = w->side;

    CVA_CUDA_TRY(cudaEventRecord(w->ev_fork, st));
    CVA_CUDA_TRY(cudaStreamWaitEvent(mst, w->ev_fork, 0));
    CVA_CUDA_TRY(cudaStreamWaitEvent(sst, w->ev_fork, 0));

    mlp_stats_kernel<<<dim3(kIn, (unsigned)n_dates), 256, 0, mst>>>(feat0, F, (uint32_t)M, feat_stride, pl.stats);
    CVA_CUDA_TRY(cudaGetLastError());

    TrainArgs ta = {};
    ta.F = F;
    ta.M = (uint32_t)M;
    ta.tiles_per_batch = tiles_per_batch;
    ta.lr = lr;
    ta.beta1 = 0.9f;
    ta.beta2 = 0.999f;
    ta.eps = 1e-8f;
    ta.params = params_dev;
    ta.adam_m = pl.adam;
    ta.adam_v = pl.adam + L::NPpad;
    ta.grad_out = grad_out_dev;
    ta.err = w->err;

    SweepArgs sw = {};
    sw.F = F;
    sw.M = (uint32_t)M;
    sw.count = w->count + 1;
    sw.part = pl.part_loss;
    sw.loss_out = loss_out_dev;
    sw.err = w->err;

    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)pl.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)pl.cluster);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = L::bytes_train;
    cfg.stream = mst;
    cfg.attrs = at;
    cfg.numAttrs = 2;

    bool stopped = false;
    int steps_left = max_steps > 0 ? max_steps : INT_MAX;
    for (int d = n_dates - 1; d >= 0 && !stopped; --d) {
        const int par = d & 1;
        const float *feat = feat0 + (size_t)d * feat_stride, *targ = targ0 + (size_t)d * targ_stride;
        CUtensorMap tm;
        r = features_map(&tm, feat, F, M);
        if (r != CVA_OK) return r;
        ta.feat = sw.feat = feat;
        ta.targ = sw.targ = targ;
        ta.stats = sw.stats = pl.stats + (size_t)d * 2 * kIn;
        ta.best = pl.best[par];
        ta.best_loss = pl.best_loss[par];
        sw.best = pl.best[par];
        sw.best_loss = pl.best_loss[par];
        for (int e = 1; e <= epochs; ++e) {
            float *snap = pl.snaps + (size_t)(e - 1) * L::NPpad;
            ta.init = (e == 1 && d < n_dates - 1) ? pl.best[par ^ 1] : params_dev;   // Algorithm 2's warm start
            ta.snap = snap;
            ta.n_steps = n_batches < steps_left ? n_batches : steps_left;
            ta.step0 = (e - 1) * n_batches;
            ta.pos = (epochs / 2 >= 1 && e > epochs / 2) ? 1 : 0;   // on once the refit of epoch floor(E/2) ran
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            const bool timed = timing_pair_locked(*w, t0, t1);
            if (timed) CVA_CUDA_TRY(cudaEventRecord(t0, mst));
            CVA_CUDA_TRY(cudaLaunchKernelEx(&cfg, mlp_train_kernel<64>, ta, tm));
            if (timed) CVA_CUDA_TRY(cudaEventRecord(t1, mst));
            steps_left -= ta.n_steps;
            if (max_steps > 0 && steps_left <= 0) {
                stopped = true;
                break;
            }
            if (e == epochs / 2) {
                SweepArgs g = sw;
                g.mode = 1;
                g.theta = params_dev;
                g.part = pl.part_gram;
                g.loss_out = nullptr;
                mlp_sweep_kernel<64><<<pl.sweep_grid, kThreads, L::bytes_sweep, mst>>>(g, tm);
                CVA_CUDA_TRY(cudaGetLastError());
                mlp_refit_kernel<64><<<Z, 256, refit_smem_bytes(64), mst>>>(pl.part_gram, pl.sweep_grid, pl.G,
                                                                             w->count + 2, params_dev, snap);
                CVA_CUDA_TRY(cudaGetLastError());
            }
            // the epoch's loss on the side stream, from its snapshot
            CVA_CUDA_TRY(cudaEventRecord(w->ev_train, mst));
            CVA_CUDA_TRY(cudaStreamWaitEvent(sst, w->ev_train, 0));
            sw.mode = 0;
            sw.theta = snap;
            sw.epoch = e;
            mlp_sweep_kernel<64><<<pl.sweep_grid, kThreads, L::bytes_sweep, sst>>>(sw, tm);
            CVA_CUDA_TRY(cudaGetLastError());
        }
        if (stopped) break;
        // the best parameters are known once the last loss pass ran: the next date
        // (main) starts from them; the predictions (side) overlap its training
        CVA_CUDA_TRY(cudaEventRecord(w->ev_side, sst));
        CVA_CUDA_TRY(cudaStreamWaitEvent(mst, w->ev_side, 0));
        if (pred0) {
            SweepArgs pv = sw;
            pv.mode = 2;
            pv.theta = pl.best[par];
            pv.pred = pred0 + (size_t)d * M;
            pv.params_out = nullptr;
            mlp_sweep_kernel<64><<<pl.sweep_grid, kThreads, L::bytes_sweep, sst>>>(pv, tm);
            CVA_CUDA_TRY(cudaGetLastError());
        }
        if (d == 0)
            CVA_CUDA_TRY(cudaMemcpyAsync(params_dev, pl.best[par], L::NP * sizeof(float), cudaMemcpyDeviceToDevice,
                                         mst));
    }
    CVA_CUDA_TRY(cudaEventRecord(w->ev_join, sst));
    CVA_CUDA_TRY(cudaStreamWaitEvent(mst, w->ev_join, 0));
    CVA_CUDA_TRY(cudaEventRecord(w->ev_join, mst));
    CVA_CUDA_TRY(cudaStreamWaitEvent(st, w->ev_join, 0));
    return CVA_OK;
}

}  // namespace cva
