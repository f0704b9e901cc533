// Neural regression of Sec. 2 on tcgen05 tensor cores: the NN+ network of eq.
// (e:nnp) (two hidden ReLU layers of width U, output zeta^+ + mu) trained at one
// pricing date by Algorithm 1 (BaseAlg):
//   * mini-batch Adam over contiguous path ranges, output ReLU off for the first
//     floor(E/2) epochs;
//   * at epoch floor(E/2) the last layer (w3, b3) is refitted in closed form by
//     least squares on the last hidden layer (normal equations in FP64);
//   * after every epoch the full-sample loss (output ReLU on) decides whether the
//     parameters are the best so far.
// Algorithm 2 (backward learning) calls this once per date, from the last date
// down, each date starting from the previous date's best parameters.
//
// One cooperative launch per date. Every block owns 128-row tiles; per tile:
//   GEMM1  D = X W1^T            (K = 32 padded inputs)
//   GEMM2  D = H1 W2^T           (K = U)
//   GEMM3  D = dH2 W2            (K = U)
//   GEMMW  D = [dH2^T; dH1^T] [H1 | 1 | X | 1]   (K = 128 rows): dW2, db2, dW1, db1,
//          accumulated in tensor memory over the block's tiles of a batch
// with BF16 operands in shared memory and FP32 accumulators in tensor memory;
// biases, ReLU, the output layer and the loss run on the CUDA cores in FP32.
// Blocks exchange FP32 gradient partials through global memory; a bounded grid
// barrier separates the reduction + Adam update from the next step.
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>

#include "cva_internal.h"
#include "umma.cuh"

namespace cva {

namespace {

constexpr int kRows = 128;      // rows per tile (tcgen05 M)
constexpr int kIn = 32;         // padded input width
constexpr uint32_t kMbarPolls = 1u << 26;
constexpr uint32_t kGridPolls = 1u << 24;

template <int U>
struct Layout {
    static constexpr int NP = 35 * U + U * U + 2;     // parameters
    static constexpr int oW1 = 0, ob1 = kIn * U, oW2 = ob1 + U, ob2 = oW2 + U * U, ow3 = ob2 + U,
                         ob3 = ow3 + U, omu = ob3 + 1;
    static constexpr int BROWS = U + 64;               // [H1^T | 1 | X^T | 1]
    static constexpr int bOnes1 = U, bX = U + 16, bOnes2 = U + 48;
    // shared memory (bytes)
    static constexpr int sX = 0;                                    // [128][32]
    static constexpr int sB = sX + kRows * kIn * 2;                 // [BROWS][128]
    static constexpr int sW1 = sB + BROWS * kRows * 2;              // [U][32]
    static constexpr int sW2 = sW1 + U * kIn * 2;                   // [U][U]
    static constexpr int sW2t = sW2 + U * U * 2;                    // [U][U]
    static constexpr int sH = sW2t + U * U * 2;                     // [128][U]
    static constexpr int sA = sH + kRows * U * 2;                   // [2U][128]
    static constexpr int sP = sA + 2 * U * kRows * 2;               // [128][U+1] FP32 h2 * dout
    static constexpr int sVec = sP + kRows * (U + 1) * 4;           // floats
    static constexpr int nVec = 3 * U + 2 + 2 * kIn + 4 * (U + 2) + 64;
    static constexpr int sMisc = sVec + nVec * 4;
    static constexpr int bytes = sMisc + 64;
    static_assert((U + 2) * (U + 2) * 8 <= sP - sH, "refit normal matrix must fit over H and A");
    static constexpr uint32_t tmem_cols = (U + 128 <= 256) ? 256 : 512;   // D at [0,U), DW at [U, U+128)
};

struct MlpArgs {
    const float *feat;      // [F][M] state at the date
    const float *targ;      // [M]
    int F;
    uint32_t M;
    int n_batches, epochs, max_steps;   // max_steps > 0 stops after that many Adam steps (validation)
    float lr, beta1, beta2, eps;
    float *params, *adam_m, *adam_v, *best;   // [NP]
    uint16_t *img_w1, *img_w2, *img_w2t;      // BF16 operand images in the tile layout
    float *partial;                            // [grid][NP]
    double *red;                               // [grid][red_stride]
    int red_stride;
    float *pred;                               // [M] predictions (nullable)
    float *grad_out;                           // [NP] gradient of the first step (nullable)
    float *loss_out;                           // [epochs] full-sample losses (nullable)
    unsigned *bar_count, *bar_gen;
    int *err;
};

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    return (uint32_t)bf16_bits(a) | ((uint32_t)bf16_bits(b) << 16);
}

template <int U>
struct Mlp {
    using L = Layout<U>;
    const MlpArgs &a;
    unsigned char *smem;
    uint32_t tmem;
    uint64_t *mbar;
    uint32_t phase;
    unsigned gen;
    int nblk, tid, warp, lane;
    float *b1, *b2, *w3, *misc, *mean, *istd, *gslot;   // gslot[4][U+2]: per-warp dw3, db3, dmu

    __device__ Mlp(const MlpArgs &args, unsigned char *s) : a(args), smem(s)
    {
        tid = threadIdx.x;
        warp = tid >> 5;
        lane = tid & 31;
        nblk = gridDim.x;
        float *v = reinterpret_cast<float *>(smem + L::sVec);
        b1 = v;
        b2 = b1 + U;
        w3 = b2 + U;
        misc = w3 + U;             // [0] = b3, [1] = mu
        mean = misc + 2;
        istd = mean + kIn;
        gslot = istd + kIn;
        mbar = reinterpret_cast<uint64_t *>(smem + L::sMisc);
        phase = 0;
        gen = 0;
    }

    __device__ uint32_t saddr(int off) const { return umma::smem_u32(smem + off); }

    __device__ bool barrier() { return umma::flag_barrier(a.bar_count, nblk, gen, a.err, kGridPolls); }

    // issue D (+)= A B^T over K with A at `aoff` (rows 128, width K) and B at `boff`
    // (N rows, width K); thread 0 only
    __device__ void gemm(uint32_t dcol, int aoff, int boff, int K, int N, bool acc_in)
    {
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        const uint32_t id = umma::idesc_bf16_f32(kRows, (uint32_t)N);
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ad = umma::smem_desc(saddr(aoff) + kk * 256u, 128u, sbo);
            const uint64_t bd = umma::smem_desc(saddr(boff) + kk * 256u, 128u, sbo);
            umma::mma_bf16(tmem + dcol, ad, bd, id, (acc_in || kk > 0) ? 1u : 0u);
        }
    }

    // operand writes done -> issue (thread 0) -> wait for completion; false on timeout
    __device__ bool run(uint32_t dcol, int aoff, int boff, int K, int N, bool acc_in)
    {
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            gemm(dcol, aoff, boff, K, N, acc_in);
            umma::commit(mbar);
        }
        const bool ok = umma::mbar_wait(mbar, phase, kMbarPolls);
        phase ^= 1u;
        umma::fence_after_sync();
        if (!ok) atomicExch(a.err, 2);
        return ok;
    }

    __device__ uint32_t lane_addr(uint32_t col) const { return tmem + ((uint32_t)(warp * 32) << 16) + col; }

    __device__ void ld16(uint32_t col, float (&v)[16]) { umma::tmem_ld16(lane_addr(col), v); }

    // ---- operand staging ----
    // tile rows [r0, r0+128): standardised inputs into X (row layout) and X^T (rows of B)
    __device__ void load_tile(uint32_t r0, float &y)
    {
        const uint32_t r = r0 + tid;
        float x[kIn];
#pragma unroll
        for (int f = 0; f < kIn; ++f) x[f] = 0.f;
#pragma unroll
        for (int f = 0; f < kIn; ++f)
            if (f < a.F) x[f] = (__ldg(a.feat + (size_t)f * a.M + r) - mean[f]) * istd[f];
        y = __ldg(a.targ + r);
        unsigned char *sx = smem + L::sX, *sb = smem + L::sB;
#pragma unroll
        for (int g = 0; g < kIn / 8; ++g) {
            uint4 v;
            v.x = pack2(x[8 * g], x[8 * g + 1]);
            v.y = pack2(x[8 * g + 2], x[8 * g + 3]);
            v.z = pack2(x[8 * g + 4], x[8 * g + 5]);
            v.w = pack2(x[8 * g + 6], x[8 * g + 7]);
            *reinterpret_cast<uint4 *>(sx + umma::kmajor_offset(tid, 8 * g, kIn)) = v;
        }
#pragma unroll
        for (int f = 0; f < kIn; ++f)
            *reinterpret_cast<uint16_t *>(sb + umma::kmajor_offset(L::bX + f, tid, kRows)) = bf16_bits(x[f]);
    }

    // fixed rows of B: one row of ones after H1^T and after X^T, zeros elsewhere
    __device__ void init_b_constants()
    {
        unsigned char *sb = smem + L::sB;
        for (int i = tid; i < 16 * kRows; i += blockDim.x) {
            const int rr = i / kRows, k = i % kRows;
            const uint16_t one = bf16_bits(1.f), zero = 0;
            *reinterpret_cast<uint16_t *>(sb + umma::kmajor_offset(L::bOnes1 + rr, k, kRows)) = rr == 0 ? one : zero;
            *reinterpret_cast<uint16_t *>(sb + umma::kmajor_offset(L::bOnes2 + rr, k, kRows)) = rr == 0 ? one : zero;
        }
    }

    // parameters from global memory into shared memory
    __device__ void load_params(const float *P)
    {
        const uint4 *g1 = reinterpret_cast<const uint4 *>(a.img_w1), *g2 = reinterpret_cast<const uint4 *>(a.img_w2),
                    *g3 = reinterpret_cast<const uint4 *>(a.img_w2t);
        uint4 *s1 = reinterpret_cast<uint4 *>(smem + L::sW1), *s2 = reinterpret_cast<uint4 *>(smem + L::sW2),
              *s3 = reinterpret_cast<uint4 *>(smem + L::sW2t);
        for (int i = tid; i < U * kIn * 2 / 16; i += blockDim.x) s1[i] = __ldcg(g1 + i);
        for (int i = tid; i < U * U * 2 / 16; i += blockDim.x) {
            s2[i] = __ldcg(g2 + i);
            s3[i] = __ldcg(g3 + i);
        }
        for (int i = tid; i < U; i += blockDim.x) {
            b1[i] = __ldcg(P + L::ob1 + i);
            b2[i] = __ldcg(P + L::ob2 + i);
            w3[i] = __ldcg(P + L::ow3 + i);
        }
        if (tid == 0) {
            misc[0] = __ldcg(P + L::ob3);
            misc[1] = __ldcg(P + L::omu);
        }
        __syncthreads();
    }

    // BF16 operand images of parameter p (grid-stride writers)
    __device__ void write_image(int p, float v)
    {
        if (p < L::ob1) {
            const int o = p / kIn, f = p % kIn;
            a.img_w1[umma::kmajor_offset(o, f, kIn) / 2] = bf16_bits(v);
        } else if (p >= L::oW2 && p < L::ob2) {
            const int q = p - L::oW2, o = q / U, i = q % U;
            a.img_w2[umma::kmajor_offset(o, i, U) / 2] = bf16_bits(v);
            a.img_w2t[umma::kmajor_offset(i, o, U) / 2] = bf16_bits(v);
        }
    }

    // ---- forward to the second hidden layer; h2 of this thread's row stays in TMEM ----
    // returns the h1 > 0 mask bits in m1 and writes H1 (rows) and H1^T (rows of B)
    __device__ bool forward12(uint32_t (&m1)[U / 32])
    {
        if (!run(0, L::sX, L::sW1, kIn, U, false)) return false;
        unsigned char *sh = smem + L::sH, *sb = smem + L::sB;
#pragma unroll
        for (int c = 0; c < U / 16; ++c) {
            float v[16];
            ld16(16 * c, v);
            umma::tmem_wait_ld();
            uint32_t bits = 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = fmaxf(v[i] + b1[16 * c + i], 0.f);
                bits |= (v[i] > 0.f ? 1u : 0u) << i;
            }
            if (c % 2 == 0) m1[c / 2] = bits;
            else m1[c / 2] |= bits << 16;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint4 q;
                q.x = pack2(v[8 * g], v[8 * g + 1]);
                q.y = pack2(v[8 * g + 2], v[8 * g + 3]);
                q.z = pack2(v[8 * g + 4], v[8 * g + 5]);
                q.w = pack2(v[8 * g + 6], v[8 * g + 7]);
                *reinterpret_cast<uint4 *>(sh + umma::kmajor_offset(tid, 16 * c + 8 * g, U)) = q;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
                *reinterpret_cast<uint16_t *>(sb + umma::kmajor_offset(16 * c + i, tid, kRows)) = bf16_bits(v[i]);
        }
        return run(0, L::sH, L::sW2, U, U, false);
    }

    // output of this thread's row from the second-layer accumulator
    __device__ float output(int pos, float &outv)
    {
        float out = misc[0];
#pragma unroll
        for (int c = 0; c < U / 16; ++c) {
            float v[16];
            ld16(16 * c, v);
            umma::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) out = fmaf(fmaxf(v[i] + b2[16 * c + i], 0.f), w3[16 * c + i], out);
        }
        outv = out;
        return (pos ? fmaxf(out, 0.f) : out) + misc[1];
    }

    // warp sum of 32 lanes' values of one column, result in every lane
    __device__ static float warp_sum(float v)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }

    // one tile of forward + backward; weight gradients accumulate in TMEM columns
    // [U, U+128), output-layer gradients in the per-warp slots
    __device__ bool tile_step(uint32_t r0, int pos, float inv_batch, bool first)
    {
        float y;
        load_tile(r0, y);
        uint32_t m1[U / 32];
        if (!forward12(m1)) return false;
        float out;
        const float pred = output(pos, out);
        const float dpred = 2.f * (pred - y) * inv_batch;
        const float dout = pos ? (out > 0.f ? dpred : 0.f) : dpred;
        // dH2 = dout w3 (h2 > 0): rows into H (A of GEMM3), columns into A rows [0, U)
        unsigned char *sh = smem + L::sH, *sa = smem + L::sA;
        float *slot = gslot + warp * (U + 2);
#pragma unroll
        for (int c = 0; c < U / 16; ++c) {
            float v[16];
            ld16(16 * c, v);
            umma::tmem_wait_ld();
            float d[16];
            float *prod = reinterpret_cast<float *>(smem + L::sP) + tid * (U + 1);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float h2 = fmaxf(v[i] + b2[16 * c + i], 0.f);
                d[i] = h2 > 0.f ? dout * w3[16 * c + i] : 0.f;
                prod[16 * c + i] = h2 * dout;            // dw3 contribution of this row
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint4 q;
                q.x = pack2(d[8 * g], d[8 * g + 1]);
                q.y = pack2(d[8 * g + 2], d[8 * g + 3]);
                q.z = pack2(d[8 * g + 4], d[8 * g + 5]);
                q.w = pack2(d[8 * g + 6], d[8 * g + 7]);
                *reinterpret_cast<uint4 *>(sh + umma::kmajor_offset(tid, 16 * c + 8 * g, U)) = q;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
                *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(16 * c + i, tid, kRows)) = bf16_bits(d[i]);
        }
        {
            const float s3 = warp_sum(dout), smu = warp_sum(dpred);
            if (lane == 0) {
                slot[U] += s3;
                slot[U + 1] += smu;
            }
        }
        // GEMM3: dH1 pre-activation = dH2 W2 (B = W2^T rows)
        if (!run(0, L::sH, L::sW2t, U, U, false)) return false;
        if (tid < U) {   // dw3[i] += sum over the tile's rows of h2[r][i] dout[r] (FP32, fixed order)
            const float *prod = reinterpret_cast<const float *>(smem + L::sP) + tid;
            float s = 0.f;
            for (int r = 0; r < kRows; ++r) s += prod[r * (U + 1)];
            gslot[tid] += s;
        }
#pragma unroll
        for (int c = 0; c < U / 16; ++c) {
            float v[16];
            ld16(16 * c, v);
            umma::tmem_wait_ld();
            const uint32_t bits = m1[c / 2] >> (16 * (c % 2));
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float d1 = ((bits >> i) & 1u) ? v[i] : 0.f;
                *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(U + 16 * c + i, tid, kRows)) = bf16_bits(d1);
            }
        }
        // GEMMW: [dH2^T; dH1^T] x [H1^T | 1 | X^T | 1]^T, accumulated over the batch's tiles
        static_assert(2 * U == kRows, "stacked weight-gradient GEMM needs 2U = 128");
        return run(U, L::sA, L::sB, kRows, L::BROWS, !first);
    }

    // write this block's gradient partials (TMEM weight gradients + output slots)
    __device__ void write_partials()
    {
        float *P = a.partial + (size_t)blockIdx.x * L::NP;
        if (warp < 2) {   // rows 0..U-1: dW2[o][:] at cols [0,U), db2[o] at col U
            const int o = tid;
#pragma unroll
            for (int c = 0; c < U / 16 + 1; ++c) {
                float v[16];
                ld16(U + 16 * c, v);
                umma::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = 16 * c + i;
                    if (col < U) P[L::oW2 + col * U + o] = v[i];     // column-major: coalesced over o
                    else if (col == U) P[L::ob2 + o] = v[i];
                }
            }
        } else {          // rows U..2U-1: dW1[i][:] at cols [U+16, U+48), db1[i] at col U+48
            const int i0 = tid - U;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float v[16];
                ld16(U + U + 16 + 16 * c, v);
                umma::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = 16 * c + i;     // relative to X^T rows
                    if (col < kIn) P[L::oW1 + col * U + i0] = v[i];   // column-major: coalesced over i0
                    else if (col == kIn) P[L::ob1 + i0] = v[i];
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < U + 2; i += blockDim.x) {
            const float s = gslot[i] + gslot[(U + 2) + i] + gslot[2 * (U + 2) + i] + gslot[3 * (U + 2) + i];
            if (i < U) P[L::ow3 + i] = s;
            else if (i == U) P[L::ob3] = s;
            else P[L::omu] = s;
        }
        __syncthreads();   // every slot is read before any is cleared
        for (int i = tid; i < 4 * (U + 2); i += blockDim.x) gslot[i] = 0.f;
        __syncthreads();
    }

    // sum of the partials over blocks (fixed order), Adam, new images
    __device__ void adam_update(int step)
    {
        const float bc1 = 1.f - powf(a.beta1, (float)step), bc2 = 1.f - powf(a.beta2, (float)step);
        for (int p = blockIdx.x * blockDim.x + tid; p < L::NP; p += nblk * blockDim.x) {
            int q = p;   // position of parameter p in the (column-major) partial layout
            if (p < L::ob1) q = L::oW1 + (p % kIn) * U + p / kIn;
            else if (p >= L::oW2 && p < L::ob2) q = L::oW2 + ((p - L::oW2) % U) * U + (p - L::oW2) / U;
            float g = 0.f;
            for (int b = 0; b < nblk; ++b) g += __ldcg(a.partial + (size_t)b * L::NP + q);
            if (step == 1 && a.grad_out) a.grad_out[p] = g;
            if (p >= L::oW1 && p < L::ob1 && (p % kIn) >= a.F) continue;   // padded inputs
            const float m = a.beta1 * a.adam_m[p] + (1.f - a.beta1) * g;
            const float v = a.beta2 * a.adam_v[p] + (1.f - a.beta2) * g * g;
            a.adam_m[p] = m;
            a.adam_v[p] = v;
            const float th = __ldcg(a.params + p) - a.lr * (m / bc1) / (sqrtf(v / bc2) + a.eps);
            a.params[p] = th;
            write_image(p, th);
        }
    }

    // full-sample loss (output ReLU on) over this block's tiles, or the refit Gram
    __device__ bool sweep(int mode /*0 loss, 1 gram, 2 predict*/, double &acc)
    {
        const uint32_t tiles = a.M / kRows;
        bool first = true;
        for (uint32_t t = blockIdx.x; t < tiles; t += nblk) {
            const uint32_t r0 = t * kRows;
            float y;
            load_tile(r0, y);
            uint32_t m1[U / 32];
            if (!forward12(m1)) return false;
            if (mode == 0 || mode == 2) {
                float out;
                const float pred = output(1, out);
                if (mode == 2) a.pred[r0 + tid] = pred;
                else acc += (double)((pred - y) * (pred - y));
            } else {
                // Z^T = [h2^T; 1; (y - mu)] into A rows [0, U+2), rows [U+2, 2U) zero
                unsigned char *sa = smem + L::sA;
#pragma unroll
                for (int c = 0; c < U / 16; ++c) {
                    float v[16];
                    ld16(16 * c, v);
                    umma::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(16 * c + i, tid, kRows)) =
                            bf16_bits(fmaxf(v[i] + b2[16 * c + i], 0.f));
                }
                *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(U, tid, kRows)) = bf16_bits(1.f);
                *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(U + 1, tid, kRows)) = bf16_bits(y - misc[1]);
                for (int rr = U + 2; rr < 2 * U; ++rr)
                    *reinterpret_cast<uint16_t *>(sa + umma::kmajor_offset(rr, tid, kRows)) = 0;
                // G (+)= Z^T Z over this block's tiles, rows/cols [0, U+2) of an M=128, N=U+16 product
                if (!run(U, L::sA, L::sA, kRows, U + 16, !first)) return false;
            }
            first = false;
        }
        if (mode == 1 && first) {   // block without tiles: zero Gram
            for (int i = tid; i < (U + 2) * (U + 2); i += blockDim.x) a.red[(size_t)blockIdx.x * a.red_stride + i] = 0.0;
        } else if (mode == 1) {
            // every warp executes the collective loads; rows >= U+2 are discarded
            for (int c = 0; c < (U + 16) / 16; ++c) {
                float v[16];
                ld16(U + 16 * c, v);
                umma::tmem_wait_ld();
                if (tid < U + 2)
                    for (int i = 0; i < 16; ++i) {
                        const int col = 16 * c + i;
                        if (col < U + 2) a.red[(size_t)blockIdx.x * a.red_stride + tid * (U + 2) + col] = (double)v[i];
                    }
            }
        }
        return true;
    }
};

template <int U>
__global__ void __launch_bounds__(128, 1) mlp_train_kernel(MlpArgs a)
{
    using L = Layout<U>;
    extern __shared__ __align__(1024) unsigned char smem[];
    Mlp<U> m(a, smem);
    __shared__ uint32_t s_tmem;
    __shared__ double s_red[128];
    __shared__ int s_flag;

    if (m.warp == 0) {
        umma::tmem_alloc(&s_tmem, L::tmem_cols);
        umma::tmem_relinquish();
    }
    if (m.tid == 0) {
        umma::mbar_init(m.mbar, 1);
        umma::fence_mbar_init();
    }
    for (int i = m.tid; i < 4 * (U + 2); i += blockDim.x) m.gslot[i] = 0.f;
    m.init_b_constants();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    m.tmem = s_tmem;

    const int nblk = gridDim.x;
    bool ok = true;
    // ---- start of the date: Adam state, images, input standardisation ----
    for (int p = blockIdx.x * blockDim.x + m.tid; p < L::NP; p += nblk * blockDim.x) {
        a.adam_m[p] = 0.f;
        a.adam_v[p] = 0.f;
        m.write_image(p, __ldcg(a.params + p));
    }
    {
        // per-feature sums over this block's rows (FP64), then every block combines all
        double s1[kIn], s2[kIn];
        for (int f = 0; f < kIn; ++f) s1[f] = s2[f] = 0.0;
        for (uint32_t r = blockIdx.x * blockDim.x + m.tid; r < a.M; r += nblk * blockDim.x)
            for (int f = 0; f < a.F; ++f) {
                const double x = (double)__ldg(a.feat + (size_t)f * a.M + r);
                s1[f] += x;
                s2[f] += x * x;
            }
        for (int f = 0; f < a.F; ++f) {
            s_red[m.tid] = s1[f];
            __syncthreads();
            for (int s = 64; s > 0; s >>= 1) {
                if (m.tid < s) s_red[m.tid] += s_red[m.tid + s];
                __syncthreads();
            }
            if (m.tid == 0) a.red[(size_t)blockIdx.x * a.red_stride + f] = s_red[0];
            __syncthreads();
            s_red[m.tid] = s2[f];
            __syncthreads();
            for (int s = 64; s > 0; s >>= 1) {
                if (m.tid < s) s_red[m.tid] += s_red[m.tid + s];
                __syncthreads();
            }
            if (m.tid == 0) a.red[(size_t)blockIdx.x * a.red_stride + kIn + f] = s_red[0];
            __syncthreads();
        }
    }
    ok = m.barrier();
    if (ok) {
        if (m.tid < kIn) {
            const int f = m.tid;
            double t1 = 0.0, t2 = 0.0;
            if (f < a.F)
                for (int b = 0; b < nblk; ++b) {
                    t1 += __ldcg(a.red + (size_t)b * a.red_stride + f);
                    t2 += __ldcg(a.red + (size_t)b * a.red_stride + kIn + f);
                }
            const double mu = t1 / a.M, var = t2 / a.M - mu * mu;
            m.mean[f] = f < a.F ? (float)mu : 0.f;
            m.istd[f] = (f < a.F && var > 0.0) ? (float)(1.0 / sqrt(var)) : 0.f;
        }
        ok = m.barrier();   // everyone has read the sums before they are overwritten
    }
    if (ok) m.load_params(a.params);

    const uint32_t per_batch = a.M / (uint32_t)a.n_batches;
    const uint32_t tiles_per_batch = per_batch / kRows;
    const float inv_batch = 1.f / (float)per_batch;
    int pos = 0, step = 0;
    double best = 1e300;
    for (int epoch = 1; ok && epoch <= a.epochs; ++epoch) {
        for (int bt = 0; ok && bt < a.n_batches; ++bt) {
            bool first = true;
            for (uint32_t t = blockIdx.x; ok && t < tiles_per_batch; t += nblk) {
                ok = m.tile_step((uint32_t)bt * per_batch + t * kRows, pos, inv_batch, first);
                first = false;
            }
            if (!ok) break;
            if (first) {   // a block without a tile in this batch contributes zero
                float *P = a.partial + (size_t)blockIdx.x * L::NP;
                for (int i = m.tid; i < L::NP; i += blockDim.x) P[i] = 0.f;
                __syncthreads();
            } else {
                m.write_partials();
            }
            if (!(ok = m.barrier())) break;
            ++step;
            m.adam_update(step);
            if (!(ok = m.barrier())) break;
            m.load_params(a.params);
            if (a.max_steps > 0 && step >= a.max_steps) break;
        }
        if (!ok || (a.max_steps > 0 && step >= a.max_steps)) break;
        if (epoch == a.epochs / 2) {
            // closed-form least squares of (w3, b3) on the last hidden layer, mu fixed
            double dummy = 0.0;
            ok = m.sweep(1, dummy);
            if (ok) ok = m.barrier();
            if (ok && blockIdx.x == 0) {
                constexpr int Z = U + 2;
                double *G = reinterpret_cast<double *>(smem + L::sH);   // [Z][Z] FP64 over H and A
                for (int i = m.tid; i < Z * Z; i += blockDim.x) {
                    double s = 0.0;
                    for (int b = 0; b < nblk; ++b) s += __ldcg(a.red + (size_t)b * a.red_stride + i);
                    G[i] = s;
                }
                __syncthreads();
                if (m.tid == 0) {
                    // Jacobi-scaled Cholesky of the (U+1) x (U+1) normal matrix, in place
                    constexpr int n1 = U + 1;
                    double sc[n1];
                    for (int i = 0; i < n1; ++i) sc[i] = G[i * Z + i] > 0.0 ? 1.0 / sqrt(G[i * Z + i]) : 0.0;
                    for (int i = 0; i < n1; ++i)
                        for (int j = 0; j < n1; ++j) G[i * Z + j] *= sc[i] * sc[j];
                    for (int i = 0; i < n1; ++i) G[i * Z + n1] *= sc[i];
                    bool singular = false;
                    for (int j = 0; j < n1; ++j) {
                        double d = G[j * Z + j];
                        for (int p = 0; p < j; ++p) d -= G[j * Z + p] * G[j * Z + p];
                        if (!(d > 1e-12)) {
                            singular = true;
                            d = 1.0;
                        }
                        d = sqrt(d);
                        G[j * Z + j] = d;
                        for (int i = j + 1; i < n1; ++i) {
                            double s = G[i * Z + j];
                            for (int p = 0; p < j; ++p) s -= G[i * Z + p] * G[j * Z + p];
                            G[i * Z + j] = s / d;
                        }
                    }
                    double y[n1];
                    for (int i = 0; i < n1; ++i) {
                        double s = G[i * Z + n1];
                        for (int p = 0; p < i; ++p) s -= G[i * Z + p] * y[p];
                        y[i] = s / G[i * Z + i];
                    }
                    for (int i = n1 - 1; i >= 0; --i) {
                        double s = y[i];
                        for (int p = i + 1; p < n1; ++p) s -= G[p * Z + i] * y[p];
                        y[i] = s / G[i * Z + i];
                    }
                    if (!singular) {
                        for (int i = 0; i < U; ++i) a.params[L::ow3 + i] = (float)(y[i] * sc[i]);
                        a.params[L::ob3] = (float)(y[U] * sc[U]);
                    }
                }
            }
            if (ok) ok = m.barrier();
            if (ok) m.load_params(a.params);
            pos = 1;
        }
        // full-sample loss with the output ReLU; keep the best parameters
        double acc = 0.0;
        if (ok) ok = m.sweep(0, acc);
        if (!ok) break;
        s_red[m.tid] = acc;
        __syncthreads();
        for (int s = 64; s > 0; s >>= 1) {
            if (m.tid < s) s_red[m.tid] += s_red[m.tid + s];
            __syncthreads();
        }
        if (m.tid == 0) a.red[(size_t)blockIdx.x * a.red_stride + 0] = s_red[0];
        if (!(ok = m.barrier())) break;
        if (m.tid == 0) {
            double tot = 0.0;
            for (int b = 0; b < nblk; ++b) tot += __ldcg(a.red + (size_t)b * a.red_stride);
            tot /= (double)a.M;
            s_flag = tot < best;
            if (tot < best) best = tot;
            if (blockIdx.x == 0 && a.loss_out) a.loss_out[epoch - 1] = (float)tot;
        }
        __syncthreads();
        if (s_flag)
            for (int p = blockIdx.x * blockDim.x + m.tid; p < L::NP; p += nblk * blockDim.x) a.best[p] = __ldcg(a.params + p);
        if (!(ok = m.barrier())) break;   // the sums are read before the next epoch overwrites them
    }
    // ---- end of the date: best parameters become the current ones; predictions ----
    if (ok && a.max_steps == 0) {
        for (int p = blockIdx.x * blockDim.x + m.tid; p < L::NP; p += nblk * blockDim.x) {
            const float v = __ldcg(a.best + p);
            a.params[p] = v;
            m.write_image(p, v);
        }
        ok = m.barrier();
        if (ok) m.load_params(a.params);
        double dummy = 0.0;
        if (ok && a.pred) ok = m.sweep(2, dummy);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (m.warp == 0) umma::tmem_dealloc(m.tmem, L::tmem_cols);
}

struct MlpWork {
    float *buf = nullptr;
    size_t cap = 0;
    unsigned *bar = nullptr;
    int *err = nullptr;
};
std::mutex g_mlp_mu;
MlpWork g_mlp[64];

}  // namespace

int mlp_num_params(int U) { return 35 * U + U * U + 2; }

cva_status mlp_train_date(const float *feat, int F, const float *targ, uint64_t M, int U, int n_batches,
                          int epochs, float lr, int max_steps, float *params_dev, float *pred_dev,
                          float *grad_out_dev, float *loss_out_dev, cudaStream_t st)
{
    if (U != 64) return fail(CVA_ENOTSUP, "mlp: hidden width 64 is compiled");
    if (F < 1 || F > kIn) return fail(CVA_EINVAL, "mlp: need 1 <= F <= 32 inputs");
    if (n_batches < 1 || epochs < 1) return fail(CVA_EINVAL, "mlp: need batches >= 1, epochs >= 1");
    if (M % ((uint64_t)n_batches * kRows) != 0 || M > 0x7fffffffull)
        return fail(CVA_EINVAL, "mlp: M must be a multiple of 128 * batches");
    using L = Layout<64>;
    const int tiles_per_batch = (int)(M / n_batches / kRows);
    int dev = 0, sms = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    static bool attr = false;
    if (!attr) {
        CVA_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::bytes));
        attr = true;
    }
    int per_sm = 0;
    CVA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_train_kernel<64>, 128, L::bytes));
    int grid = 1;   // largest divisor of the tiles per batch that fits co-resident
    for (int g = 1; g <= tiles_per_batch; ++g)
        if (tiles_per_batch % g == 0 && g <= sms * per_sm && g <= 256) grid = g;
    const int red_stride = (L::NP > (64 + 2) * (64 + 2) ? L::NP : (64 + 2) * (64 + 2));
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    MlpWork &w = g_mlp[dev];
    auto al = [](size_t n) { return (n + 63) & ~(size_t)63; };   // 256-byte aligned pieces (in floats)
    const size_t nNP = al(L::NP), nPart = al((size_t)grid * L::NP), nRed = al(2 * (size_t)grid * red_stride),
                 nImg = al((64 * kIn + 2 * 64 * 64) / 2);
    const size_t need = 3 * nNP + nPart + nRed + nImg;
    if (w.cap < need) {
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        if (w.buf) cudaFree(w.buf);
        w.buf = nullptr;
        w.cap = 0;
        if (cudaMalloc(&w.buf, need * sizeof(float)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: workspace");
        w.cap = need;
    }
    if (!w.bar) {
        if (cudaMalloc(&w.bar, 256 * sizeof(unsigned)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: barrier");
        if (cudaMalloc(&w.err, sizeof(int)) != cudaSuccess) return fail(CVA_ENOMEM, "mlp: status");
    }
    CVA_CUDA_TRY(cudaMemsetAsync(w.bar, 0, 256 * sizeof(unsigned), st));
    CVA_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    MlpArgs a;
    a.feat = feat;
    a.targ = targ;
    a.F = F;
    a.M = (uint32_t)M;
    a.n_batches = n_batches;
    a.epochs = epochs;
    a.max_steps = max_steps;
    a.lr = lr;
    a.beta1 = 0.9f;
    a.beta2 = 0.999f;
    a.eps = 1e-8f;
    a.params = params_dev;
    a.adam_m = w.buf;
    a.adam_v = a.adam_m + nNP;
    a.best = a.adam_v + nNP;
    a.partial = a.best + nNP;
    a.red = reinterpret_cast<double *>(a.partial + nPart);
    a.red_stride = red_stride;
    uint16_t *img = reinterpret_cast<uint16_t *>(a.partial + nPart + nRed);
    a.img_w1 = img;
    a.img_w2 = img + 64 * kIn;
    a.img_w2t = a.img_w2 + 64 * 64;
    a.pred = pred_dev;
    a.grad_out = grad_out_dev;
    a.loss_out = loss_out_dev;
    a.bar_count = w.bar;
    a.bar_gen = w.bar + 1;
    a.err = w.err;
    void *kargs[] = {&a};
    CVA_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)mlp_train_kernel<64>, dim3(grid), dim3(128), kargs,
                                             (size_t)L::bytes, st));
    int herr = 0;
    CVA_CUDA_TRY(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr != 0) return fail(CVA_ETIMEOUT, "mlp: a bounded device wait gave up (status " + std::to_string(herr) + ")");
    return CVA_OK;
}

}  // namespace cva
