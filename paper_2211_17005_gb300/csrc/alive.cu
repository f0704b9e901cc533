// Least squares on the hierarchically simulated sample (Sec. "Learning on
// Hierarchically Simulated Paths"): at pricing date i, one row per (outer path k,
// inner draw l) with the features (X_i^{k,l}, Y_i^k), X the default indicators of
// the counterparties and Y the market state (Sec. 4.1), and the per-draw target
//   xi_i^{k,l} = beta_i^{-1} sum_c (1 - R_c) beta_j MtM_c(t_j)^+ 1{i < j <= n},  j = idx_c^{k,l},
// of eq. (eq:CVA_portfolio). The basis is [1, Y - Y^0, X_1..X_C] (Y^0: path 0's state).
//
// The M N rows are never formed. The rows of path k all carry its state and the
// indicators are 0/1, so the normal equations need only these sums over the N draws
// of each path (an exact regrouping of the sum over (k, l)):
//   d_c  = #{l : X_c = 1}            (column sum of X_c, and its products with Y)
//   P_cd = #{l : X_c = X_d = 1}      (c < d: the X_c X_d products)
//   q_c  = sum_l X_c xi^{k,l}        (right-hand side of X_c)
// and N xi_bar^k for the right-hand side of Y. alive_stats_kernel computes them
// (a warp per path, lanes over draws; exact integer counts from warp ballots, a
// fixed-order butterfly for q_c). alive_gram_kernel accumulates
// sum_k [1, Y - Y^0]^T [1, Y - Y^0, d, xi_bar] and the plain sums of P_cd and q_c
// (only the intercept row of those is needed) in FP32 runs of 512 rows per thread,
// then FP64, reduced in a fixed order; and
// alive_solve_kernel assembles the (1 + F + C)-square system and solves it by a
// Jacobi-scaled Cholesky factorisation in FP64, dropping a column whose pivot
// vanishes (a counterparty with no default by t_i anywhere in the sample).
#include <math.h>

#include "cva_internal.h"

namespace cva {

namespace {

constexpr int kGramThreads = 320;   // 79 blocks of 4x4 at the 27-factor, 8-counterparty shape, four row groups
constexpr int kTileRows = 128;
constexpr int kMaxUnknowns = 40;    // 1 + F + C
constexpr int kMaxAug = 80;         // augmented columns of the Gram tile, padded
constexpr int kStatBudget = 160 * 1024;

template <int C>
struct Shape {
    static constexpr int NP = C * (C - 1) / 2;    // pairs c < d
    static constexpr int NS = 2 * C + NP;         // statistics per (path, date): d_c, P_cd, q_c
    static constexpr int LOGC = C == 8 ? 3 : C == 4 ? 2 : C == 2 ? 1 : 0;
    static_assert((1 << LOGC) == C && NP <= 32, "counterparty count must be 2, 4 or 8");
};

// A draw's C default steps (bytes) and C losses at those steps, vector loads.
template <int C>
__device__ __forceinline__ void load_draw(const uint8_t *jp, const float *ep, int (&j)[C], float (&e)[C])
{
    if constexpr (C == 8) {
        const uint2 v = *reinterpret_cast<const uint2 *>(jp);
        const float4 a = reinterpret_cast<const float4 *>(ep)[0], b = reinterpret_cast<const float4 *>(ep)[1];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            j[c] = (v.x >> (8 * c)) & 255u;
            j[4 + c] = (v.y >> (8 * c)) & 255u;
        }
        e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w;
        e[4] = b.x; e[5] = b.y; e[6] = b.z; e[7] = b.w;
    } else if constexpr (C == 4) {
        const uint32_t v = *reinterpret_cast<const uint32_t *>(jp);
        const float4 a = *reinterpret_cast<const float4 *>(ep);
#pragma unroll
        for (int c = 0; c < 4; ++c) j[c] = (v >> (8 * c)) & 255u;
        e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w;
    } else {
        const unsigned short v = *reinterpret_cast<const unsigned short *>(jp);
        const float2 a = *reinterpret_cast<const float2 *>(ep);
        j[0] = v & 255u;
        j[1] = v >> 8;
        e[0] = a.x; e[1] = a.y;
    }
}

struct AliveArgs {
    uint32_t M, N;
    int n, F, C, mY, NS;
    const uint8_t *idx;       // [M][N][C] default steps, n+1 = none
    const float *expo;        // [n+1][C][M] of the portfolio
    const float *disc;        // [n+1][M]
    const float *feat;        // [n+1][F][M]
    const float *targ;        // [n][M] of the portfolio
    float *stats;             // [n][NS][M]: d_c, P_cd (c < d), q_c
    int chunks;
    uint32_t rows_per_chunk;
    int NA, NBf, NB, RS;      // Gram 4x4 blocks: NA rows x NBf full columns, then row 0 x (NB - NBf) sum-only columns
    double *part;             // [n-1][chunks][NBLK*16]
    double *coef;             // [n-1][1+F+C] centred basis
    double *coef_raw;         // [n-1][1+F+C] raw basis
    int *status;              // [n-1] dropped columns
    float *pred;              // [n][M] or null
};

// One warp per path (blockDim.x / 32 paths per block), lanes over the draws. For a
// chunk of 32 draws, the ballot of "c has defaulted by t_i" gives d_c (popc) and,
// ANDed with the ballot of d, P_cd (lane p owns pair p); q_c is the sum over the
// draws of X_c times the draw's later losses, reduced over the warp by a transposed
// butterfly (log2 C halving levels, then plain ones) in a fixed order.
template <int C>
__global__ void __launch_bounds__(256) alive_stats_kernel(AliveArgs a)
{
    using S = Shape<C>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t N = a.N, M = a.M;
    const int n = a.n;
    float *e_s = reinterpret_cast<float *>(smem) + (size_t)warp * N * C;                // [N][C]
    uint8_t *j_s = smem + (size_t)W * N * C * sizeof(float) + (size_t)warp * N * C;     // [N][C]
    const uint32_t kl = blockIdx.x * (uint32_t)W + warp;
    if (kl >= M) return;        // warps are independent: no block barrier below
    {
        const uint8_t *src = a.idx + (size_t)kl * N * C;
        for (uint32_t e = lane; e < N * C; e += 32) {
            const int j = src[e];
            j_s[e] = (uint8_t)j;
            e_s[e] = (j <= n) ? __ldg(a.expo + ((size_t)j * C + e % C) * M + kl) : 0.f;
        }
    }
    __syncwarp();
    int cA = 0, cB = 0;                 // the pair this lane counts
    {
        int p = 0;
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int d = c + 1; d < C; ++d, ++p)
                if (p == lane) {
                    cA = c;
                    cB = d;
                }
    }
    int cq = 0;                         // the counterparty whose q this lane ends up holding
#pragma unroll
    for (int h = 0; h < S::LOGC; ++h)
        if (lane & (16 >> h)) cq += C >> (h + 1);
    const bool q_writer = (lane & ((16 >> S::LOGC) * 2 - 1)) == 0;

    for (int i = 1; i < n; ++i) {
        {
            uint32_t pcnt = 0u, dcnt[C];
            float v[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                dcnt[c] = 0u;
                v[c] = 0.f;
            }
            for (uint32_t l0 = 0; l0 < N; l0 += 32) {
                const uint32_t l = l0 + lane;
                uint32_t x = 0u;        // bit c: counterparty c has defaulted by t_i
                float fut = 0.f;        // the draw's losses after t_i, discounted to 0
                if (l < N) {
                    int j[C];
                    float e[C];
                    load_draw<C>(j_s + (size_t)l * C, e_s + (size_t)l * C, j, e);
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (j[c] <= i) x |= 1u << c;
                        else fut += e[c];
                    }
                }
                uint32_t mA = 0u, mB = 0u;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t mk = __ballot_sync(0xffffffffu, (x >> c) & 1u);
                    dcnt[c] += __popc(mk);
                    mA = (c == cA) ? mk : mA;
                    mB = (c == cB) ? mk : mB;
                    v[c] += ((x >> c) & 1u) ? fut : 0.f;
                }
                pcnt += __popc(mA & mB);
            }
#pragma unroll
            for (int h = 0; h < S::LOGC; ++h) {
                const int off = 16 >> h, half = C >> (h + 1);
                const bool hi = (lane & off) != 0;
#pragma unroll
                for (int t = 0; t < half; ++t) {
                    const float send = hi ? v[t] : v[t + half];
                    const float keep = hi ? v[t + half] : v[t];
                    v[t] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
#pragma unroll
            for (int off = 16 >> S::LOGC; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
            uint32_t dsel = 0u;
#pragma unroll
            for (int c = 0; c < C; ++c) dsel = (c == lane) ? dcnt[c] : dsel;
            // the warps of a block hold neighbouring paths: their stores meet in L2 sectors
            float *out = a.stats + (size_t)i * S::NS * M + kl;
            if (lane < C) out[(size_t)lane * M] = (float)dsel;
            if (lane < S::NP) out[(size_t)(C + lane) * M] = (float)pcnt;
            if (q_writer) out[(size_t)(C + S::NP + cq) * M] = v[0] * expf(__ldg(a.disc + (size_t)i * M + kl));
        }
    }
}

// The column feeding augmented column `col` of the Gram tile at date i: the basis
// [1, Y - Y^0] (mY), then d_c (C), xi_bar, zero padding up to 4 NBf, then P_cd and
// q_c (sum-only columns), zero padding. kind: 0 = the constant 1, 1 = a load
// (minus `sub`), 2 = zero.
struct ColSrc {
    const float *p;
    float sub;
    int kind;
};

__device__ __forceinline__ ColSrc column_source(const AliveArgs &a, const float *feat, const float *stats,
                                                const float *targ, const float *c0, int col)
{
    const int mY = a.mY, C = a.C, NP = C * (C - 1) / 2;
    if (col == 0) return {nullptr, 0.f, 0};
    if (col < mY) return {feat + (size_t)(col - 1) * a.M, c0[col - 1], 1};
    if (col < mY + C) return {stats + (size_t)(col - mY) * a.M, 0.f, 1};
    if (col == mY + C) return {targ, 0.f, 1};
    const int s = col - 4 * a.NBf;
    if (s >= 0 && s < NP + C) return {stats + (size_t)(C + s) * a.M, 0.f, 1};
    return {nullptr, 0.f, 2};
}

// Block b of the Gram: (bi, bj) over NA x NBf, then (0, NBf + t) for the sum-only columns.
__device__ __forceinline__ void gram_block(const AliveArgs &a, int b, int &bi, int &bj)
{
    const int full = a.NA * a.NBf;
    if (b < full) {
        bi = b / a.NBf;
        bj = b % a.NBf;
    } else {
        bi = 0;
        bj = a.NBf + (b - full);
    }
}

// sum over paths of [1, Y - Y^0]^T [1, Y - Y^0, d, xi_bar] and of [P, q] at date i = g + 1
__global__ void __launch_bounds__(kGramThreads, 2) alive_gram_kernel(AliveArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int NB = a.NB, RS = a.RS;
    float *tile = reinterpret_cast<float *>(smem);            // [kTileRows][RS]
    const int g = blockIdx.y, i = g + 1, chunk = blockIdx.x, tid = threadIdx.x;
    const uint32_t M = a.M;
    const float *feat = a.feat + (size_t)i * a.F * M;
    const float *stats = a.stats + (size_t)i * a.NS * M;
    const float *targ = a.targ + (size_t)i * M;
    const uint32_t r_begin = (uint32_t)chunk * a.rows_per_chunk;
    const uint32_t r_end = min(M, r_begin + a.rows_per_chunk);
    const int NBLK = a.NA * a.NBf + (NB - a.NBf), NRG = kGramThreads / NBLK;
    const int b = tid % NBLK, rg = tid / NBLK;
    int bi, bj;
    gram_block(a, b, bi, bj);
    // per augmented column: source array (null: the constant 1 or zero padding) and centring
    __shared__ const float *csrc[kMaxAug];
    __shared__ float csub[kMaxAug], cconst[kMaxAug];
    __shared__ float c0[kMaxUnknowns];
    for (int f = tid; f < a.F; f += kGramThreads) c0[f] = __ldg(feat + (size_t)f * M);
    __syncthreads();
    for (int col = tid; col < 4 * NB; col += kGramThreads) {
        const ColSrc cs = column_source(a, feat, stats, targ, c0, col);
        csrc[col] = cs.kind == 1 ? cs.p : nullptr;
        csub[col] = cs.sub;
        cconst[col] = cs.kind == 0 ? 1.f : 0.f;
    }
    double dacc[16];
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        dacc[e] = 0.0;
        acc[e] = 0.f;
    }
    int since_flush = 0;
    // each thread stages (column, row) elements e = tid + t * kGramThreads of the tile,
    // in two passes of kPer loads issued before their stores
    constexpr int kPer = (kMaxAug * kTileRows / 2 + kGramThreads - 1) / kGramThreads;
    const int n_el = 4 * NB * kTileRows;
    for (uint32_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
        __syncthreads();
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            float stg[kPer];
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int e = tid + (pass * kPer + t) * kGramThreads, col = e / kTileRows, r = e % kTileRows;
                const uint32_t k = r0 + r;
                float v = 0.f;
                if (e < n_el && k < r_end) {
                    const float *src = csrc[col];
                    v = src ? __ldg(src + k) - csub[col] : cconst[col];
                }
                stg[t] = v;
            }
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int e = tid + (pass * kPer + t) * kGramThreads, col = e / kTileRows, r = e % kTileRows;
                if (e < n_el) tile[r * RS + col] = stg[t];
            }
        }
        __syncthreads();
        if (rg < NRG) {
            for (int r = rg; r < kTileRows; r += NRG) {
                const float4 x = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bi);
                const float4 y = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bj);
                const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(xv[u], yv[v], acc[u * 4 + v]);
                if (++since_flush == 512) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        dacc[e] += (double)acc[e];
                        acc[e] = 0.f;
                    }
                    since_flush = 0;
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) dacc[e] += (double)acc[e];
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem);          // [NRG][NBLK*16]
    if (rg < NRG)
#pragma unroll
        for (int e = 0; e < 16; ++e) red[(size_t)rg * NBLK * 16 + b * 16 + e] = dacc[e];
    __syncthreads();
    double *out = a.part + ((size_t)g * a.chunks + chunk) * NBLK * 16;
    for (int e = tid; e < NBLK * 16; e += kGramThreads) {
        double s = 0.0;
        for (int q = 0; q < NRG; ++q) s += red[(size_t)q * NBLK * 16 + e];
        out[e] = s;
    }
}

__global__ void __launch_bounds__(128) alive_solve_kernel(AliveArgs a)
{
    constexpr int MX = kMaxUnknowns;
    __shared__ double R[(MX / 4) * (kMaxAug / 4) * 16];
    __shared__ double A[MX * MX];
    __shared__ double rhs[MX];
    const int g = blockIdx.x, tid = threadIdx.x, i = g + 1;
    const int NBf = a.NBf, NBLK = a.NA * NBf + (a.NB - NBf), mY = a.mY, C = a.C, m = mY + C;
    const int NP = C * (C - 1) / 2;
    for (int e = tid; e < NBLK * 16; e += blockDim.x) {
        double s = 0.0;
        const double *p = a.part + (size_t)g * a.chunks * NBLK * 16 + e;
        for (int c = 0; c < a.chunks; ++c) s += p[(size_t)c * NBLK * 16];
        R[e] = s;
    }
    __syncthreads();
    // R(p, q): row p of [1, Y - Y^0], augmented column q (sum-only columns: row 0 only)
    auto Rv = [&](int p, int q) -> double {
        const int blk = q < 4 * NBf ? (p / 4) * NBf + q / 4 : a.NA * NBf + (q / 4 - NBf);
        return R[blk * 16 + (p % 4) * 4 + (q % 4)];
    };
    if (tid == 0) {   // assemble the (1+F+C)-square system
        const double Nd = (double)a.N;
        for (int p = 0; p < mY; ++p) {
            for (int q = 0; q < mY; ++q) A[p * MX + q] = Nd * Rv(p, q);
            for (int c = 0; c < C; ++c) {
                A[p * MX + mY + c] = Rv(p, mY + c);
                A[(mY + c) * MX + p] = Rv(p, mY + c);
            }
            rhs[p] = Nd * Rv(p, mY + C);
        }
        for (int c = 0; c < C; ++c) {
            A[(mY + c) * MX + mY + c] = Rv(0, mY + c);
            for (int d = c + 1; d < C; ++d) {
                const double v = Rv(0, 4 * NBf + c * (2 * C - c - 1) / 2 + (d - c - 1));
                A[(mY + c) * MX + mY + d] = v;
                A[(mY + d) * MX + mY + c] = v;
            }
            rhs[mY + c] = Rv(0, 4 * NBf + NP + c);
        }
    }
    __syncthreads();
    // Jacobi scaling, then a right-looking Cholesky factorisation of the scaled matrix by
    // the whole block (L overwrites the lower triangle); a column whose pivot vanishes is
    // dropped: its part of L is zero and its coefficient 0
    __shared__ double sc[MX];
    __shared__ int drop[MX];
    for (int r = tid; r < m; r += blockDim.x) {
        const double d = A[r * MX + r];
        drop[r] = !(d > 0.0);
        sc[r] = drop[r] ? 0.0 : 1.0 / sqrt(d);
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        if (c <= r) A[r * MX + c] *= sc[r] * sc[c];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            const double s = A[j * MX + j];
            if (drop[j] || !(s > 1e-12)) {
                drop[j] = 1;
                A[j * MX + j] = 1.0;
            } else {
                A[j * MX + j] = sqrt(s);
            }
        }
        __syncthreads();
        const double inv = drop[j] ? 0.0 : 1.0 / A[j * MX + j];
        for (int r = j + 1 + tid; r < m; r += blockDim.x) A[r * MX + j] *= inv;
        __syncthreads();
        const int t = m - j - 1;
        for (int e = tid; e < t * t; e += blockDim.x) {
            const int r = j + 1 + e / t, c = j + 1 + e % t;
            if (c <= r) A[r * MX + c] -= A[r * MX + j] * A[c * MX + j];
        }
        __syncthreads();
    }
    if (tid != 0) return;
    double y[MX], w[MX];
    int dropped = 0;
    for (int r = 0; r < m; ++r) {                 // L y = D^{-1/2} b
        double s = rhs[r] * sc[r];
        for (int p = 0; p < r; ++p) s -= A[r * MX + p] * y[p];
        y[r] = drop[r] ? 0.0 : s / A[r * MX + r];
        dropped += drop[r];
    }
    for (int r = m - 1; r >= 0; --r) {            // L^T z = y, w = D^{-1/2} z
        double s = y[r];
        for (int p = r + 1; p < m; ++p) s -= A[p * MX + r] * w[p];
        w[r] = drop[r] ? 0.0 : s / A[r * MX + r];
    }
    for (int r = 0; r < m; ++r) w[r] *= sc[r];
    double *co = a.coef + (size_t)g * m, *cr = a.coef_raw + (size_t)g * m;
    double w0 = w[0];
    for (int r = 0; r < m; ++r) {
        co[r] = w[r];
        cr[r] = w[r];
    }
    const float *feat = a.feat + (size_t)i * a.F * a.M;
    for (int f = 0; f < a.F; ++f) w0 -= w[1 + f] * (double)feat[(size_t)f * a.M];
    cr[0] = w0;
    a.status[g] = dropped;
}

// the fitted value at X = 0 (every counterparty alive) per path, date i = blockIdx.y + 1
__global__ void __launch_bounds__(256) alive_predict_kernel(AliveArgs a)
{
    __shared__ float cs[kMaxUnknowns], f0[kMaxUnknowns];
    const int g = blockIdx.y, i = g + 1, m = a.mY + a.C;
    const uint32_t M = a.M;
    const float *feat = a.feat + (size_t)i * a.F * M;
    for (int r = threadIdx.x; r < a.mY; r += blockDim.x) cs[r] = (float)a.coef[(size_t)g * m + r];
    for (int f = threadIdx.x; f < a.F; f += blockDim.x) f0[f] = __ldg(feat + (size_t)f * M);
    __syncthreads();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    float acc = cs[0];
    for (int f = 0; f < a.F; ++f) acc = fmaf(cs[1 + f], __ldg(feat + (size_t)f * M + k) - f0[f], acc);
    a.pred[(size_t)i * M + k] = acc;
}

template <int C>
cva_status launch_stats(const AliveArgs &a, cudaStream_t st)
{
    using S = Shape<C>;
    const size_t per_warp = (size_t)a.N * C * (sizeof(float) + 1);
    int W = (int)(kStatBudget / per_warp);
    if (W > 8) W = 8;
    if (W < 1) return fail(CVA_ENOTSUP, "regress_alive: N * C too large for the per-path draw tables");
    const size_t smem = (size_t)W * per_warp;
    CVA_CUDA_TRY(cudaFuncSetAttribute(alive_stats_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned blocks = (unsigned)((a.M + W - 1) / W);
    alive_stats_kernel<C><<<blocks, 32 * W, smem, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

}  // namespace

cva_status alive_regress(Sim &s, int pf, float *pred_dev, double *coef_host, int *dropped_host, cudaStream_t st)
{
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "regress_alive: portfolio index out of range");
    if (s.n < 2) return fail(CVA_EINVAL, "regress_alive: need at least two pricing steps");
    if (!s.d_idx) return fail(CVA_EINVAL, "regress_alive: the simulation keeps no default steps (CVA_KEEP_DEFAULTS)");
    if (s.C != 2 && s.C != 8) return fail(CVA_ENOTSUP, "regress_alive: compiled for 2 or 8 counterparties");
    if (s.M > 0x7fffffffull) return fail(CVA_EINVAL, "regress_alive: M too large");
    const int C = s.C, NS = 2 * C + C * (C - 1) / 2, mY = s.F + 1, m = mY + C;
    if (m > kMaxUnknowns) return fail(CVA_ENOTSUP, "regress_alive: 1 + F + C must be <= 40");
    // Gram columns: [1, Y - Y^0] (mY), d (C), xi_bar, padding to 4 NBf; then P, q (sum-only), padding
    const int NP = C * (C - 1) / 2, NA = (mY + 3) / 4, NBf = (mY + C + 1 + 3) / 4, NB = NBf + (NP + C + 3) / 4;
    const int RS = (NB & 1) ? 4 * NB : 4 * NB + 4;   // a row stride of 4 x odd floats: column stores hit 8 banks
    if (4 * NB > kMaxAug) return fail(CVA_ENOTSUP, "regress_alive: too many statistics columns");
    if (NA * NBf + (NB - NBf) > kGramThreads) return fail(CVA_ENOTSUP, "regress_alive: Gram blocks exceed the block size");
    const size_t M = s.M;
    const int groups = s.n - 1;
    uint64_t chunks = ((uint64_t)(s.tune_lsq_chunks > 0 ? s.tune_lsq_chunks : 2432) + groups - 1) / groups;
    const uint64_t max_chunks = (M + 1023) / 1024;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const size_t NBLK = (size_t)NA * NBf + (NB - NBf);
    const size_t need = (size_t)groups * chunks * NBLK * 16 + 2 * (size_t)groups * m + (size_t)groups;
    const size_t need_stats = (size_t)s.n * NS * M;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CVA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (s.alive_cap < need || s.alive_stats_cap < need_stats) {
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CVA_EINVAL, "regress_alive: call once before capturing so that the scratch exists");
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        if (s.alive_cap < need) {
            cudaFree(s.d_alive);
            s.d_alive = nullptr;
            s.alive_cap = 0;
            if (cudaMalloc(&s.d_alive, need * sizeof(double)) != cudaSuccess)
                return fail(CVA_ENOMEM, "regress_alive: scratch allocation failed");
            s.alive_cap = need;
        }
        if (s.alive_stats_cap < need_stats) {
            cudaFree(s.d_alive_stats);
            s.d_alive_stats = nullptr;
            s.alive_stats_cap = 0;
            if (cudaMalloc(&s.d_alive_stats, need_stats * sizeof(float)) != cudaSuccess)
                return fail(CVA_ENOMEM, "regress_alive: statistics allocation failed");
            s.alive_stats_cap = need_stats;
        }
    }
    AliveArgs a;
    a.M = (uint32_t)M;
    a.N = s.N;
    a.n = s.n;
    a.F = s.F;
    a.C = C;
    a.mY = mY;
    a.NS = NS;
    a.idx = s.d_idx;
    a.expo = s.d_expo + (size_t)pf * (s.n + 1) * C * M;
    a.disc = s.d_disc;
    a.feat = s.d_features;
    a.targ = s.d_targets + (size_t)pf * s.n * M;
    a.stats = s.d_alive_stats;
    a.chunks = (int)chunks;
    a.rows_per_chunk = (uint32_t)((M + chunks - 1) / chunks);
    a.NA = NA;
    a.NBf = NBf;
    a.NB = NB;
    a.RS = RS;
    a.part = s.d_alive;
    a.coef = a.part + (size_t)groups * chunks * NBLK * 16;
    a.coef_raw = a.coef + (size_t)groups * m;
    a.status = reinterpret_cast<int *>(a.coef_raw + (size_t)groups * m);
    a.pred = pred_dev;
    cva_status r = (C == 2) ? launch_stats<2>(a, st) : launch_stats<8>(a, st);
    if (r != CVA_OK) return r;
    const size_t tile_bytes = (size_t)kTileRows * RS * sizeof(float);
    const size_t red_bytes = (size_t)(kGramThreads / NBLK) * NBLK * 16 * sizeof(double);
    const size_t gsmem = tile_bytes > red_bytes ? tile_bytes : red_bytes;
    CVA_CUDA_TRY(cudaFuncSetAttribute(alive_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem));
    alive_gram_kernel<<<dim3((unsigned)chunks, (unsigned)groups), kGramThreads, gsmem, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    alive_solve_kernel<<<groups, 128, 0, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    if (pred_dev) {
        alive_predict_kernel<<<dim3((unsigned)((M + 255) / 256), (unsigned)groups), 256, 0, st>>>(a);
        CVA_CUDA_TRY(cudaGetLastError());
    }
    if (coef_host || dropped_host) {
        std::vector<double> cr((size_t)groups * m);
        std::vector<int> status(groups);
        CVA_CUDA_TRY(cudaMemcpyAsync(cr.data(), a.coef_raw, sizeof(double) * cr.size(), cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaMemcpyAsync(status.data(), a.status, sizeof(int) * groups, cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        if (coef_host)
            for (int g = 0; g < groups; ++g)
                for (int c = 0; c < m; ++c) coef_host[(size_t)(g + 1) * m + c] = cr[(size_t)g * m + c];
        if (dropped_host) {
            dropped_host[0] = 0;
            for (int g = 0; g < groups; ++g) dropped_host[g + 1] = status[g];
        }
    }
    return CVA_OK;
}

}  // namespace cva
