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
// and N xi_bar^k for the right-hand side of Y. P_cd and q_c enter only through their
// sums over the paths, d_c also through its products with Y.
//
// alive_stats_kernel walks the dates of a path once (a warp per path, lanes over the
// draws, work only at the draws' default steps), stores d_c per path and the sums of
// P_cd and q_c over its block's paths. alive_gram_kernel accumulates
// sum_k [1, Y - Y^0]^T [1, Y - Y^0, d, xi_bar] in FP32 runs of 512 rows per thread,
// then FP64, reduced in a fixed order (tiles staged by cp.async, two buffers), and
// adds up the P_cd and q_c block sums of its rows. alive_solve_kernel adds the chunks,
// assembles the (1 + F + C)-square system and solves it by a Jacobi-scaled Cholesky
// factorisation in FP64, dropping a column whose pivot vanishes (a counterparty with
// no default by t_i anywhere in the sample).
#include <math.h>

#include "cva_internal.h"

namespace cva {

namespace {

constexpr int kGramThreads = 288;   // 70 blocks of 4x4 at the 27-factor, 8-counterparty shape, four row groups
constexpr int kTileRows = 128;
constexpr int kMaxUnknowns = 40;    // 1 + F + C
constexpr int kMaxAug = 44;         // [1, Y - Y^0, d, xi_bar], padded to 4
constexpr int kStatWarps = 8;       // paths per block of the statistics kernel (stage rows are 8 wide)
constexpr int kStatBudget = 160 * 1024;
constexpr int kSolveThreads = 128;

template <int C>
struct Shape {
    static constexpr int NP = C * (C - 1) / 2;    // pairs c < d
    static constexpr int NQ = NP + C;             // block-summed statistics: P_cd, q_c
    static_assert(C >= 1 && C <= 8 && NP <= 32, "one lane per counterparty pair: at most 8 counterparties");
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
    } else if constexpr (C == 2) {
        const unsigned short v = *reinterpret_cast<const unsigned short *>(jp);
        const float2 a = *reinterpret_cast<const float2 *>(ep);
        j[0] = v & 255u;
        j[1] = v >> 8;
        e[0] = a.x; e[1] = a.y;
    } else {   // other counts: byte and float loads
#pragma unroll
        for (int c = 0; c < C; ++c) {
            j[c] = jp[c];
            e[c] = ep[c];
        }
    }
}

struct AliveArgs {
    uint32_t M, N;
    int n, F, C, mY, NQ;
    const uint8_t *idx;       // [M][N][C] default steps, n+1 = none
    const float *expo;        // [n+1][C][M] of the portfolio
    const float *disc;        // [n+1][M]
    const float *feat;        // [n+1][F][M]
    const float *targ;        // [n][M] of the portfolio
    float *dstat;             // [n][C][M] d_c per path
    float *qsum;              // [n][NQ][nblk] P_cd, q_c summed over a statistics block's paths
    uint32_t nblk;            // blocks of the statistics kernel
    int chunks;
    uint32_t rows_per_chunk;
    int NA, NB, RS;           // Gram: NA x NB blocks of 4x4, tile row stride
    double *part;             // [n-1][chunks][NA*NB*16 + NQ]: Gram blocks, then the chunk's P_cd, q_c sums
    int W;                    // paths per statistics block (a power of two)
    double *coef;             // [n-1][1+F+C] centred basis
    double *coef_raw;         // [n-1][1+F+C] raw basis
    int *status;              // [n-1] dropped columns
    float *pred;              // [n][M] or null
};

// Shared-memory layout of the statistics kernel: the float tables of the W warps,
// rounded up to 16 bytes, the byte tables (8-byte aligned for every warp), rounded
// up to 16 bytes, then the two stage buffers.
__host__ __device__ inline size_t stats_float_bytes(int W, uint32_t N, int C)
{
    return ((size_t)W * N * (C + 1) * sizeof(float) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t stats_stage_offset(int W, uint32_t N, int C)
{
    return (stats_float_bytes(W, N, C) + (size_t)W * N * (C + 2) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t stats_stage_floats(int C)
{
    return 2 * (size_t)(2 * C + C * (C - 1) / 2) * kStatWarps;   // [2][d, P, q][8 paths]
}

// One warp per path, lanes over the draws; the dates are walked in order and only
// the draws with a default at date i change. A draw keeps its defaulted mask, its
// later losses and its next default step; when it moves from (x, f) to (x', f') the
// warp applies d_c += x'_c - x_c, P_cd += x'_c x'_d - x_c x_d (lane p owns pair p) and
// q_c += x'_c f' - x_c f (lane c owns d_c and q_c), in lane order. The counts are
// exact; f' is recomputed from the draw's table at each of its events. Each date's
// values go through shared memory: d_c leaves as 8-path rows (one 32-byte sector),
// P_cd and q_c as the sum over the block's paths.
template <int C>
__global__ void __launch_bounds__(kStatWarps * 32) alive_stats_kernel(AliveArgs a)
{
    using S = Shape<C>;
    constexpr int NS = C + S::NQ;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const uint32_t N = a.N, M = a.M;
    const int n = a.n;
    const size_t fb = stats_float_bytes(W, N, C);
    float *e_s = reinterpret_cast<float *>(smem) + (size_t)warp * N * C;                   // [N][C] loss at the default step
    float *f_s = reinterpret_cast<float *>(smem) + (size_t)W * N * C + (size_t)warp * N;   // [N] losses after the date
    uint8_t *j_s = smem + fb + (size_t)warp * N * C;                                       // [N][C] default steps
    uint8_t *x_s = smem + fb + (size_t)W * N * C + (size_t)warp * N * 2;                   // [N][2] mask, next step
    float *stage0 = reinterpret_cast<float *>(smem + stats_stage_offset(W, N, C));         // [2][NS][8]
    const uint32_t kl0 = blockIdx.x * (uint32_t)W, kl = kl0 + warp;
    const bool live = kl < M;
    if (live) {
        const uint8_t *src = a.idx + (size_t)kl * N * C;
        if ((N * C) % 16 == 0) {
            // 16 steps per lane, then their 16 independent gathers
            for (uint32_t seg = lane; seg < N * C / 16; seg += 32) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src) + seg);
                *reinterpret_cast<uint4 *>(j_s + (size_t)seg * 16) = v;
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    const int j = (w4[b >> 2] >> (8 * (b & 3))) & 255u;
                    const uint32_t e = seg * 16 + b;
                    e_s[e] = (j <= n) ? __ldg(a.expo + ((size_t)j * C + (e % C)) * M + kl) : 0.f;
                }
            }
        } else {
            for (uint32_t e = lane; e < N * C; e += 32) {
                const int j = src[e];
                j_s[e] = (uint8_t)j;
                e_s[e] = (j <= n) ? __ldg(a.expo + ((size_t)j * C + e % C) * M + kl) : 0.f;
            }
        }
        __syncwarp();
        for (uint32_t l = lane; l < N; l += 32) {
            int j[C];
            float e[C];
            load_draw<C>(j_s + (size_t)l * C, e_s + (size_t)l * C, j, e);
            float fut = 0.f;
            int nx = 255;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                fut += e[c];
                nx = min(nx, j[c]);
            }
            f_s[l] = fut;
            x_s[2 * l] = 0;
            x_s[2 * l + 1] = (uint8_t)nx;
        }
        __syncwarp();
    }
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
    uint32_t dcount = 0u, pcount = 0u;  // lane c: d_c; lane p: P_p
    float qsum = 0.f;                   // lane c: q_c before the discount factor
    float dnext = (live && lane < C) ? __ldg(a.disc + (size_t)1 * M + kl) : 0.f;
    for (int i = 1; i < n; ++i) {
        const float dcur = dnext;
        if (live && lane < C && i + 1 < n) dnext = __ldg(a.disc + (size_t)(i + 1) * M + kl);
        float *stage = stage0 + (i & 1) * NS * kStatWarps;
        if (live) {
            for (uint32_t l0 = 0; l0 < N; l0 += 32) {
                const uint32_t l = l0 + lane;
                const bool has = l < N && (int)x_s[2 * l + 1] == i;
                uint32_t m = __ballot_sync(0xffffffffu, has);
                if (m == 0u) continue;
                uint32_t xo = 0u, xn = 0u;
                float fo = 0.f, fn = 0.f;
                if (has) {
                    int j[C];
                    float e[C];
                    load_draw<C>(j_s + (size_t)l * C, e_s + (size_t)l * C, j, e);
                    xo = x_s[2 * l];
                    fo = f_s[l];
                    int nx = 255;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (j[c] <= i) {
                            xn |= 1u << c;
                        } else {
                            fn += e[c];
                            nx = min(nx, j[c]);
                        }
                    }
                    x_s[2 * l] = (uint8_t)xn;
                    x_s[2 * l + 1] = (uint8_t)nx;
                    f_s[l] = fn;
                }
                while (m) {
                    const int s = __ffs(m) - 1;
                    m &= m - 1u;
                    const uint32_t bxo = __shfl_sync(0xffffffffu, xo, s), bxn = __shfl_sync(0xffffffffu, xn, s);
                    const float bfo = __shfl_sync(0xffffffffu, fo, s), bfn = __shfl_sync(0xffffffffu, fn, s);
                    const uint32_t now = (bxn >> lane) & 1u, before = (bxo >> lane) & 1u;
                    dcount += now - before;
                    qsum += (now ? bfn : 0.f) - (before ? bfo : 0.f);
                    pcount += ((bxn >> cA) & (bxn >> cB) & 1u) - ((bxo >> cA) & (bxo >> cB) & 1u);
                }
            }
            if (lane < C) {
                stage[lane * kStatWarps + warp] = (float)dcount;
                stage[(C + S::NP + lane) * kStatWarps + warp] = qsum * expf(dcur);
            }
            if (lane < S::NP) stage[(C + lane) * kStatWarps + warp] = (float)pcount;
        }
        __syncthreads();        // the stage of date i is complete; the other buffer is free
        for (int t = tid; t < C * kStatWarps + S::NQ; t += blockDim.x) {
            if (t < C * kStatWarps) {
                const int c = t >> 3, w = t & 7;
                if (w < W && kl0 + w < M) a.dstat[((size_t)i * C + c) * M + kl0 + w] = stage[c * kStatWarps + w];
            } else {
                const int q = t - C * kStatWarps;
                float s = 0.f;
                for (int w = 0; w < W; ++w)
                    if (kl0 + w < M) s += stage[(C + q) * kStatWarps + w];
                a.qsum[((size_t)i * S::NQ + q) * a.nblk + blockIdx.x] = s;
            }
        }
    }
}

// The array feeding augmented column `col` (1 <= col <= F + C + 1) of the Gram tile at
// date i: the state Y (F), then d_c (C), then xi_bar; column 0 is the constant 1.
__device__ __forceinline__ const float *column_source(const AliveArgs &a, const float *feat, const float *dstat,
                                                      const float *targ, int col)
{
    const int mY = a.mY, C = a.C;
    if (col < mY) return feat + (size_t)(col - 1) * a.M;
    if (col < mY + C) return dstat + (size_t)(col - mY) * a.M;
    return targ;
}

__device__ __forceinline__ void cp_async4_zfill(uint32_t saddr, const void *g, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(g), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_groups() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// sum over paths of [1, Y - Y^0]^T [1, Y - Y^0, d, xi_bar] at date i = g + 1. Tiles of
// 128 rows are copied by cp.async into two buffers: the copies of the next tile run
// during the products of the current one. After a tile lands, the state columns are
// centred on path 0 in place and the constant column is set (0 on rows past the end).
__global__ void __launch_bounds__(kGramThreads, 2) alive_gram_kernel(AliveArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int NB = a.NB, RS = a.RS, TS = kTileRows * a.RS;
    float *tiles = reinterpret_cast<float *>(smem);           // [2][kTileRows][RS]
    const int g = blockIdx.y, i = g + 1, chunk = blockIdx.x, tid = threadIdx.x;
    const uint32_t M = a.M;
    const float *feat = a.feat + (size_t)i * a.F * M;
    const float *dstat = a.dstat + (size_t)i * a.C * M;
    const float *targ = a.targ + (size_t)i * M;
    const uint32_t r_begin = (uint32_t)chunk * a.rows_per_chunk;
    const uint32_t r_end = min(M, r_begin + a.rows_per_chunk);
    const int NBLK = a.NA * NB, NRG = kGramThreads / NBLK;
    const int b = tid % NBLK, rg = tid / NBLK, bi = b / NB, bj = b % NB;
    const int mY = a.mY, nload = a.F + a.C + 1;              // copied columns 1..nload: Y, d, xi_bar
    __shared__ const float *csrc[kMaxAug];
    __shared__ float c0[kMaxUnknowns];
    for (int f = tid; f < a.F; f += kGramThreads) c0[f] = __ldg(feat + (size_t)f * M);
    __syncthreads();
    for (int lc = tid; lc < nload; lc += kGramThreads) csrc[lc] = column_source(a, feat, dstat, targ, lc + 1);
    for (int e = tid; e < 2 * kTileRows; e += kGramThreads)   // padding columns stay zero
        for (int c = nload + 1; c < 4 * NB; ++c) tiles[e * RS + c] = 0.f;
    __syncthreads();
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tiles);
    auto issue = [&](uint32_t r0, int buf) {
        for (int e = tid; e < nload * kTileRows; e += kGramThreads) {
            const int lc = e / kTileRows, r = e % kTileRows;
            const uint32_t k = r0 + r;
            const bool ok = k < r_end;
            cp_async4_zfill(sbase + (uint32_t)(buf * TS + r * RS + 1 + lc) * 4u, csrc[lc] + (ok ? k : 0u), ok);
        }
        cp_async_commit_group();
    };
    double dacc[16];
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        dacc[e] = 0.0;
        acc[e] = 0.f;
    }
    int since_flush = 0;
    if (r_begin < r_end) issue(r_begin, 0);
    // the chunk's share of the P_cd and q_c sums: the statistics blocks of its rows
    // (chunks start at multiples of 128 rows, W divides 128), 8 threads per column
    double pq = 0.0;
    {
        const int q = tid >> 3, sub = tid & 7;
        const uint32_t bk0 = r_begin / a.W, bk1 = min(a.nblk, (r_end + a.W - 1) / a.W);
        if (q < a.NQ && r_begin < r_end) {
            const float *src = a.qsum + ((size_t)i * a.NQ + q) * a.nblk;
#pragma unroll 4
            for (uint32_t bk = bk0 + sub; bk < bk1; bk += 8) pq += (double)__ldg(src + bk);
        }
        pq += __shfl_xor_sync(0xffffffffu, pq, 4);
        pq += __shfl_xor_sync(0xffffffffu, pq, 2);
        pq += __shfl_xor_sync(0xffffffffu, pq, 1);
    }
    int buf = 0;
    for (uint32_t r0 = r_begin; r0 < r_end; r0 += kTileRows, buf ^= 1) {
        cp_async_wait_groups();
        __syncthreads();                          // tile r0 is in buffer buf; buf ^ 1 is free
        float *tile = tiles + buf * TS;
        for (int e = tid; e < mY * kTileRows; e += kGramThreads) {
            const int col = e / kTileRows, r = e % kTileRows;
            const bool ok = r0 + r < r_end;
            float *v = tile + r * RS + col;
            if (col == 0) *v = ok ? 1.f : 0.f;
            else if (ok) *v -= c0[col - 1];
        }
        __syncthreads();
        if (r0 + kTileRows < r_end) issue(r0 + kTileRows, buf ^ 1);
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
    double *out = a.part + ((size_t)g * a.chunks + chunk) * (NBLK * 16 + a.NQ);
    for (int e = tid; e < NBLK * 16; e += kGramThreads) {
        double s = 0.0;
        for (int q = 0; q < NRG; ++q) s += red[(size_t)q * NBLK * 16 + e];
        out[e] = s;
    }
    if ((tid & 7) == 0 && (tid >> 3) < a.NQ) out[NBLK * 16 + (tid >> 3)] = pq;
}

__global__ void __launch_bounds__(kSolveThreads) alive_solve_kernel(AliveArgs a)
{
    constexpr int MX = kMaxUnknowns;
    __shared__ double R[(MX / 4) * (kMaxAug / 4) * 16];
    __shared__ double A[MX * MX];
    __shared__ double rhs[MX];
    __shared__ double PQ[32 + 8];                 // sums over paths of P_cd, then q_c
    const int g = blockIdx.x, tid = threadIdx.x, i = g + 1;
    const int NB = a.NB, NBLK = a.NA * NB, mY = a.mY, C = a.C, m = mY + C, NQ = a.NQ;
    const int NP = C * (C - 1) / 2, PS = NBLK * 16 + NQ;
    for (int e = tid; e < PS; e += blockDim.x) {
        double s = 0.0;
        const double *p = a.part + (size_t)g * a.chunks * PS + e;
        for (int c = 0; c < a.chunks; ++c) s += p[(size_t)c * PS];
        if (e < NBLK * 16) R[e] = s;
        else PQ[e - NBLK * 16] = s;
    }
    __syncthreads();
    // R(p, q): row p of [1, Y - Y^0], augmented column q
    auto Rv = [&](int p, int q) -> double { return R[((p / 4) * NB + q / 4) * 16 + (p % 4) * 4 + (q % 4)]; };
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
                const double v = PQ[c * (2 * C - c - 1) / 2 + (d - c - 1)];
                A[(mY + c) * MX + mY + d] = v;
                A[(mY + d) * MX + mY + c] = v;
            }
            rhs[mY + c] = PQ[NP + c];
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

size_t stats_smem(int W, uint32_t N, int C)
{
    return stats_stage_offset(W, N, C) + stats_stage_floats(C) * sizeof(float);
}

// warps (paths) per block of the statistics kernel for N draws of C counterparties: a
// power of two, so that the Gram chunks (multiples of 128 rows) hold whole blocks
int stats_warps(uint32_t N, int C)
{
    for (int W = kStatWarps; W >= 1; W >>= 1)
        if (stats_smem(W, N, C) <= (size_t)kStatBudget) return W;
    return 0;
}

// The dynamic shared memory limits are raised outside stream capture: the first call,
// which also allocates the scratch, sets them before any capture.
template <int C>
cva_status launch_stats(const AliveArgs &a, int W, bool capturing, cudaStream_t st)
{
    const size_t smem = stats_smem(W, a.N, C);
    if (!capturing)
        CVA_CUDA_TRY(cudaFuncSetAttribute(alive_stats_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    alive_stats_kernel<C><<<a.nblk, 32 * W, smem, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

}  // namespace

cva_status alive_regress(Sim &s, int pf, float *pred_dev, double *coef_host, int *dropped_host, cudaStream_t st)
{
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "regress_alive: portfolio index out of range");
    if (s.n < 2) return fail(CVA_EINVAL, "regress_alive: need at least two pricing steps");
    if (!s.d_idx) return fail(CVA_EINVAL, "regress_alive: the simulation keeps no default steps (CVA_KEEP_DEFAULTS)");
    if (s.C < 1 || s.C > 8) return fail(CVA_ENOTSUP, "regress_alive: at most 8 counterparties");
    if (s.M > 0x7fffffffull) return fail(CVA_EINVAL, "regress_alive: M too large");
    const int C = s.C, NQ = C * (C - 1) / 2 + C, mY = s.F + 1, m = mY + C;
    if (m > kMaxUnknowns) return fail(CVA_ENOTSUP, "regress_alive: 1 + F + C must be <= 40");
    const int W = stats_warps(s.N, C);
    if (W < 1) return fail(CVA_ENOTSUP, "regress_alive: N * C too large for the per-path draw tables");
    // Gram columns: [1, Y - Y^0] (mY), d (C), xi_bar, zero padding to 4 NB
    const int NA = (mY + 3) / 4, NB = (mY + C + 1 + 3) / 4;
    const int RS = (NB & 1) ? 4 * NB : 4 * NB + 4;   // a row stride of 4 x odd floats: column stores hit 8 banks
    if (4 * NB > kMaxAug) return fail(CVA_ENOTSUP, "regress_alive: too many Gram columns");
    if (NA * NB > kGramThreads) return fail(CVA_ENOTSUP, "regress_alive: Gram blocks exceed the block size");
    const size_t M = s.M;
    const uint32_t nblk = (uint32_t)((M + W - 1) / W);
    const int groups = s.n - 1;
    uint64_t chunks = ((uint64_t)(s.tune_lsq_chunks > 0 ? s.tune_lsq_chunks : 2432) + groups - 1) / groups;
    const uint64_t max_chunks = (M + 1023) / 1024;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const size_t NBLK = (size_t)NA * NB;
    const uint64_t rows_per_chunk = ((M + chunks - 1) / chunks + kTileRows - 1) / kTileRows * kTileRows;
    const size_t need = (size_t)groups * chunks * (NBLK * 16 + NQ) + 2 * (size_t)groups * m + (size_t)groups;
    const size_t need_stats = (size_t)s.n * C * M + (size_t)s.n * NQ * nblk;
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
    a.NQ = NQ;
    a.idx = s.d_idx;
    a.expo = s.d_expo + (size_t)pf * (s.n + 1) * C * M;
    a.disc = s.d_disc;
    a.feat = s.d_features;
    a.targ = s.d_targets + (size_t)pf * s.n * M;
    a.dstat = s.d_alive_stats;
    a.qsum = s.d_alive_stats + (size_t)s.n * C * M;
    a.nblk = nblk;
    a.chunks = (int)chunks;
    a.rows_per_chunk = (uint32_t)rows_per_chunk;
    a.W = W;
    a.NA = NA;
    a.NB = NB;
    a.RS = RS;
    a.part = s.d_alive;
    a.coef = a.part + (size_t)groups * chunks * (NBLK * 16 + NQ);
    a.coef_raw = a.coef + (size_t)groups * m;
    a.status = reinterpret_cast<int *>(a.coef_raw + (size_t)groups * m);
    a.pred = pred_dev;
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    static constexpr cva_status (*by_c[8])(const AliveArgs &, int, bool, cudaStream_t) = {
        launch_stats<1>, launch_stats<2>, launch_stats<3>, launch_stats<4>,
        launch_stats<5>, launch_stats<6>, launch_stats<7>, launch_stats<8>};
    cva_status r = by_c[C - 1](a, W, capturing, st);
    if (r != CVA_OK) return r;
    const size_t tile_bytes = 2 * (size_t)kTileRows * RS * sizeof(float);
    const size_t red_bytes = (size_t)(kGramThreads / NBLK) * NBLK * 16 * sizeof(double);
    const size_t gsmem = tile_bytes > red_bytes ? tile_bytes : red_bytes;
    if (!capturing)
        CVA_CUDA_TRY(cudaFuncSetAttribute(alive_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem));
    alive_gram_kernel<<<dim3((unsigned)chunks, (unsigned)groups), kGramThreads, gsmem, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    alive_solve_kernel<<<groups, kSolveThreads, 0, st>>>(a);
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
