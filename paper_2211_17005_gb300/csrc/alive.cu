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
// (a warp per path, lanes over draws; integer counts in 16-bit fields reduced with
// redux.sync, so they are exact; the q_c butterfly has a fixed order).
// alive_gram_kernel accumulates sum_k [1, Y - Y^0]^T [1, Y - Y^0, stats, xi_bar]
// (FP32 runs of 512 rows per thread, then FP64, reduced in a fixed order), and
// alive_solve_kernel assembles the (1 + F + C)-square system and solves it by a
// Jacobi-scaled Cholesky factorisation in FP64, dropping a column whose pivot
// vanishes (a counterparty with no default by t_i anywhere in the sample).
#include <math.h>

#include "cva_internal.h"

namespace cva {

namespace {

constexpr int kGramThreads = 288;   // 133 blocks of 4x4 at the 27-factor, 8-counterparty shape, two row groups
constexpr int kTileRows = 128;
constexpr int kMaxUnknowns = 40;    // 1 + F + C
constexpr int kMaxAug = 80;         // 1 + F + statistics + target, padded to 4
constexpr int kStatBudget = 160 * 1024;

template <int C>
struct Shape {
    static constexpr int NP = C * (C - 1) / 2;    // pairs c < d
    static constexpr int NS = 2 * C + NP;         // statistics per (path, date)
    static constexpr int NW = (C + NP + 1) / 2;   // words of 16-bit count fields
};

struct AliveArgs {
    uint32_t M, N;
    int n, F, C, mY, NS;
    const uint8_t *idx;       // [M][N][C] default steps, n+1 = none
    const float *expo;        // [n+1][C][M] of the portfolio
    const float *disc;        // [n+1][M]
    const float *feat;        // [n+1][F][M]
    const float *targ;        // [n][M] of the portfolio
    float *stats;             // [n][NS][M]
    int chunks;
    uint32_t rows_per_chunk;
    int NA, NB;               // 4-column blocks: rows (1 + F) x columns (augmented)
    double *part;             // [n-1][chunks][NA*NB*16]
    double *coef;             // [n-1][1+F+C] centred basis
    double *coef_raw;         // [n-1][1+F+C] raw basis
    int *status;              // [n-1] dropped columns
    float *pred;              // [n][M] or null
};

template <int C>
__global__ void __launch_bounds__(256) alive_stats_kernel(AliveArgs a)
{
    using S = Shape<C>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t N = a.N, M = a.M;
    const int n = a.n;
    float *stage0 = reinterpret_cast<float *>(smem);                          // [2][NS][W]
    float *e_s = stage0 + 2 * S::NS * W + (size_t)warp * N * C;               // [C][N] loss at the default step
    uint8_t *j_s = reinterpret_cast<uint8_t *>(stage0 + 2 * S::NS * W + (size_t)W * N * C) + (size_t)warp * N * C;
    const uint32_t kl0 = blockIdx.x * (uint32_t)W, kl = kl0 + warp;
    const bool live = kl < M;
    if (live) {
        const uint8_t *src = a.idx + (size_t)kl * N * C;
        for (uint32_t e = lane; e < N * C; e += 32) {
            const uint32_t l = e / C, c = e % C;
            const int j = src[e];
            j_s[c * N + l] = (uint8_t)j;
            e_s[c * N + l] = (j <= n) ? __ldg(a.expo + ((size_t)j * C + c) * M + kl) : 0.f;
        }
    }
    __syncwarp();
    for (int i = 1; i < n; ++i) {
        float *stage = stage0 + (i & 1) * S::NS * W;
        if (live) {
            uint32_t cnt[S::NW];
            float q[C];
#pragma unroll
            for (int w = 0; w < S::NW; ++w) cnt[w] = 0u;
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] = 0.f;
            for (uint32_t l = lane; l < N; l += 32) {
                uint32_t x = 0u;     // bit c: counterparty c has defaulted by t_i
                float fut = 0.f;     // the draw's losses after t_i, discounted to 0
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if ((int)j_s[c * N + l] <= i) x |= 1u << c;
                    else fut += e_s[c * N + l];
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if ((x >> c) & 1u) q[c] += fut;
                    cnt[c >> 1] += ((x >> c) & 1u) << (16 * (c & 1));
                }
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int d = c + 1; d < C; ++d) {
                        const int p = C + c * (2 * C - c - 1) / 2 + (d - c - 1);
                        cnt[p >> 1] += ((x >> c) & (x >> d) & 1u) << (16 * (p & 1));
                    }
            }
#pragma unroll
            for (int w = 0; w < S::NW; ++w) cnt[w] = __reduce_add_sync(0xffffffffu, cnt[w]);
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) q[c] += __shfl_xor_sync(0xffffffffu, q[c], off);
            if (lane == 0) {
                const float binv = expf(__ldg(a.disc + (size_t)i * M + kl));
#pragma unroll
                for (int p = 0; p < C + S::NP; ++p)
                    stage[p * W + warp] = (float)((cnt[p >> 1] >> (16 * (p & 1))) & 0xffffu);
#pragma unroll
                for (int c = 0; c < C; ++c) stage[(C + S::NP + c) * W + warp] = q[c] * binv;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < S::NS * W; e += blockDim.x) {
            const int s = e / W, w = e % W;
            if (kl0 + w < M) a.stats[((size_t)i * S::NS + s) * M + kl0 + w] = stage[s * W + w];
        }
    }
}

// sum over paths of [1, Y - Y^0]^T [1, Y - Y^0, statistics, xi_bar] at date i = g + 1
__global__ void __launch_bounds__(kGramThreads) alive_gram_kernel(AliveArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int NA = a.NA, NB = a.NB, RS = 4 * NB + 4;
    float *tile = reinterpret_cast<float *>(smem);            // [kTileRows][RS]
    const int g = blockIdx.y, i = g + 1, chunk = blockIdx.x, tid = threadIdx.x;
    const uint32_t M = a.M;
    const int mY = a.mY, NS = a.NS, MB = mY + NS + 1;
    const float *feat = a.feat + (size_t)i * a.F * M;
    const float *stats = a.stats + (size_t)i * NS * M;
    const float *targ = a.targ + (size_t)i * M;
    const uint32_t r_begin = (uint32_t)chunk * a.rows_per_chunk;
    const uint32_t r_end = min(M, r_begin + a.rows_per_chunk);
    const int NBLK = NA * NB, NRG = kGramThreads / NBLK;
    const int b = tid % NBLK, rg = tid / NBLK, bi = b / NB, bj = b % NB;
    __shared__ float c0[kMaxUnknowns];
    for (int f = tid; f < a.F; f += kGramThreads) c0[f] = __ldg(feat + (size_t)f * M);
    double dacc[16];
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        dacc[e] = 0.0;
        acc[e] = 0.f;
    }
    int since_flush = 0;
    for (uint32_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
        __syncthreads();
        for (int e = tid; e < 4 * NB * kTileRows; e += kGramThreads) {
            const int col = e / kTileRows, r = e % kTileRows;
            const uint32_t k = r0 + r;
            float v = 0.f;
            if (col < MB && k < r_end) {
                if (col == 0) v = 1.f;
                else if (col < mY) v = __ldg(feat + (size_t)(col - 1) * M + k) - c0[col - 1];
                else if (col < mY + NS) v = __ldg(stats + (size_t)(col - mY) * M + k);
                else v = __ldg(targ + k);
            }
            tile[r * RS + col] = v;
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
    const int NBLK = a.NA * a.NB, NB = a.NB, mY = a.mY, C = a.C, NS = a.NS, m = mY + C;
    const int NP = C * (C - 1) / 2;
    for (int e = tid; e < NBLK * 16; e += blockDim.x) {
        double s = 0.0;
        const double *p = a.part + (size_t)g * a.chunks * NBLK * 16 + e;
        for (int c = 0; c < a.chunks; ++c) s += p[(size_t)c * NBLK * 16];
        R[e] = s;
    }
    __syncthreads();
    if (tid != 0) return;
    // R(p, q): row p of [1, Y - Y^0], column q of the augmented row
    auto Rv = [&](int p, int q) -> double {
        return R[((p / 4) * NB + q / 4) * 16 + (p % 4) * 4 + (q % 4)];
    };
    const double Nd = (double)a.N;
    for (int p = 0; p < mY; ++p) {
        for (int q = 0; q < mY; ++q) A[p * MX + q] = Nd * Rv(p, q);
        for (int c = 0; c < C; ++c) {
            A[p * MX + mY + c] = Rv(p, mY + c);
            A[(mY + c) * MX + p] = Rv(p, mY + c);
        }
        rhs[p] = Nd * Rv(p, mY + NS);
    }
    for (int c = 0; c < C; ++c) {
        A[(mY + c) * MX + mY + c] = Rv(0, mY + c);
        for (int d = c + 1; d < C; ++d) {
            const double v = Rv(0, mY + C + c * (2 * C - c - 1) / 2 + (d - c - 1));
            A[(mY + c) * MX + mY + d] = v;
            A[(mY + d) * MX + mY + c] = v;
        }
        rhs[mY + c] = Rv(0, mY + C + NP + c);
    }
    // Jacobi scaling, Cholesky of the scaled matrix, columns with a vanishing pivot dropped
    double sc[MX], L[MX * MX], y[MX], w[MX];
    bool drop[MX];
    for (int r = 0; r < m; ++r) {
        const double d = A[r * MX + r];
        drop[r] = !(d > 0.0);
        sc[r] = drop[r] ? 0.0 : 1.0 / sqrt(d);
    }
    int dropped = 0;
    for (int r = 0; r < m; ++r) {
        for (int c = 0; c <= r; ++c) {
            double s = (drop[r] || drop[c]) ? 0.0 : A[r * MX + c] * sc[r] * sc[c];
            for (int p = 0; p < c; ++p) s -= L[r * MX + p] * L[c * MX + p];
            if (r == c) {
                if (drop[r] || !(s > 1e-12)) {
                    drop[r] = true;
                    L[r * MX + r] = 1.0;
                    for (int p = 0; p < r; ++p) L[r * MX + p] = 0.0;
                    ++dropped;
                } else {
                    L[r * MX + r] = sqrt(s);
                }
            } else {
                L[r * MX + c] = drop[r] ? 0.0 : s / L[c * MX + c];
            }
        }
    }
    for (int r = 0; r < m; ++r) {                 // L y = D^{-1/2} b
        double s = drop[r] ? 0.0 : rhs[r] * sc[r];
        for (int p = 0; p < r; ++p) s -= L[r * MX + p] * y[p];
        y[r] = drop[r] ? 0.0 : s / L[r * MX + r];
    }
    for (int r = m - 1; r >= 0; --r) {            // L^T z = y, w = D^{-1/2} z
        double s = y[r];
        for (int p = r + 1; p < m; ++p) s -= L[p * MX + r] * w[p];
        w[r] = drop[r] ? 0.0 : s / L[r * MX + r];
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
    const size_t per_warp = (size_t)a.N * C * (sizeof(float) + 1) + 2 * S::NS * sizeof(float);
    int W = (int)(kStatBudget / per_warp);
    if (W > 8) W = 8;
    if (W < 1) return fail(CVA_ENOTSUP, "regress_alive: N * C too large for the per-path draw tables");
    const size_t smem = 2 * (size_t)S::NS * W * sizeof(float) + (size_t)W * a.N * C * (sizeof(float) + 1);
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
    const int MB = mY + NS + 1, NA = (mY + 3) / 4, NB = (MB + 3) / 4;
    if (4 * NB > kMaxAug) return fail(CVA_ENOTSUP, "regress_alive: too many statistics columns");
    if (NA * NB > kGramThreads) return fail(CVA_ENOTSUP, "regress_alive: Gram blocks exceed the block size");
    const size_t M = s.M;
    const int groups = s.n - 1;
    uint64_t chunks = ((uint64_t)(s.tune_lsq_chunks > 0 ? s.tune_lsq_chunks : 2432) + groups - 1) / groups;
    const uint64_t max_chunks = (M + 1023) / 1024;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const size_t NBLK = (size_t)NA * NB;
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
    a.NB = NB;
    a.part = s.d_alive;
    a.coef = a.part + (size_t)groups * chunks * NBLK * 16;
    a.coef_raw = a.coef + (size_t)groups * m;
    a.status = reinterpret_cast<int *>(a.coef_raw + (size_t)groups * m);
    a.pred = pred_dev;
    cva_status r = (C == 2) ? launch_stats<2>(a, st) : launch_stats<8>(a, st);
    if (r != CVA_OK) return r;
    const size_t tile_bytes = (size_t)kTileRows * (4 * NB + 4) * sizeof(float);
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
