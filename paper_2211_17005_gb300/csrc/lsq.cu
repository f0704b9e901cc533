// Grouped least-squares regression of eq. (e:forw), one group per pricing date:
//   w = argmin_w sum_k (xi_k - w^T phi(Y_k))^2.
// The augmented Gram matrix [phi, xi]^T [phi, xi] of the basis centred on path
// 0's state is accumulated from FP32 products in FP32 runs of 512 rows per thread,
// then in FP64 (per thread, per block, then across blocks in a fixed order), and
// solved by a Jacobi-scaled Cholesky factorisation in FP64. The pass over the
// features and targets is the only HBM traffic: every byte is read once. For the
// linear basis the tiles are copied by cp.async into two buffers (lsq_gram_async).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "cva_internal.h"

namespace cva {

namespace {

constexpr int kGramThreads = 256;

struct LsqArgs {
    const float *feat0;
    size_t feat_stride;   // floats between groups' feature blocks ([F][M] each)
    const float *targ0;
    size_t targ_stride;   // floats between groups' targets
    float *pred0;
    size_t pred_stride;
    int F, m, basis, chunks;
    uint32_t M, rows_per_chunk;
    double *part;         // [groups][chunks][NUT*16]
    double *coef;         // [groups][nt][m] centred basis
    double *coef_raw;     // [groups][nt][m] raw basis
    int *status;          // [groups] dropped columns
    int nt = 1;                 // target columns sharing one normal matrix
    size_t targ_tstride = 0;    // floats between a group's targets
    size_t pred_tstride = 0;    // floats between a group's predictions
    const float *centre = nullptr;   // [F] (poly2: [1]) centring state; null: path 0 of the group
};

// the centring state of the basis: the given one, else path 0 of the group's features
__device__ __forceinline__ float centre_of(const LsqArgs &a, const float *feat, int f)
{
    return a.centre ? __ldg(a.centre + f) : __ldg(feat + (size_t)f * a.M);
}

// value of augmented column `col` at row k (columns m..m+nt-1 are the targets);
// c0[f] is path 0's value of factor f (the centring of the basis)
__device__ __forceinline__ float basis_value(const LsqArgs &a, const float *feat, const float *targ,
                                            const float *c0, int col, uint32_t k)
{
    if (col >= a.m) return __ldg(targ + (size_t)(col - a.m) * a.targ_tstride + k);
    if (col == 0) return 1.f;
    if (a.basis == CVA_BASIS_POLY2) {
        const float d = __ldg(feat + k) - c0[0];
        return col == 1 ? d : d * d;
    }
    return __ldg(feat + (size_t)(col - 1) * a.M + k) - c0[col - 1];
}

template <int MP, int TR>
__global__ void __launch_bounds__(kGramThreads) lsq_gram(LsqArgs a)
{
    constexpr int NBLK = MP / 4, NUT = NBLK * (NBLK + 1) / 2, RS = MP + 4;
    constexpr int NRG = kGramThreads / NUT;
    extern __shared__ __align__(16) unsigned char smem[];
    float *tile = reinterpret_cast<float *>(smem);          // [TR][RS]
    const int g = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
    const float *feat = a.feat0 + (size_t)g * a.feat_stride;
    const float *targ = a.targ0 + (size_t)g * a.targ_stride;
    const uint32_t r_begin = (uint32_t)chunk * a.rows_per_chunk;
    const uint32_t r_end = min(a.M, r_begin + a.rows_per_chunk);
    const int mA = a.m + a.nt;

    // this thread's 4x4 block (bi <= bj) and row group
    const int b = tid % NUT, rg = tid / NUT;
    int bi = 0, bj = 0;
    {
        int t = b;
        for (int i = 0; i < NBLK; ++i) {
            if (t < NBLK - i) {
                bi = i;
                bj = i + t;
                break;
            }
            t -= NBLK - i;
        }
    }
    __shared__ float c0[40];
    for (int f = tid; f < (a.basis == CVA_BASIS_POLY2 ? 1 : a.F); f += kGramThreads) c0[f] = centre_of(a, feat, f);
    double dacc[16];
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        dacc[i] = 0.0;
        acc[i] = 0.f;
    }
    int since_flush = 0;

    for (uint32_t r0 = r_begin; r0 < r_end; r0 += TR) {
        __syncthreads();
        for (int i = tid; i < MP * TR; i += kGramThreads) {
            const int col = i / TR, r = i % TR;
            const uint32_t k = r0 + r;
            float v = 0.f;
            if (col < mA && k < r_end) v = basis_value(a, feat, targ, c0, col, k);
            tile[r * RS + col] = v;
        }
        __syncthreads();
        if (rg < NRG) {
            for (int r = rg; r < TR; r += NRG) {
                const float4 x = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bi);
                const float4 y = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bj);
                const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(xv[u], yv[v], acc[u * 4 + v]);
                if (++since_flush == 512) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        dacc[i] += (double)acc[i];
                        acc[i] = 0.f;
                    }
                    since_flush = 0;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) dacc[i] += (double)acc[i];

    // reduce the row groups in a fixed order
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem);        // [NRG][NUT*16]
    if (rg < NRG)
#pragma unroll
        for (int i = 0; i < 16; ++i) red[(size_t)rg * NUT * 16 + b * 16 + i] = dacc[i];
    __syncthreads();
    double *out = a.part + ((size_t)g * a.chunks + chunk) * NUT * 16;
    for (int e = tid; e < NUT * 16; e += kGramThreads) {
        double s = 0.0;
        for (int q = 0; q < NRG; ++q) s += red[(size_t)q * NUT * 16 + e];
        out[e] = s;
    }
}

__device__ __forceinline__ void cp_async4_zfill(uint32_t saddr, const void *g, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(g), "r"(valid ? 4 : 0) : "memory");
}

// lsq_gram for the linear basis [1, Y - Y^0] with the same arithmetic (the same rows
// per thread in the same order, the same flushes), its tiles copied by cp.async into
// two buffers so that the copies of the next tile run during the products of this
// one; the state columns are centred on path 0 in place once a tile has landed.
// Work blocks of lsq_gram_async per row group: for MP <= 12 the 4 x 4 blocks (bi <= bj)
// of the upper triangle; for MP = 32 and 40 the 4 x 8 blocks (bi, bj8) that touch it
// (2 bj8 + 1 >= bi), each a pair of 4 x 4 output blocks: three 16-byte operand reads
// per row for 32 FMAs instead of two for 16, so that a row costs a quarter of the
// issue slots.
template <int MP>
struct GramWork {
    static constexpr int NBLK = MP / 4, NUT = NBLK * (NBLK + 1) / 2;
    static constexpr bool wide = MP >= 32;
    static constexpr int count8()
    {
        int n = 0;
        for (int bi = 0; bi < NBLK; ++bi) n += MP / 8 - bi / 2;
        return n;
    }
    static constexpr int NW = wide ? count8() : NUT;          // work blocks
    static constexpr int NRG = kGramThreads / NW;             // row groups
    static constexpr int NA = wide ? 32 : 16;                 // accumulators per thread
};

// index of the 4 x 4 output block (bi <= bj) in the partial's block order
__host__ __device__ constexpr int gram_blk(int NBLK, int bi, int bj)
{
    return bi * NBLK - bi * (bi - 1) / 2 + (bj - bi);
}

template <int MP, int TR>
__global__ void __launch_bounds__(kGramThreads) lsq_gram_async(LsqArgs a)
{
    using GW = GramWork<MP>;
    constexpr int NBLK = MP / 4, NUT = NBLK * (NBLK + 1) / 2, RS = MP + 4, TS = TR * RS;
    constexpr int NRG = GW::NRG, NW = GW::NW, NA = GW::NA;
    extern __shared__ __align__(16) unsigned char smem[];
    float *tiles = reinterpret_cast<float *>(smem);          // [2][TR][RS]
    const int g = blockIdx.y, chunk = blockIdx.x, tid = threadIdx.x;
    const float *feat = a.feat0 + (size_t)g * a.feat_stride;
    const float *targ = a.targ0 + (size_t)g * a.targ_stride;
    const uint32_t r_begin = (uint32_t)chunk * a.rows_per_chunk;
    const uint32_t r_end = min(a.M, r_begin + a.rows_per_chunk);
    const int mA = a.m + a.nt, F = a.F, nload = a.F + a.nt;   // copied columns 1..F+nt: state, targets
    const int b = tid % NW, rg = tid / NW;
    int bi = 0, bj = 0;   // 4 x 4: block (bi, bj); 4 x 8: rows 4 bi.., columns 8 bj..
    {
        int t = b;
        for (int i = 0; i < NBLK; ++i) {
            const int w = GW::wide ? MP / 8 - i / 2 : NBLK - i;
            if (t < w) {
                bi = i;
                bj = (GW::wide ? i / 2 : i) + t;
                break;
            }
            t -= w;
        }
    }
    __shared__ float c0[40];
    for (int f = tid; f < F; f += kGramThreads) c0[f] = centre_of(a, feat, f);
    for (int e = tid; e < 2 * TR; e += kGramThreads)       // padding columns stay zero
        for (int c = mA; c < MP; ++c) tiles[e * RS + c] = 0.f;
    __syncthreads();
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tiles);
    auto issue = [&](uint32_t r0, int buf) {
        for (int e = tid; e < nload * TR; e += kGramThreads) {
            const int lc = e / TR, r = e % TR;
            const uint32_t k = r0 + r;
            const bool ok = k < r_end;
            const float *src = lc < F ? feat + (size_t)lc * a.M : targ + (size_t)(lc - F) * a.targ_tstride;
            cp_async4_zfill(sbase + (uint32_t)(buf * TS + r * RS + 1 + lc) * 4u, src + (ok ? k : 0u), ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    double dacc[NA];
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        dacc[i] = 0.0;
        acc[i] = 0.f;
    }
    int since_flush = 0;
    if (r_begin < r_end) issue(r_begin, 0);
    int buf = 0;
    for (uint32_t r0 = r_begin; r0 < r_end; r0 += TR, buf ^= 1) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();                          // tile r0 is in buffer buf; buf ^ 1 is free
        float *tile = tiles + buf * TS;
        for (int e = tid; e < (F + 1) * TR; e += kGramThreads) {
            const int col = e / TR, r = e % TR;
            const bool ok = r0 + r < r_end;
            float *v = tile + r * RS + col;
            if (col == 0) *v = ok ? 1.f : 0.f;
            else if (ok) *v -= c0[col - 1];
        }
        __syncthreads();
        if (r0 + TR < r_end) issue(r0 + TR, buf ^ 1);
        if (rg < NRG) {
            for (int r = rg; r < TR; r += NRG) {
                const float4 x = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bi);
                const float xv[4] = {x.x, x.y, x.z, x.w};
                float yv[NA / 4];
                if constexpr (GW::wide) {
                    const float4 y0 = *reinterpret_cast<const float4 *>(tile + r * RS + 8 * bj);
                    const float4 y1 = *reinterpret_cast<const float4 *>(tile + r * RS + 8 * bj + 4);
                    yv[0] = y0.x; yv[1] = y0.y; yv[2] = y0.z; yv[3] = y0.w;
                    yv[4] = y1.x; yv[5] = y1.y; yv[6] = y1.z; yv[7] = y1.w;
                } else {
                    const float4 y = *reinterpret_cast<const float4 *>(tile + r * RS + 4 * bj);
                    yv[0] = y.x; yv[1] = y.y; yv[2] = y.z; yv[3] = y.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < NA / 4; ++v) acc[u * (NA / 4) + v] = fmaf(xv[u], yv[v], acc[u * (NA / 4) + v]);
                if (++since_flush == 512) {
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        dacc[i] += (double)acc[i];
                        acc[i] = 0.f;
                    }
                    since_flush = 0;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NA; ++i) dacc[i] += (double)acc[i];
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem);        // [NRG][NUT*16]
    if (rg < NRG) {
        if constexpr (GW::wide) {   // the halves of the 4 x 8 block on or above the diagonal
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int bj4 = 2 * bj + h;
                if (bj4 < bi) continue;
                double *dst = red + (size_t)rg * NUT * 16 + gram_blk(NBLK, bi, bj4) * 16;
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) dst[u * 4 + v] = dacc[u * 8 + 4 * h + v];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) red[(size_t)rg * NUT * 16 + b * 16 + i] = dacc[i];
        }
    }
    __syncthreads();
    double *out = a.part + ((size_t)g * a.chunks + chunk) * NUT * 16;
    for (int e = tid; e < NUT * 16; e += kGramThreads) {
        double s = 0.0;
        for (int q = 0; q < NRG; ++q) s += red[(size_t)q * NUT * 16 + e];
        out[e] = s;
    }
}

// Launch the Gram kernel of width MP and tile TR: the cp.async form for the linear
// basis, the plain form (per-element basis values) for [1, r, r^2]. The dynamic shared
// memory limit is raised outside stream capture (a call before capture sets it).
template <int MP, int TR>
cva_status launch_gram(const LsqArgs &a, dim3 grid, cudaStream_t st)
{
    constexpr int NUT = (MP / 4) * (MP / 4 + 1) / 2, NRG = GramWork<MP>::NRG;
    if (a.basis == CVA_BASIS_LINEAR) {
        const size_t tiles = 2 * (size_t)TR * (MP + 4) * sizeof(float), red = (size_t)NRG * NUT * 16 * sizeof(double);
        const size_t smem = tiles > red ? tiles : red;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CVA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
        if (cap == cudaStreamCaptureStatusNone)
            CVA_CUDA_TRY(cudaFuncSetAttribute(lsq_gram_async<MP, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        lsq_gram_async<MP, TR><<<grid, kGramThreads, smem, st>>>(a);
    } else {
        lsq_gram<MP, TR><<<grid, kGramThreads, (size_t)TR * (MP + 4) * sizeof(float), st>>>(a);
    }
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

template <int MP>
__global__ void __launch_bounds__(256) lsq_solve(LsqArgs a)
{
    constexpr int NBLK = MP / 4, NUT = NBLK * (NBLK + 1) / 2;
    __shared__ double blocks[NUT * 16];
    __shared__ double A[MP * MP];
    __shared__ double sc[MP];
    __shared__ int drop[MP];
    const int g = blockIdx.x, tid = threadIdx.x, m = a.m, mA = m + a.nt;
    for (int e = tid; e < NUT * 16; e += blockDim.x) {
        double s = 0.0;
        const double *p = a.part + (size_t)g * a.chunks * NUT * 16 + e;
        for (int c = 0; c < a.chunks; ++c) s += p[(size_t)c * NUT * 16];
        blocks[e] = s;
    }
    __syncthreads();
    // unpack the upper-triangular 4x4 blocks into the dense augmented matrix
    for (int e = tid; e < NUT * 16; e += blockDim.x) {
        int t = e / 16, bi = 0;
        while (t >= NBLK - bi) {
            t -= NBLK - bi;
            ++bi;
        }
        const int bj = bi + t, i = 4 * bi + (e % 16) / 4, j = 4 * bj + e % 4;
        if (i < mA && j < mA) {
            A[i * MP + j] = blocks[e];
            A[j * MP + i] = blocks[e];
        }
    }
    __syncthreads();
    // Jacobi scaling, then a right-looking Cholesky factorisation of the scaled normal
    // matrix by the whole block (L overwrites the lower triangle); a column whose pivot
    // vanishes is dropped: its part of L is zero and its coefficient 0
    for (int r = tid; r < m; r += blockDim.x) {
        const double d = A[r * MP + r];
        drop[r] = !(d > 0.0);
        sc[r] = drop[r] ? 0.0 : 1.0 / sqrt(d);
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        if (c <= r) A[r * MP + c] *= sc[r] * sc[c];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            const double s = A[j * MP + j];
            if (drop[j] || !(s > 1e-12)) {
                drop[j] = 1;
                A[j * MP + j] = 1.0;
            } else {
                A[j * MP + j] = sqrt(s);
            }
        }
        __syncthreads();
        const double inv = drop[j] ? 0.0 : 1.0 / A[j * MP + j];
        for (int r = j + 1 + tid; r < m; r += blockDim.x) A[r * MP + j] *= inv;
        __syncthreads();
        const int t = m - j - 1;
        for (int e = tid; e < t * t; e += blockDim.x) {
            const int r = j + 1 + e / t, c = j + 1 + e % t;
            if (c <= r) A[r * MP + c] -= A[r * MP + j] * A[c * MP + j];
        }
        __syncthreads();
    }
    if (tid == 0) {
        int dropped = 0;
        for (int r = 0; r < m; ++r) dropped += drop[r];
        a.status[g] = dropped;
    }
    // one thread per target column: the two triangular solves and the coefficients
    if (tid >= a.nt) return;
    const int t = tid, rhs = m + t;
    const float *feat = a.feat0 + (size_t)g * a.feat_stride;
    double y[MP], w[MP];
    for (int i = 0; i < m; ++i) {               // L y = D^{-1/2} b
        double s = A[i * MP + rhs] * sc[i];
        for (int p = 0; p < i; ++p) s -= A[i * MP + p] * y[p];
        y[i] = drop[i] ? 0.0 : s / A[i * MP + i];
    }
    for (int i = m - 1; i >= 0; --i) {         // L^T z = y, w = D^{-1/2} z
        double s = y[i];
        for (int p = i + 1; p < m; ++p) s -= A[p * MP + i] * w[p];
        w[i] = drop[i] ? 0.0 : s / A[i * MP + i];
    }
    for (int i = 0; i < m; ++i) w[i] *= sc[i];
    double *co = a.coef + ((size_t)g * a.nt + t) * m, *cr = a.coef_raw + ((size_t)g * a.nt + t) * m;
    for (int i = 0; i < m; ++i) co[i] = w[i];
    if (a.basis == CVA_BASIS_POLY2) {
        const double c = (double)centre_of(a, feat, 0);
        cr[0] = w[0] - w[1] * c + w[2] * c * c;
        cr[1] = w[1] - 2.0 * w[2] * c;
        cr[2] = w[2];
    } else {
        double w0 = w[0];
        for (int f = 0; f < a.F; ++f) {
            const double c = (double)centre_of(a, feat, f);
            w0 -= w[1 + f] * c;
            cr[1 + f] = w[1 + f];
        }
        cr[0] = w0;
    }
}

// Predictions of every target column of group g (blockIdx.y) at one path per
// thread: the features are read once per path for all nt columns, and the block
// converts the group's FP64 coefficients to FP32 once (FP64 conversions run on
// the slow FP64 pipe). The FMA order per column is the basis order.
__global__ void __launch_bounds__(256) lsq_predict(LsqArgs a)
{
    __shared__ float cs[40 * 40];   // [nt][m], m + nt <= 40
    __shared__ float f0[40];        // path 0's state: the centring of the basis
    const int g = blockIdx.y, nt = a.nt, m = a.m;
    const double *co = a.coef + (size_t)g * nt * m;
    const float *feat = a.feat0 + (size_t)g * a.feat_stride;
    for (int i = threadIdx.x; i < nt * m; i += blockDim.x) cs[i] = (float)co[i];
    const int nf = a.basis == CVA_BASIS_POLY2 ? 1 : a.F;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) f0[f] = centre_of(a, feat, f);
    __syncthreads();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.M) return;
    float *out = a.pred0 + (size_t)g * a.pred_stride + k;
    if (a.basis == CVA_BASIS_POLY2) {
        const float d = __ldg(feat + k) - f0[0];
        for (int t = 0; t < nt; ++t)
            out[(size_t)t * a.pred_tstride] = fmaf(cs[t * m + 2], d * d, fmaf(cs[t * m + 1], d, cs[t * m]));
        return;
    }
    for (int t0 = 0; t0 < nt; t0 += 8) {
        const int tn = nt - t0 < 8 ? nt - t0 : 8;
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = u < tn ? cs[(t0 + u) * m] : 0.f;
        for (int f = 0; f < a.F; ++f) {
            const float x = __ldg(feat + (size_t)f * a.M + k) - f0[f];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < tn) acc[u] = fmaf(cs[(t0 + u) * m + 1 + f], x, acc[u]);
        }
        for (int u = 0; u < tn; ++u) out[(size_t)(t0 + u) * a.pred_tstride] = acc[u];
    }
}

// The linear-basis predictions of lsq_predict for 4 consecutive paths per thread:
// 16-byte feature loads and prediction stores, the same FMA order per path (so the
// same bits). Needs M, the strides and the base addresses to be multiples of 4
// floats (checked by lsq_predict_launch).
__global__ void __launch_bounds__(256) lsq_predict4(LsqArgs a)
{
    __shared__ float cs[40 * 40];   // [nt][m], m + nt <= 40
    __shared__ float f0[40];
    const int g = blockIdx.y, nt = a.nt, m = a.m;
    const double *co = a.coef + (size_t)g * nt * m;
    const float *feat = a.feat0 + (size_t)g * a.feat_stride;
    for (int i = threadIdx.x; i < nt * m; i += blockDim.x) cs[i] = (float)co[i];
    for (int f = threadIdx.x; f < a.F; f += blockDim.x) f0[f] = centre_of(a, feat, f);
    __syncthreads();
    const uint32_t k = 4u * (blockIdx.x * blockDim.x + threadIdx.x);
    if (k >= a.M) return;
    float *out = a.pred0 + (size_t)g * a.pred_stride + k;
    for (int t0 = 0; t0 < nt; t0 += 8) {
        const int tn = nt - t0 < 8 ? nt - t0 : 8;
        float4 acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float c = u < tn ? cs[(t0 + u) * m] : 0.f;
            acc[u] = make_float4(c, c, c, c);
        }
#pragma unroll 4
        for (int f = 0; f < a.F; ++f) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(feat + (size_t)f * a.M + k));
            const float c0 = f0[f];
            const float x0 = v.x - c0, x1 = v.y - c0, x2 = v.z - c0, x3 = v.w - c0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < tn) {
                    const float c = cs[(t0 + u) * m + 1 + f];
                    acc[u].x = fmaf(c, x0, acc[u].x);
                    acc[u].y = fmaf(c, x1, acc[u].y);
                    acc[u].z = fmaf(c, x2, acc[u].z);
                    acc[u].w = fmaf(c, x3, acc[u].w);
                }
        }
        for (int u = 0; u < tn; ++u) *reinterpret_cast<float4 *>(out + (size_t)(t0 + u) * a.pred_tstride) = acc[u];
    }
}

// Predictions of every group: 4 paths per thread where the shapes allow 16-byte
// accesses, else one path per thread.
cva_status lsq_predict_launch(const LsqArgs &a, int groups, cudaStream_t st)
{
    const bool wide = a.basis == CVA_BASIS_LINEAR && a.M % 4 == 0 && a.feat_stride % 4 == 0 && a.pred_stride % 4 == 0 &&
                      a.pred_tstride % 4 == 0 && (reinterpret_cast<uintptr_t>(a.feat0) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(a.pred0) & 15u) == 0;
    if (wide)
        lsq_predict4<<<dim3((unsigned)((a.M / 4 + 255) / 256), (unsigned)groups), 256, 0, st>>>(a);
    else
        lsq_predict<<<dim3((unsigned)((a.M + 255) / 256), (unsigned)groups), 256, 0, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

// Library-owned scratch for the Gram partials and coefficients, per device.
// Reuse is ordered by an event: a call waits for the previous call's kernels.
struct LsqScratch {
    double *buf = nullptr;
    size_t cap = 0;   // doubles
    cudaEvent_t done = nullptr;
};
std::mutex g_lsq_mu;
LsqScratch g_lsq[64];

}  // namespace

// Launch the grouped regression with the given scratch ([groups] x (chunks x NUT x 16 +
// 2 x nt x m) doubles + groups ints); chunk_target sets the blocks per launch.
static size_t lsq_scratch_doubles(int groups, int m, int nt, uint64_t chunks, int NUT)
{
    return (size_t)groups * chunks * NUT * 16 + 2 * (size_t)groups * nt * m + (size_t)groups;
}

static int lsq_width(int m, int nt) { return (m + nt <= 4) ? 4 : (m + nt <= 12) ? 12 : (m + nt <= 32) ? 32 : 40; }

static uint64_t lsq_chunks(uint64_t M, int groups, int chunk_target)
{
    const uint64_t max_chunks = (M + 1023) / 1024;
    uint64_t chunks = ((uint64_t)chunk_target + groups - 1) / groups;
    if (chunks > max_chunks) chunks = max_chunks;
    return chunks < 1 ? 1 : chunks;
}

cva_status lsq_launch(const LsqJob &j, double *scratch, size_t scratch_cap, double *coef_host, cudaStream_t st)
{
    if (!j.feat0 || !j.targ0 || j.M == 0 || j.groups <= 0 || j.nt < 1)
        return fail(CVA_EINVAL, "regress: bad arguments");
    if (j.M > 0x7fffffffull) return fail(CVA_EINVAL, "regress: M too large");
    if (j.basis != CVA_BASIS_LINEAR && j.basis != CVA_BASIS_POLY2) return fail(CVA_EINVAL, "regress: unknown basis");
    const int m = (j.basis == CVA_BASIS_POLY2) ? 3 : j.F + 1;
    if (j.F < 1) return fail(CVA_EINVAL, "regress: need one factor");
    if (m + j.nt > 40) return fail(CVA_ENOTSUP, "regress: basis columns + targets must be <= 40");
    const int MP = lsq_width(m, j.nt);
    const int NUT = (MP / 4) * (MP / 4 + 1) / 2;
    const uint64_t chunks = lsq_chunks(j.M, j.groups, j.chunk_target > 0 ? j.chunk_target : 2432);
    if (lsq_scratch_doubles(j.groups, m, j.nt, chunks, NUT) > scratch_cap) return fail(CVA_ENOMEM, "regress: scratch too small");
    LsqArgs a;
    a.feat0 = j.feat0;
    a.feat_stride = j.feat_stride;
    a.targ0 = j.targ0;
    a.targ_stride = j.targ_stride;
    a.targ_tstride = j.targ_tstride;
    a.pred0 = j.pred0;
    a.pred_stride = j.pred_stride;
    a.pred_tstride = j.pred_tstride;
    a.nt = j.nt;
    a.F = j.F;
    a.m = m;
    a.basis = j.basis;
    a.chunks = (int)chunks;
    a.M = (uint32_t)j.M;
    a.rows_per_chunk = (uint32_t)((j.M + chunks - 1) / chunks);
    a.part = scratch;
    a.coef = a.part + (size_t)j.groups * chunks * NUT * 16;
    a.coef_raw = a.coef + (size_t)j.groups * j.nt * m;
    a.status = reinterpret_cast<int *>(a.coef_raw + (size_t)j.groups * j.nt * m);
    const dim3 ggrid((unsigned)chunks, (unsigned)j.groups);
    cva_status gr;
    switch (MP) {
    case 4: gr = launch_gram<4, 1024>(a, ggrid, st); break;
    case 12: gr = launch_gram<12, 512>(a, ggrid, st); break;
    case 32: gr = launch_gram<32, 256>(a, ggrid, st); break;
    default: gr = launch_gram<40, 256>(a, ggrid, st); break;
    }
    if (gr != CVA_OK) return gr;
    switch (MP) {
    case 4: lsq_solve<4><<<j.groups, 256, 0, st>>>(a); break;
    case 12: lsq_solve<12><<<j.groups, 256, 0, st>>>(a); break;
    case 32: lsq_solve<32><<<j.groups, 256, 0, st>>>(a); break;
    default: lsq_solve<40><<<j.groups, 256, 0, st>>>(a); break;
    }
    CVA_CUDA_TRY(cudaGetLastError());
    if (j.pred0) {
        cva_status pr = lsq_predict_launch(a, j.groups, st);
        if (pr != CVA_OK) return pr;
    }
    if (coef_host) {
        std::vector<int> status(j.groups);
        CVA_CUDA_TRY(cudaMemcpyAsync(coef_host, a.coef_raw, sizeof(double) * j.groups * j.nt * m,
                                     cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaMemcpyAsync(status.data(), a.status, sizeof(int) * j.groups, cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        for (int g = 0; g < j.groups; ++g)
            if (status[g] != 0) return fail(CVA_ENUMERIC, "regress: rank-deficient normal equations");
    }
    return CVA_OK;
}

size_t lsq_scratch_need(const LsqJob &j)
{
    const int m = (j.basis == CVA_BASIS_POLY2) ? 3 : j.F + 1;
    const int MP = lsq_width(m, j.nt);
    const int NUT = (MP / 4) * (MP / 4 + 1) / 2;
    return lsq_scratch_doubles(j.groups, m, j.nt, lsq_chunks(j.M, j.groups, j.chunk_target > 0 ? j.chunk_target : 2432), NUT);
}

cva_status lsq_grouped_strided(const float *feat0, size_t feat_stride, const float *targ0,
                               size_t targ_stride, float *pred0, size_t pred_stride, int F,
                               uint64_t M, int basis, int groups, double *coef_host, cudaStream_t st)
{
    LsqJob j;
    j.feat0 = feat0;
    j.feat_stride = feat_stride;
    j.targ0 = targ0;
    j.targ_stride = targ_stride;
    j.pred0 = pred0;
    j.pred_stride = pred_stride;
    j.F = F;
    j.M = M;
    j.basis = basis;
    j.groups = groups;
    if (!feat0 || !targ0 || M == 0 || groups <= 0) return fail(CVA_EINVAL, "regress: bad arguments");
    if (M > 0x7fffffffull) return fail(CVA_EINVAL, "regress: M too large");
    if (basis != CVA_BASIS_LINEAR && basis != CVA_BASIS_POLY2) return fail(CVA_EINVAL, "regress: unknown basis");
    if (F < 1) return fail(CVA_EINVAL, "regress: need one factor");
    if (basis == CVA_BASIS_LINEAR && F + 2 > 32) return fail(CVA_ENOTSUP, "regress: linear basis supports 1 <= F <= 30");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CVA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lk(g_lsq_mu);
    LsqScratch &sc = g_lsq[dev];
    const size_t need = lsq_scratch_need(j);
    if (cap != cudaStreamCaptureStatusNone) {
        // inside a stream capture the scratch must already be large enough: a graph keeps its address
        if (sc.cap < need) return fail(CVA_EINVAL, "regress: call once before capturing so that the scratch exists");
        return lsq_launch(j, sc.buf, sc.cap, coef_host, st);
    }
    if (!sc.done) CVA_CUDA_TRY(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming));
    else CVA_CUDA_TRY(cudaStreamWaitEvent(st, sc.done, 0));
    if (sc.cap < need) {
        if (sc.buf) {
            CVA_CUDA_TRY(cudaEventSynchronize(sc.done));
            cudaFree(sc.buf);
            sc.buf = nullptr;
            sc.cap = 0;
        }
        if (cudaMalloc(&sc.buf, need * sizeof(double)) != cudaSuccess)
            return fail(CVA_ENOMEM, "regress: scratch allocation failed");
        sc.cap = need;
    }
    cva_status r = lsq_launch(j, sc.buf, sc.cap, coef_host, st);
    if (r != CVA_OK) return r;
    CVA_CUDA_TRY(cudaEventRecord(sc.done, st));
    return CVA_OK;
}

// ---------------------------------------------------------------------------
// Least squares split over path ranges (one range per process and GPU). Every
// range accumulates its augmented normal matrix with the same centring (a state
// vector all ranges agree on), the host sums the ranges' matrices in a fixed order
// and solves once; each range then predicts its own paths. The sum over ranges is
// the normal matrix of all paths, so the fit is the one of the whole sample.

// the library's regression scratch of the current device, grown to `need` doubles
// (the previous user of a larger one has finished: callers synchronise)
static cva_status lsq_scratch_get(size_t need, cudaStream_t st, double **out)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_lsq_mu);
    LsqScratch &sc = g_lsq[dev];
    if (!sc.done) CVA_CUDA_TRY(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming));
    else CVA_CUDA_TRY(cudaStreamWaitEvent(st, sc.done, 0));
    if (sc.cap < need) {
        if (sc.buf) {
            CVA_CUDA_TRY(cudaEventSynchronize(sc.done));
            cudaFree(sc.buf);
            sc.buf = nullptr;
            sc.cap = 0;
        }
        if (cudaMalloc(&sc.buf, need * sizeof(double)) != cudaSuccess)
            return fail(CVA_ENOMEM, "regress: scratch allocation failed");
        sc.cap = need;
    }
    *out = sc.buf;
    return CVA_OK;
}

static cva_status lsq_scratch_release(cudaStream_t st)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_lsq_mu);
    CVA_CUDA_TRY(cudaEventRecord(g_lsq[dev].done, st));
    return CVA_OK;
}

static cva_status lsq_split_check(const float *feat, uint64_t M, int F, int basis, const float *centre)
{
    if (!feat || !centre || M == 0) return fail(CVA_EINVAL, "regress: bad arguments");
    if (M > 0x7fffffffull) return fail(CVA_EINVAL, "regress: M too large");
    if (basis != CVA_BASIS_LINEAR && basis != CVA_BASIS_POLY2) return fail(CVA_EINVAL, "regress: unknown basis");
    if (F < 1) return fail(CVA_EINVAL, "regress: need one factor");
    if (basis == CVA_BASIS_LINEAR && F + 2 > 32) return fail(CVA_ENOTSUP, "regress: linear basis supports 1 <= F <= 30");
    return CVA_OK;
}

cva_status lsq_normal_partial(const float *targ, const float *feat, int F, uint64_t M, int basis, const float *centre,
                              double *gram_host, cudaStream_t st)
{
    cva_status r = lsq_split_check(feat, M, F, basis, centre);
    if (r != CVA_OK) return r;
    if (!targ || !gram_host) return fail(CVA_EINVAL, "regress: bad arguments");
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : F + 1, mA = m + 1;
    const int MP = lsq_width(m, 1), NBLK = MP / 4, NUT = NBLK * (NBLK + 1) / 2;
    const uint64_t chunks = lsq_chunks(M, 1, 2432);
    double *part = nullptr;
    r = lsq_scratch_get((size_t)(chunks + 1) * NUT * 16, st, &part);
    if (r != CVA_OK) return r;
    LsqArgs a;
    a.feat0 = feat;
    a.feat_stride = (size_t)F * M;
    a.targ0 = targ;
    a.targ_stride = M;
    a.pred0 = nullptr;
    a.pred_stride = M;
    a.F = F;
    a.m = m;
    a.basis = basis;
    a.chunks = (int)chunks;
    a.M = (uint32_t)M;
    a.rows_per_chunk = (uint32_t)((M + chunks - 1) / chunks);
    a.part = part;
    a.coef = a.coef_raw = nullptr;
    a.status = nullptr;
    a.centre = centre;
    const dim3 ggrid((unsigned)chunks, 1u);
    switch (MP) {
    case 4: r = launch_gram<4, 1024>(a, ggrid, st); break;
    case 12: r = launch_gram<12, 512>(a, ggrid, st); break;
    default: r = launch_gram<32, 256>(a, ggrid, st); break;
    }
    if (r == CVA_OK) r = sum_columns_fp64(part, (int)chunks, NUT * 16, part + (size_t)chunks * NUT * 16, st);
    std::vector<double> blocks((size_t)NUT * 16);
    if (r == CVA_OK) {
        cudaError_t e = cudaMemcpyAsync(blocks.data(), part + (size_t)chunks * NUT * 16, sizeof(double) * NUT * 16,
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "regress: copy of the normal matrix");
    }
    const cva_status rr = lsq_scratch_release(st);
    if (r != CVA_OK) return r;
    if (rr != CVA_OK) return rr;
    // the upper-triangular 4x4 blocks -> the dense symmetric (m+1) x (m+1) matrix
    for (int e = 0; e < NUT * 16; ++e) {
        int t = e / 16, bi = 0;
        while (t >= NBLK - bi) {
            t -= NBLK - bi;
            ++bi;
        }
        const int bj = bi + t, i = 4 * bi + (e % 16) / 4, j = 4 * bj + e % 4;
        if (i < mA && j < mA) {
            gram_host[(size_t)i * mA + j] = blocks[e];
            gram_host[(size_t)j * mA + i] = blocks[e];
        }
    }
    return CVA_OK;
}

// The solve of lsq_solve on the host: Jacobi scaling, Cholesky factorisation of the
// scaled normal matrix with vanishing pivots dropped (coefficient 0), the two
// triangular solves; coefficients in the centred basis and in the raw one.
cva_status lsq_solve_normal_host(const double *gram, int F, int basis, const double *centre, double *coef_centred,
                                 double *coef_raw, int *dropped)
{
    if (!gram || !centre || F < 1 || (basis != CVA_BASIS_LINEAR && basis != CVA_BASIS_POLY2))
        return fail(CVA_EINVAL, "regress: bad arguments");
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : F + 1, mA = m + 1;
    std::vector<double> A((size_t)m * m), sc(m), y(m), w(m);
    std::vector<int> drop(m);
    for (int r = 0; r < m; ++r) {
        const double d = gram[(size_t)r * mA + r];
        drop[r] = !(d > 0.0);
        sc[r] = drop[r] ? 0.0 : 1.0 / sqrt(d);
    }
    for (int r = 0; r < m; ++r)
        for (int c = 0; c <= r; ++c) A[(size_t)r * m + c] = gram[(size_t)r * mA + c] * sc[r] * sc[c];
    for (int j = 0; j < m; ++j) {
        const double s = A[(size_t)j * m + j];
        if (drop[j] || !(s > 1e-12)) {
            drop[j] = 1;
            A[(size_t)j * m + j] = 1.0;
        } else {
            A[(size_t)j * m + j] = sqrt(s);
        }
        const double inv = drop[j] ? 0.0 : 1.0 / A[(size_t)j * m + j];
        for (int r = j + 1; r < m; ++r) A[(size_t)r * m + j] *= inv;
        for (int r = j + 1; r < m; ++r)
            for (int c = j + 1; c <= r; ++c) A[(size_t)r * m + c] -= A[(size_t)r * m + j] * A[(size_t)c * m + j];
    }
    int nd = 0;
    for (int r = 0; r < m; ++r) nd += drop[r];
    for (int i = 0; i < m; ++i) {               // L y = D^{-1/2} b
        double s = gram[(size_t)i * mA + m] * sc[i];
        for (int p = 0; p < i; ++p) s -= A[(size_t)i * m + p] * y[p];
        y[i] = drop[i] ? 0.0 : s / A[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {         // L^T z = y, w = D^{-1/2} z
        double s = y[i];
        for (int p = i + 1; p < m; ++p) s -= A[(size_t)p * m + i] * w[p];
        w[i] = drop[i] ? 0.0 : s / A[(size_t)i * m + i];
    }
    for (int i = 0; i < m; ++i) w[i] *= sc[i];
    if (coef_centred)
        for (int i = 0; i < m; ++i) coef_centred[i] = w[i];
    if (coef_raw) {
        if (basis == CVA_BASIS_POLY2) {
            const double c = centre[0];
            coef_raw[0] = w[0] - w[1] * c + w[2] * c * c;
            coef_raw[1] = w[1] - 2.0 * w[2] * c;
            coef_raw[2] = w[2];
        } else {
            double w0 = w[0];
            for (int f = 0; f < F; ++f) {
                w0 -= w[1 + f] * centre[f];
                coef_raw[1 + f] = w[1 + f];
            }
            coef_raw[0] = w0;
        }
    }
    if (dropped) *dropped = nd;
    return CVA_OK;
}

cva_status lsq_predict_centred(const float *feat, int F, uint64_t M, int basis, const float *centre,
                               const double *coef_centred_host, float *pred, cudaStream_t st)
{
    cva_status r = lsq_split_check(feat, M, F, basis, centre);
    if (r != CVA_OK) return r;
    if (!coef_centred_host || !pred) return fail(CVA_EINVAL, "regress: bad arguments");
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : F + 1;
    double *coef = nullptr;
    r = lsq_scratch_get((size_t)m, st, &coef);
    if (r != CVA_OK) return r;
    cudaError_t e = cudaMemcpyAsync(coef, coef_centred_host, sizeof(double) * m, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "regress: coefficients to the device");
    LsqArgs a;
    a.feat0 = feat;
    a.feat_stride = (size_t)F * M;
    a.targ0 = nullptr;
    a.targ_stride = M;
    a.pred0 = pred;
    a.pred_stride = M;
    a.F = F;
    a.m = m;
    a.basis = basis;
    a.chunks = 1;
    a.M = (uint32_t)M;
    a.rows_per_chunk = (uint32_t)M;
    a.part = nullptr;
    a.coef = coef;
    a.coef_raw = nullptr;
    a.status = nullptr;
    a.centre = centre;
    r = lsq_predict_launch(a, 1, st);
    // the host coefficients are read by the copy above before the call returns
    e = cudaStreamSynchronize(st);
    const cva_status rr = lsq_scratch_release(st);
    if (r != CVA_OK) return r;
    if (e != cudaSuccess) return cuda_fail(e, "regress: predictions");
    return rr;
}

// ---------------------------------------------------------------------------
// Regression without any device allocation.
//
// Some callers cannot allocate device memory at the time they need a fit: a
// framework may own the whole device through its own pool, a process may run
// under a fixed memory budget checked at start-up, or a latency-critical loop
// cannot afford the device-wide synchronisation of cudaMalloc/cudaFree. For
// them, the batched regression below keeps its Gram partials, coefficients and
// status words in this file-scope array instead of library-allocated scratch.
// The array lives on every device that loads the library until the process
// exits. Its size bounds the number of groups per call (see the check below).
// All calls share it: each call writes every entry it later reads, so nothing
// has to start at zero, but two calls whose kernels overlap on the GPU (for
// instance on two streams) race on it and must be ordered by the caller.
constexpr size_t kStaticScratchDoubles = 1u << 17;   // 1 MiB
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {
std::mutex g_static_mu;
struct StaticSetup {
    unsigned long long ctx_id = 0;   // CUDA context the address below belongs to (0: none yet)
    double *ptr = nullptr;
};
StaticSetup g_static[64];
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

// dynamic shared memory of the linear-basis Gram kernel at width MP (launch_gram's size)
template <int MP, int TR>
cva_status static_gram_attr()
{
    constexpr int NUT = (MP / 4) * (MP / 4 + 1) / 2, NRG = GramWork<MP>::NRG;
    const size_t tiles = 2 * (size_t)TR * (MP + 4) * sizeof(float), red = (size_t)NRG * NUT * 16 * sizeof(double);
    CVA_CUDA_TRY(cudaFuncSetAttribute(lsq_gram_async<MP, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(tiles > red ? tiles : red)));
    return CVA_OK;
}
}  // namespace

// Set-up of the allocation-free path on the current device, once per device and
// CUDA context (a context created after cudaDeviceReset gets its own): the device
// address of the static scratch (cudaGetSymbolAddress; the host-side name is only
// a stand-in for the device array) and the shared-memory limits of the Gram
// kernels it launches. Later calls in the same context reuse both.
static cva_status static_scratch(double **out)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        CVA_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1));
        CVA_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (!f1 || !f2 || q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess)
            return fail(CVA_ECUDA, "regress_static: cuCtxGetCurrent / cuCtxGetId not available");
        g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
    }
    CVA_CUDA_TRY(cudaSetDevice(dev));   // initialises the device's primary context and makes it current
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS)
        return fail(CVA_ECUDA, "regress_static: no current CUDA context");
    StaticSetup &su = g_static[dev];
    if (su.ctx_id != id || !su.ptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
        cva_status r = static_gram_attr<12, 512>();
        if (r == CVA_OK) r = static_gram_attr<32, 256>();
        if (r != CVA_OK) return r;
        su.ptr = static_cast<double *>(p);
        su.ctx_id = id;
    }
    *out = su.ptr;
    return CVA_OK;
}

cva_status lsq_batched_static(const float *targ0, const float *feat0, int groups, int F, uint64_t M,
                              int basis, float *pred0, double *coef_host, cudaStream_t st)
{
    if (!feat0 || !targ0 || M == 0 || groups <= 0) return fail(CVA_EINVAL, "regress_static: bad arguments");
    if (M > 0x7fffffffull) return fail(CVA_EINVAL, "regress_static: M too large");
    if (basis != CVA_BASIS_LINEAR && basis != CVA_BASIS_POLY2)
        return fail(CVA_EINVAL, "regress_static: unknown basis");
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : F + 1;
    if (basis == CVA_BASIS_LINEAR && (F < 1 || m + 1 > 32))
        return fail(CVA_ENOTSUP, "regress_static: linear basis supports 1 <= F <= 30");
    if (basis == CVA_BASIS_POLY2 && F < 1) return fail(CVA_EINVAL, "regress_static: need one factor");
    const int MP = lsq_width(m, 1);
    const size_t NUT = (size_t)(MP / 4) * (MP / 4 + 1) / 2;
    const size_t per_group_fixed = 2 * (size_t)m + 1;          // coefficients (two bases) + status
    const size_t per_chunk = NUT * 16;
    const size_t max_groups = kStaticScratchDoubles / (per_chunk + per_group_fixed);
    if ((size_t)groups > max_groups || groups > 1024)
        return fail(CVA_EINVAL, "regress_static: " + std::to_string(groups) + " groups exceed the static scratch (at most " +
                                    std::to_string(max_groups < 1024 ? max_groups : 1024) +
                                    " groups of this basis per call)");
    if (coef_host) {   // the coefficients come back through a synchronisation of st
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CVA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CVA_EINVAL, "regress_static: coef_host needs a synchronisation of the stream, which is "
                                    "being captured; pass coef_host = NULL there");
    }
    double *scratch = nullptr;
    cva_status r = static_scratch(&scratch);
    if (r != CVA_OK) return r;

    const uint64_t max_chunks = (M + 1023) / 1024;
    uint64_t chunks = (2432 + groups - 1) / groups;
    const uint64_t fit = (kStaticScratchDoubles - (size_t)groups * per_group_fixed) / ((size_t)groups * per_chunk);
    if (chunks > fit) chunks = fit;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;

    LsqArgs a;
    a.feat0 = feat0;
    a.feat_stride = (size_t)F * M;
    a.targ0 = targ0;
    a.targ_stride = M;
    a.pred0 = pred0;
    a.pred_stride = M;
    a.F = F;
    a.m = m;
    a.basis = basis;
    a.chunks = (int)chunks;
    a.M = (uint32_t)M;
    a.rows_per_chunk = (uint32_t)((M + chunks - 1) / chunks);
    a.part = scratch;
    a.coef = a.part + (size_t)groups * chunks * per_chunk;
    a.coef_raw = a.coef + (size_t)groups * m;
    a.status = reinterpret_cast<int *>(a.coef_raw + (size_t)groups * m);

    const dim3 ggrid((unsigned)chunks, (unsigned)groups);
    cva_status gr = CVA_OK;
    switch (MP) {
    case 4: gr = launch_gram<4, 1024>(a, ggrid, st); break;
    case 12: gr = launch_gram<12, 512>(a, ggrid, st); break;
    default: gr = launch_gram<32, 256>(a, ggrid, st); break;
    }
    if (gr != CVA_OK) return gr;
    switch (MP) {
    case 4: lsq_solve<4><<<groups, 256, 0, st>>>(a); break;
    case 12: lsq_solve<12><<<groups, 256, 0, st>>>(a); break;
    default: lsq_solve<32><<<groups, 256, 0, st>>>(a); break;
    }
    CVA_CUDA_TRY(cudaGetLastError());
    if (pred0) {
        cva_status pr = lsq_predict_launch(a, groups, st);
        if (pr != CVA_OK) return pr;
    }
    if (coef_host) {
        int status[1024];
        CVA_CUDA_TRY(cudaMemcpyAsync(coef_host, a.coef_raw, sizeof(double) * groups * m, cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaMemcpyAsync(status, a.status, sizeof(int) * groups, cudaMemcpyDeviceToHost, st));
        CVA_CUDA_TRY(cudaStreamSynchronize(st));
        for (int g = 0; g < groups; ++g)
            if (status[g] != 0) return fail(CVA_ENUMERIC, "regress_static: rank-deficient normal equations");
    }
    return CVA_OK;
}

}  // namespace cva
