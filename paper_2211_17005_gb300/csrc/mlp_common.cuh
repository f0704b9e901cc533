// Pieces shared by the neural-regression kernels of both hidden widths (mlp.cu,
// mlp_wide.cu): tile constants, BF16 packing, warp reductions, the input
// standardisation of every date, the closed-form output-layer refit (FP64
// Cholesky) and the TMA descriptor of a date's feature array. Each translation
// unit that includes this file gets its own copy (internal linkage).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <string>

#include "cva_internal.h"

namespace cva {
namespace {

constexpr int kRows = 128;        // rows per tile (tcgen05 M)
constexpr int kIn = 32;           // padded input width
constexpr uint32_t kMbarPolls = 1u << 26;

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    return (uint32_t)bf16_bits(a) | ((uint32_t)bf16_bits(b) << 16);
}

__device__ __forceinline__ uint4 pack8(const float *v)
{
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

// Adam's parameter step lr m_hat / (sqrt(v_hat) + eps) (Kingma & Ba) with the bias
// corrections applied as reciprocals computed once per step, and the square root and
// the division by the hardware approximations (about 2 ulp). The IEEE-rounded
// division and square root take a slow path on subnormal moments (squared gradients
// below 1.2e-38, common for the weights of nearly inactive units), which made the
// owners of such parameters several times slower than the others at every step;
// a subnormal v_hat is flushed to zero here, against eps = 1e-8 it weighs nothing.
__device__ __forceinline__ float adam_delta(float m, float v, float inv_bc1, float inv_bc2, float lr, float eps)
{
    float s;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(v * inv_bc2));
    return __fdividef(lr * (m * inv_bc1), s + eps);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of 64 columns over the 32 lanes of a warp by recursive halving (levels
// 16, 8, 4, 2, 1): lane l ends with the totals of columns 2l and 2l + 1.
__device__ __forceinline__ float2 column_sums64(const float (&v)[64], int lane)
{
    float a32[32], a16[16], a8[8], a4[4];
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2, u1 = lane & 1;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float send = u16 ? v[i] : v[32 + i], keep = u16 ? v[32 + i] : v[i];
        a32[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float send = u8 ? a32[i] : a32[16 + i], keep = u8 ? a32[16 + i] : a32[i];
        a16[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float send = u4 ? a16[i] : a16[8 + i], keep = u4 ? a16[8 + i] : a16[i];
        a8[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = u2 ? a8[i] : a8[4 + i], keep = u2 ? a8[4 + i] : a8[i];
        a4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    float r[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = u1 ? a4[i] : a4[2 + i], keep = u1 ? a4[2 + i] : a4[i];
        r[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
    return make_float2(r[0], r[1]);
}

// Refit of (w3, b3) at epoch floor(E/2) for hidden width U: block i sums row i of
// the CTAs' Gram partials of Z = [h2 | 1 | y - mu] (fixed order) and stores it in FP64
// (G) and FP32 (Gf, after G); the last block solves the normal equations of
// [h2 | 1] (w3, b3) = y - mu Jacobi-scaled to a unit diagonal (S A S z = S b, x = S z;
// any positive S gives the same x, so S is taken at FP32 accuracy). It factorises the
// scaled matrix in FP32 (right-looking Cholesky over register tiles, one barrier per
// column) and refines z by FP64 residuals of the unscaled system, r = b - A x, with
// FP32 blocked triangular solves, until |S r| <= 1e-12 (|S b| + |z|) (at most 6
// rounds): the FP64 solution, with the factorisation at the FP32 rate (FP64
// arithmetic runs at a small fraction of it on this GPU). A pivot below 1e-5 of the
// unit diagonal or no convergence falls back to the FP64 Cholesky and triangular
// solves of the scaled system. A ReLU unit that is zero on every path has a zero row
// and column: it gets a unit diagonal and the weight 0 (the minimum-norm choice). The
// FP64 factor drops a column whose pivot is at or below 1e-12 (it lies in the span of
// the columns before it); a pivot that is not finite keeps the old (w3, b3). The new
// values go to params and, when not null, to params2. Dynamic shared memory:
// refit_smem_bytes(U); G holds refit_g_bytes(U).

// Register tiles of the FP32 factor: side T, NT tile rows over the U + 1 unknowns,
// one tile of the lower triangle per thread.
__host__ __device__ constexpr int refit_tile(int U) { return U >= 128 ? 8 : 4; }
__host__ __device__ constexpr int refit_ntiles(int U) { return (U + 1 + refit_tile(U) - 1) / refit_tile(U); }
__host__ __device__ constexpr size_t refit_g_bytes(int U)
{
    return (size_t)(U + 2) * (U + 2) * (sizeof(double) + sizeof(float));
}
__host__ __device__ constexpr size_t refit_smem_bytes(int U)
{
    return ((size_t)(U + 2) * (U + 2) + 3 * (size_t)(U + 1) + 256) * sizeof(double) +
           5 * (size_t)refit_ntiles(U) * refit_tile(U) * sizeof(float);
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only), its group commit
// and the wait for every copy of this thread.
__device__ __forceinline__ void refit_cp16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void refit_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void refit_cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Largest v over the warp, in every lane.
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// y <- (L L^T)^{-1} y in FP32 for the factor held in register tiles (the tile (R, C)
// of side T in each owning thread, the reciprocal diagonal in invf): blocked
// forward and back substitution over the NT tile columns, two barriers per tile
// column. The thread of a diagonal tile solves its T x T triangle; the threads of
// the tiles below it (forward) or left of it (backward) then update their own block
// of y, a different block for each thread.
template <int T, int NT>
__device__ __forceinline__ void refit_tile_solve(const float (&a)[T][T], bool own, int R, int C, float *yf,
                                                 const float *invf)
{
    for (int J = 0; J < NT; ++J) {
        if (own && R == J && C == J) {
            float y[T];
#pragma unroll
            for (int q = 0; q < T; ++q) y[q] = yf[J * T + q];
#pragma unroll
            for (int k = 0; k < T; ++k) {
                y[k] *= invf[J * T + k];
#pragma unroll
                for (int ii = k + 1; ii < T; ++ii) y[ii] = fmaf(-a[ii][k], y[k], y[ii]);
            }
#pragma unroll
            for (int q = 0; q < T; ++q) yf[J * T + q] = y[q];
        }
        __syncthreads();
        if (own && C == J && R > J) {
            float yj[T];
#pragma unroll
            for (int k = 0; k < T; ++k) yj[k] = yf[J * T + k];
#pragma unroll
            for (int ii = 0; ii < T; ++ii) {
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < T; ++k) s = fmaf(a[ii][k], yj[k], s);
                yf[R * T + ii] -= s;
            }
        }
        __syncthreads();
    }
    for (int J = NT - 1; J >= 0; --J) {
        if (own && R == J && C == J) {
            float y[T];
#pragma unroll
            for (int q = 0; q < T; ++q) y[q] = yf[J * T + q];
#pragma unroll
            for (int k = T - 1; k >= 0; --k) {
                y[k] *= invf[J * T + k];
#pragma unroll
                for (int ii = 0; ii < k; ++ii) y[ii] = fmaf(-a[k][ii], y[k], y[ii]);
            }
#pragma unroll
            for (int q = 0; q < T; ++q) yf[J * T + q] = y[q];
        }
        __syncthreads();
        if (own && R == J && C < J) {
            float xj[T];
#pragma unroll
            for (int q = 0; q < T; ++q) xj[q] = yf[J * T + q];
#pragma unroll
            for (int k = 0; k < T; ++k) {
                float s = 0.f;
#pragma unroll
                for (int ii = 0; ii < T; ++ii) s = fmaf(a[ii][k], xj[ii], s);
                yf[C * T + k] -= s;
            }
        }
        __syncthreads();
    }
}

template <int U>
__global__ void __launch_bounds__(256) mlp_refit_kernel(const double *part, int nparts, double *G, unsigned *count,
                                                        float *params, float *params2)
{
    constexpr int Z = U + 2, n1 = U + 1;
    constexpr int T = refit_tile(U), NT = refit_ntiles(U), P = NT * T;
    static_assert(NT * (NT + 1) / 2 <= 256, "one register tile per thread");
    constexpr int ow3 = 34 * U + U * U, ob3 = ow3 + U;
    extern __shared__ double refit_smem[];
    double *A = refit_smem, *sc = A + Z * Z, *xv = sc + n1, *inv_d = xv + n1, *half = inv_d + n1;
    float *colbuf = reinterpret_cast<float *>(half + 256), *invf = colbuf + 2 * P, *yf = invf + P, *scf = yf + P;
    __shared__ int s_last, s_singular;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = (int)blockDim.x >> 5;
    const int i = blockIdx.x;
    float *Gf = reinterpret_cast<float *>(G + Z * Z);
    {   // row i of the total Gram matrix: nh fixed ranges of the partials per column,
        // each added in order (the loads issued 32 at a time), the ranges added in order
        const int nh = (int)blockDim.x / Z > 0 ? (int)blockDim.x / Z : 1;
        for (int t = tid; t < nh * Z; t += blockDim.x) {
            const int c = t % Z, h = t / Z;
            const int b0 = nparts * h / nh, b1 = nparts * (h + 1) / nh;
            const double *src = part + (size_t)i * Z + c;
            double sum = 0.0;
            for (int b = b0; b < b1; b += 32) {
                double v[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = b + q < b1 ? __ldg(src + (size_t)(b + q) * Z * Z) : 0.0;
#pragma unroll
                for (int q = 0; q < 32; ++q) sum += v[q];
            }
            half[t] = sum;
        }
        __syncthreads();
        for (int c = tid; c < Z; c += blockDim.x) {
            double sum = 0.0;
            for (int h = 0; h < nh; ++h) sum += half[h * Z + c];
            G[i * Z + c] = sum;
            Gf[i * Z + c] = (float)sum;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the FP64 matrix reaches shared memory by asynchronous copies while the FP32
    // factor runs (waited for before the first residual or the fallback)
    for (int e = tid; e < Z * Z / 2; e += blockDim.x) refit_cp16(A + 2 * e, G + 2 * e);
    refit_cp_commit();
    if (tid == 0) {
        *count = 0u;
        s_singular = 0;
    }
    for (int j = tid; j < P; j += blockDim.x) {
        double s = 0.0;
        if (j < n1) {
            const double d = __ldcg(G + j * Z + j);
            const float df = (float)d;
            s = d > 0.0 ? (df > 1e-30f && df < 1e30f ? (double)rsqrtf(df) : 1.0 / sqrt(d)) : 0.0;
            sc[j] = s;
        }
        scf[j] = (float)s;
        invf[j] = 0.f;
        colbuf[j] = colbuf[P + j] = 0.f;
    }
    __syncthreads();

    // ---- FP32 factor of the scaled matrix over register tiles ----
    // Thread t owns the lower-triangle tile (R, C), R >= C, of side T; tiles are
    // numbered column by column, so the threads of finished tile columns idle
    // together. Rows and columns past U are zero. Column j of the trailing matrix is
    // published in colbuf (two buffers, alternating): at step j every thread takes
    // the pivot d = colbuf[j], writes l = colbuf / sqrt(d) into column j of its tile
    // and subtracts l_r l_c from its entries (r, c), r >= c > j; the owners of column
    // j + 1 then publish it. The factor's diagonal is kept as its reciprocal invf.
    int R = NT, C = NT;
    {
        int rem = tid, c = 0;
        while (c < NT && rem >= NT - c) {
            rem -= NT - c;
            ++c;
        }
        if (c < NT) {
            C = c;
            R = c + rem;
        }
    }
    const bool own = C < NT;
    float a[T][T];
#pragma unroll
    for (int ii = 0; ii < T; ++ii)
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int r = R * T + ii, c = C * T + k;
            float v = 0.f;
            if (own && r < n1 && c < n1 && r >= c)
                v = (r == c && scf[r] == 0.f) ? 1.f : __ldcg(Gf + r * Z + c) * scf[r] * scf[c];
            a[ii][k] = v;
        }
    if (own && C == 0)
#pragma unroll
        for (int ii = 0; ii < T; ++ii) colbuf[R * T + ii] = a[ii][0];
    __syncthreads();
    bool fb = false;   // the same in every thread: each decision reads the same shared values
    for (int j = 0; j < n1; ++j) {
        const float *cb = colbuf + (j & 1) * P;
        const float d = cb[j];
        if (!(d > 1e-5f)) {
            fb = true;
            break;
        }
        const float s = rsqrtf(d);
        if (tid == 0) invf[j] = s;
        if (own && C * T + T > j) {
            // branch-free: rows r <= j and columns c <= j of the tile get zero factors
            // (the entries above a diagonal tile's diagonal are never read)
            const int kj = j - C * T;   // column j's place in this tile column, if in [0, T)
            float lr[T], lc[T];
#pragma unroll
            for (int q = 0; q < T; ++q) {
                const float vr = cb[R * T + q] * s, vc = cb[C * T + q] * s;
                lr[q] = R * T + q > j ? vr : 0.f;
                lc[q] = q > kj ? vc : 0.f;
            }
#pragma unroll
            for (int ii = 0; ii < T; ++ii)
#pragma unroll
                for (int k = 0; k < T; ++k) a[ii][k] = fmaf(-lr[ii], lc[k], a[ii][k]);
            if (kj >= 0 && kj < T)   // column j of the factor: l
#pragma unroll
                for (int ii = 0; ii < T; ++ii)
#pragma unroll
                    for (int k = 0; k < T; ++k) a[ii][k] = k == kj ? lr[ii] : a[ii][k];
            const int k1 = kj + 1;
            if (k1 >= 0 && k1 < T) {   // publish column j + 1 (rows > j)
                float *nb = colbuf + ((j + 1) & 1) * P;
#pragma unroll
                for (int ii = 0; ii < T; ++ii) {
                    float v = a[ii][0];
#pragma unroll
                    for (int k = 1; k < T; ++k) v = k == k1 ? a[ii][k] : v;
                    if (R * T + ii > j) nb[R * T + ii] = v;
                }
            }
        }
        __syncthreads();
    }
    if (!fb) {
        // ---- FP64 iterative refinement: z += (L L^T)^{-1} S (b - A S z) ----
        double bm = 0.0;
        for (int r = tid; r < P; r += blockDim.x) {
            double rs = 0.0;
            if (r < n1) {
                rs = sc[r] * __ldcg(G + r * Z + n1);
                xv[r] = 0.0;
                bm = fmax(bm, fabs(rs));
            }
            yf[r] = (float)rs;
        }
        bm = warp_max(bm);
        if (lane == 0) half[64 + warp] = bm;
        refit_cp_wait();
        __syncthreads();
        double bmax = 0.0;
        for (int w = 0; w < nwarps; ++w) bmax = fmax(bmax, half[64 + w]);
        bool conv = false;
        for (int it = 0; it < 6 && !conv; ++it) {
            refit_tile_solve<T, NT>(a, own, R, C, yf, invf);
            for (int r = tid; r < n1; r += blockDim.x) {   // z += y; x = S z into inv_d
                const double z = xv[r] + (double)yf[r];
                xv[r] = z;
                inv_d[r] = sc[r] * z;
            }
            __syncthreads();
            double rmax = 0.0, xmax = 0.0;
            for (int r0 = 0; r0 < n1; r0 += (int)blockDim.x >> 1) {   // S (b - A x), two threads a row
                const int r = r0 + (tid >> 1);   // the same trip count in every lane (the shuffle)
                double acc = 0.0;
                if (r < n1)
                    for (int c = tid & 1; c < n1; c += 2) acc = fma(A[r * Z + c], inv_d[c], acc);
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                if (r < n1 && (tid & 1) == 0) {
                    const double rs = sc[r] * (A[r * Z + n1] - acc);
                    yf[r] = (float)rs;
                    rmax = fmax(rmax, fabs(rs));
                    xmax = fmax(xmax, fabs(xv[r]));
                }
            }
            rmax = warp_max(rmax);
            xmax = warp_max(xmax);
            if (lane == 0) {
                half[2 * warp] = rmax;
                half[2 * warp + 1] = xmax;
            }
            __syncthreads();
            rmax = xmax = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                rmax = fmax(rmax, half[2 * w]);
                xmax = fmax(xmax, half[2 * w + 1]);
            }
            conv = rmax <= 1e-12 * (bmax + xmax);
        }
        if (conv) {
            for (int r = tid; r < n1; r += blockDim.x) {
                const float v = (float)inv_d[r];
                const int p = r < U ? ow3 + r : ob3;
                params[p] = v;
                if (params2) params2[p] = v;
            }
            return;
        }
    }

    // ---- FP64 Cholesky and triangular solves of the scaled system (the fallback) ----
    refit_cp_wait();
    __syncthreads();
    for (int e = tid; e < n1 * (n1 + 1); e += blockDim.x) {
        const int r = e / (n1 + 1), c = e % (n1 + 1);
        A[r * Z + c] = (r == c && sc[r] == 0.0) ? 1.0 : A[r * Z + c] * sc[r] * (c < n1 ? sc[c] : 1.0);
    }
    __syncthreads();
    // lower Cholesky factor in place, one barrier per column. Every thread takes
    // column j's pivot d and 1/sqrt(d) by two Newton-Raphson steps
    // y <- y (3 - d y^2) / 2 from an FP32 seed (relative error 2^-22 -> 2^-44 ->
    // below FP64 rounding); the trailing lower triangle is updated from the
    // unscaled column (A[r][c] -= A[r][j] A[c][j] / d) and column j is scaled by
    // 1/sqrt(d) during the next column's step, which does not read it. Thread t
    // updates column j + 1 + (t mod U), rows c + (t / U) + k (blockDim / U). The
    // diagonal of the factor is kept as its reciprocal inv_d.
    // A pivot at or below 1e-12 of the unit diagonal means the column lies in the span
    // of the columns kept before it: it is dropped (1/sqrt(d) taken as 0, so it updates
    // nothing and its weight is 0). The fitted values, the projection of the targets on
    // the span, are the least-squares ones. A pivot that is not finite leaves the
    // parameters as they are.
    for (int j = 0; j < n1; ++j) {
        const double d = A[j * Z + j];
        const bool drop = !(d > 1e-12);
        double y = 0.0;
        if (!drop) {
            y = (double)rsqrtf((float)d);
            y = y * (1.5 - 0.5 * d * y * y);
            y = y * (1.5 - 0.5 * d * y * y);
        }
        if (tid == 0) {
            inv_d[j] = y;
            if (!isfinite(d)) s_singular = 1;
        }
        if (j > 0)
            for (int r = j + tid; r < n1; r += blockDim.x) A[r * Z + j - 1] *= inv_d[j - 1];
        const double id = y * y;
        const int c = j + 1 + (tid % U);
        if (c < n1) {
            const double lcj = A[c * Z + j] * id;
            for (int r = c + tid / U; r < n1; r += (int)blockDim.x / U) A[r * Z + c] -= A[r * Z + j] * lcj;
        }
        __syncthreads();
    }
    if (tid < 32) {   // L y = b, then L^T x = y (column-oriented, one warp)
        for (int r = lane; r < n1; r += 32) xv[r] = A[r * Z + n1];
        __syncwarp();
        for (int j = 0; j < n1; ++j) {
            const double yj = xv[j] * inv_d[j];
            __syncwarp();
            if (lane == 0) xv[j] = yj;
            for (int r = j + 1 + lane; r < n1; r += 32) xv[r] -= A[r * Z + j] * yj;
            __syncwarp();
        }
        for (int j = n1 - 1; j >= 0; --j) {
            const double xj = xv[j] * inv_d[j];
            __syncwarp();
            if (lane == 0) xv[j] = xj;
            for (int r = lane; r < j; r += 32) xv[r] -= A[j * Z + r] * xj;
            __syncwarp();
        }
        if (!s_singular)
            for (int r = lane; r < n1; r += 32) {
                const float v = (float)(xv[r] * sc[r]);
                const int p = r < U ? ow3 + r : ob3;
                params[p] = v;
                if (params2) params2[p] = v;
            }
    }
}

// Input standardisation of every date: block (f, d) computes the mean and
// 1/std (population) of factor f at date d from FP32 sums of the values less the
// date's first value (per thread), gathered in FP64 over the block. Factors
// f >= F get zeros. stats: [n_dates][mean[32] | 1/std[32]].
__global__ void __launch_bounds__(256) mlp_stats_kernel(const float *feat, int F, uint32_t M, size_t date_stride,
                                                        float *stats)
{
    __shared__ double red[2][8];
    const int f = blockIdx.x, d = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *out = stats + (size_t)d * 2 * kIn;
    if (f >= F) {
        if (tid == 0) out[f] = out[kIn + f] = 0.f;
        return;
    }
    const float *x = feat + (size_t)d * date_stride + (size_t)f * M;
    const float c = __ldg(x);
    float s1 = 0.f, s2 = 0.f;
    for (uint32_t r = 4u * tid; r < M; r += 4u * blockDim.x) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(x + r));
        const float a0 = v.x - c, a1 = v.y - c, a2 = v.z - c, a3 = v.w - c;
        s1 += (a0 + a1) + (a2 + a3);
        s2 += (a0 * a0 + a1 * a1) + (a2 * a2 + a3 * a3);
    }
    double t1 = s1, t2 = s2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    }
    if (lane == 0) {
        red[0][warp] = t1;
        red[1][warp] = t2;
    }
    __syncthreads();
    if (tid == 0) {
        double u1 = 0.0, u2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            u1 += red[0][w];
            u2 += red[1][w];
        }
        const double m1 = u1 / M, var = u2 / M - m1 * m1;
        out[f] = (float)(c + m1);
        out[kIn + f] = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.f;
    }
}

// 2-D tensor map of one date's feature array [F][M] (FP32, path index innermost):
// boxes of 128 paths x F features. The encoder is the driver's, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cva_status features_map(CUtensorMap *tm, const float *feat, int F, uint64_t M)
{
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        CVA_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (!fn || q != cudaDriverEntryPointSuccess) return fail(CVA_ECUDA, "mlp: cuTensorMapEncodeTiled not available");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)F};
    const cuuint64_t strides[1] = {(cuuint64_t)M * 4u};
    const cuuint32_t box[2] = {(cuuint32_t)kRows, (cuuint32_t)F};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(feat), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CVA_ECUDA, "mlp: tensor map encoding failed (" + std::to_string((int)r) + ")");
    return CVA_OK;
}

}  // namespace
}  // namespace cva
