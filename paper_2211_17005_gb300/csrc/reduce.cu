// CVA_0 = mean over outer paths of the date-0 averaged targets (eq.
// (eq:CVA_portfolio) at i = 0), with its Monte Carlo standard error. Two-stage
// FP64 reduction with a fixed grid and a fixed tree, so the result does not
// depend on scheduling.
#include <math.h>

#include <mutex>

#include "cva_internal.h"
#include "rng.cuh"

namespace cva {

namespace {

constexpr int kRedBlocks = 304;    // 2 x 152 SMs
constexpr int kRedThreads = 256;

__device__ __forceinline__ void block_sum2(double &a, double &b, double2 *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = make_double2(a, b);
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) {
            sh[tid].x += sh[tid + s].x;
            sh[tid].y += sh[tid + s].y;
        }
        __syncthreads();
    }
    a = sh[0].x;
    b = sh[0].y;
}

__global__ void __launch_bounds__(kRedThreads) sum_stage1(const float *__restrict__ x, uint64_t M,
                                                          double2 *__restrict__ part)
{
    __shared__ double2 sh[kRedThreads];
    double s = 0.0, q = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double v = (double)__ldg(x + i);
        s += v;
        q = fma(v, v, q);
    }
    block_sum2(s, q, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s, q);
}

__global__ void __launch_bounds__(kRedThreads) sum_stage2(const double2 *__restrict__ part, int nparts,
                                                          double2 *__restrict__ out)
{
    __shared__ double2 sh[kRedThreads];
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s += part[i].x;
        q += part[i].y;
    }
    block_sum2(s, q, sh);
    if (threadIdx.x == 0) out[0] = make_double2(s, q);
}

__global__ void philox_fill(const uint4 *__restrict__ ctr, uint4 *__restrict__ out, uint64_t n,
                            uint32_t k0, uint32_t k1)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

// Twin Monte Carlo validation (Sec. ss:twin, eq. (e:val1)): per path the FP64
// term phi^2 - (xi1 + xi2) phi + xi1 xi2 of two conditionally independent copies;
// block sums of the terms and of their squares.
__global__ void __launch_bounds__(kRedThreads) twin_stage1(const float *__restrict__ phi,
                                                           const float *__restrict__ xi1,
                                                           const float *__restrict__ xi2, uint64_t M,
                                                           double2 *__restrict__ part)
{
    __shared__ double2 sh[kRedThreads];
    double s = 0.0, q = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double f = (double)__ldg(phi + i), a = (double)__ldg(xi1 + i), b = (double)__ldg(xi2 + i);
        const double t = f * f - (a + b) * f + a * b;
        s += t;
        q = fma(t, t, q);
    }
    block_sum2(s, q, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s, q);
}

// Nested Monte Carlo reference (Sec. 4.3): acc (+)= x, and on the last copy the
// mean acc / copies.
__global__ void accumulate_kernel(float *__restrict__ acc, const float *__restrict__ x, uint64_t M, int first,
                                  float scale)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (uint64_t)gridDim.x * blockDim.x) {
        const float v = first ? x[i] : acc[i] + x[i];
        acc[i] = v * scale;
    }
}

// Relative error against a reference, over the paths where the reference is not
// zero: block sums of ((phi - ref) / ref)^2 and of the number of such paths (FP64).
__global__ void __launch_bounds__(kRedThreads) relerr_stage1(const float *__restrict__ phi,
                                                             const float *__restrict__ ref, uint64_t M,
                                                             double2 *__restrict__ part)
{
    __shared__ double2 sh[kRedThreads];
    double s = 0.0, q = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double r = (double)__ldg(ref + i);
        if (r != 0.0) {
            const double e = ((double)__ldg(phi + i) - r) / r;
            s = fma(e, e, s);
            q += 1.0;
        }
    }
    block_sum2(s, q, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s, q);
}

// out[c] = sum over rows r of part[r][c], in row order (one thread per column)
__global__ void sum_cols(const double *__restrict__ part, int rows, int cols, double *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += part[(size_t)r * cols + c];
    out[c] = s;
}

std::mutex g_red_mu;
double2 *g_red_buf[64] = {};

}  // namespace

cva_status philox_blocks(const uint32_t *ctr, uint32_t *out, uint64_t n, uint64_t seed, cudaStream_t st)
{
    if (!ctr || !out) return fail(CVA_EINVAL, "philox: NULL pointer");
    if (n == 0) return CVA_OK;
    if (((uintptr_t)ctr | (uintptr_t)out) & 15) return fail(CVA_EINVAL, "philox: arrays must be 16-byte aligned");
    const uint64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffull) return fail(CVA_EINVAL, "philox: n too large");
    philox_fill<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const uint4 *>(ctr), reinterpret_cast<uint4 *>(out),
                                                  n, (uint32_t)seed, (uint32_t)(seed >> 32));
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

cva_status sum_columns_fp64(const double *part, int rows, int cols, double *out, cudaStream_t st)
{
    sum_cols<<<(cols + 127) / 128, 128, 0, st>>>(part, rows, cols, out);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

cva_status accumulate_mean(float *acc, const float *x, uint64_t M, int first, int last, int copies, cudaStream_t st)
{
    accumulate_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(acc, x, M, first, last ? 1.0f / (float)copies : 1.0f);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

// sqrt(mean over paths with ref != 0 of ((phi - ref) / ref)^2) and the number of such paths
cva_status relative_rmse_fp64(const float *phi, const float *ref, uint64_t M, double *out2, cudaStream_t st)
{
    if (!phi || !ref || !out2 || M == 0) return fail(CVA_EINVAL, "relative rmse: null pointer or M == 0");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_red_mu);
    if (!g_red_buf[dev]) {
        cudaError_t e = cudaMalloc(&g_red_buf[dev], sizeof(double2) * (kRedBlocks + 1));
        if (e != cudaSuccess) return fail(CVA_ENOMEM, "relative rmse: scratch allocation failed");
    }
    double2 *part = g_red_buf[dev];
    relerr_stage1<<<kRedBlocks, kRedThreads, 0, st>>>(phi, ref, M, part);
    CVA_CUDA_TRY(cudaGetLastError());
    sum_stage2<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, part + kRedBlocks);
    CVA_CUDA_TRY(cudaGetLastError());
    double2 h;
    CVA_CUDA_TRY(cudaMemcpyAsync(&h, part + kRedBlocks, sizeof(double2), cudaMemcpyDeviceToHost, st));
    CVA_CUDA_TRY(cudaStreamSynchronize(st));
    out2[0] = h.y > 0.0 ? sqrt(h.x / h.y) : 0.0;
    out2[1] = h.y;
    return CVA_OK;
}

// mean and standard error of the per-path twin terms (two fixed-order stages)
cva_status twin_l2_fp64(const float *phi, const float *xi1, const float *xi2, uint64_t M, double *out2,
                        cudaStream_t st)
{
    if (!phi || !xi1 || !xi2 || !out2 || M == 0) return fail(CVA_EINVAL, "twin: null pointer or M == 0");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_red_mu);
    if (!g_red_buf[dev]) {
        cudaError_t e = cudaMalloc(&g_red_buf[dev], sizeof(double2) * (kRedBlocks + 1));
        if (e != cudaSuccess) return fail(CVA_ENOMEM, "twin: scratch allocation failed");
    }
    double2 *part = g_red_buf[dev];
    twin_stage1<<<kRedBlocks, kRedThreads, 0, st>>>(phi, xi1, xi2, M, part);
    CVA_CUDA_TRY(cudaGetLastError());
    sum_stage2<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, part + kRedBlocks);
    CVA_CUDA_TRY(cudaGetLastError());
    double2 h;
    CVA_CUDA_TRY(cudaMemcpyAsync(&h, part + kRedBlocks, sizeof(double2), cudaMemcpyDeviceToHost, st));
    CVA_CUDA_TRY(cudaStreamSynchronize(st));
    const double mean = h.x / (double)M;
    double var = (M > 1) ? (h.y - (double)M * mean * mean) / (double)(M - 1) : 0.0;
    if (var < 0.0) var = 0.0;
    out2[0] = mean;
    out2[1] = sqrt(var / (double)M);
    return CVA_OK;
}

// FP64 sums (sum x, sum x^2) of M floats, two stages in a fixed order: bit-reproducible.
cva_status sums_fp64(const float *x, uint64_t M, double *sum2_host, cudaStream_t st)
{
    if (!x || !sum2_host || M == 0) return fail(CVA_EINVAL, "cva0: null pointer or M == 0");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_red_mu);
    if (!g_red_buf[dev]) {
        cudaError_t e = cudaMalloc(&g_red_buf[dev], sizeof(double2) * (kRedBlocks + 1));
        if (e != cudaSuccess) return fail(CVA_ENOMEM, "cva0: scratch allocation failed");
    }
    double2 *part = g_red_buf[dev];
    sum_stage1<<<kRedBlocks, kRedThreads, 0, st>>>(x, M, part);
    CVA_CUDA_TRY(cudaGetLastError());
    sum_stage2<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, part + kRedBlocks);
    CVA_CUDA_TRY(cudaGetLastError());
    double2 h;
    CVA_CUDA_TRY(cudaMemcpyAsync(&h, part + kRedBlocks, sizeof(double2), cudaMemcpyDeviceToHost, st));
    CVA_CUDA_TRY(cudaStreamSynchronize(st));
    sum2_host[0] = h.x;
    sum2_host[1] = h.y;
    return CVA_OK;
}

// mean and Monte Carlo standard error from (count, sum x, sum x^2)
void mean_se_from_sums(double M, double s1, double s2, double *out2)
{
    const double mean = s1 / M;
    double var = (M > 1.0) ? (s2 - M * mean * mean) / (M - 1.0) : 0.0;
    if (var < 0.0) var = 0.0;
    out2[0] = mean;
    out2[1] = sqrt(var / M);
}

cva_status mean_fp64(const float *x, uint64_t M, double *out2, cudaStream_t st)
{
    double h[2];
    cva_status r = sums_fp64(x, M, h, st);
    if (r != CVA_OK) return r;
    mean_se_from_sums((double)M, h[0], h[1], out2);
    return CVA_OK;
}

}  // namespace cva
