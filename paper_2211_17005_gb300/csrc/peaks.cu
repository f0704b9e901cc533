// Throughput of the plain arithmetic pipes of the SMs, measured: the ceilings of
// the kernels of this library that no HBM or tensor-core limit binds (the
// path-simulation and pricing kernels run Philox integer rounds, FP32 FMAs and
// MUFU exponentials and logarithms). Each probe kernel runs eight independent
// dependency chains per thread of one instruction kind, on enough warps to fill
// every scheduler, so that the pipe's issue rate, not latency, sets its time.
#include <cuda_runtime.h>

#include "cva_internal.h"

namespace cva {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakUnroll = 16;   // iterations of the 8 chains per loop trip

// 0: fma.rn.f32 (FMA pipe); 1: lop3.b32 (ALU pipe); 2: mul.hi.u32 (the Philox
// multiply-high); 3: ex2.approx.f32 (MUFU); 4: lg2.approx.f32 (MUFU)
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(uint32_t *sink, int trips, uint32_t seed)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t u[8];
    float f[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        u[c] = seed ^ (t * 8u + (uint32_t)c);
        f[c] = 1.0f + 1e-7f * (float)(u[c] & 1023u);
    }
    const uint32_t k1 = seed | 1u, k2 = 0x9E3779B9u;
    const float fb = 0.9999999f, fc = 1e-7f;
    for (int it = 0; it < trips; ++it) {
#pragma unroll
        for (int r = 0; r < kPeakUnroll; ++r) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (KIND == 0) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(fb), "f"(fc));
                if (KIND == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[c]) : "r"(k1), "r"(k2));
                if (KIND == 2) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(u[c]) : "r"(k1 | 0x80000000u));
                if (KIND == 3) asm volatile("ex2.approx.f32 %0, %0;" : "+f"(f[c]));
                if (KIND == 4) asm volatile("lg2.approx.f32 %0, %0;" : "+f"(f[c]));
            }
        }
    }
    uint32_t acc = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc ^= u[c] ^ __float_as_uint(f[c]);
    if (acc == 0x12345678u) sink[t & 1023u] = acc;   // keeps the chains alive; practically never taken
}

template <int KIND>
cva_status time_kind(uint32_t *sink, int blocks, int trips, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                     double *lane_ops_per_s)
{
    peak_kernel<KIND><<<blocks, kPeakThreads, 0, st>>>(sink, trips, 12345u);   // warm-up
    CVA_CUDA_TRY(cudaGetLastError());
    CVA_CUDA_TRY(cudaEventRecord(e0, st));
    peak_kernel<KIND><<<blocks, kPeakThreads, 0, st>>>(sink, trips, 54321u);
    CVA_CUDA_TRY(cudaGetLastError());
    CVA_CUDA_TRY(cudaEventRecord(e1, st));
    CVA_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CVA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    const double ops = (double)blocks * kPeakThreads * trips * kPeakUnroll * 8.0;
    *lane_ops_per_s = ops / (ms * 1e-3);
    return CVA_OK;
}

}  // namespace
}  // namespace cva

using namespace cva;

extern "C" cva_status cva_pipe_peaks(double *out5_host, void *stream)
{
    if (!out5_host) return fail(CVA_EINVAL, "pipe_peaks: NULL output");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t *sink = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(uint32_t)) != cudaSuccess) return fail(CVA_ENOMEM, "pipe_peaks: sink");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cva_status r = CVA_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        r = fail(CVA_ECUDA, "pipe_peaks: events");
    const int blocks = sms * 8;   // 64 warps per SM
    if (r == CVA_OK) r = time_kind<0>(sink, blocks, 512, st, e0, e1, &out5_host[0]);
    if (r == CVA_OK) r = time_kind<1>(sink, blocks, 512, st, e0, e1, &out5_host[1]);
    if (r == CVA_OK) r = time_kind<2>(sink, blocks, 256, st, e0, e1, &out5_host[2]);
    if (r == CVA_OK) r = time_kind<3>(sink, blocks, 128, st, e0, e1, &out5_host[3]);
    if (r == CVA_OK) r = time_kind<4>(sink, blocks, 128, st, e0, e1, &out5_host[4]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return r;
}
