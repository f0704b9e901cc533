// Outer-path kernels of the hierarchical CVA simulation, templated on the model
// shape. Each translation unit that includes this header gets its own copy of
// the constant-memory tables and of their ownership state, so instantiations
// compile in parallel.
//
// sim_kernel (one thread per outer path k, Sec. 3.2): the time loop. Per
// Euler-Maruyama sub-step (Remark rem:finecoarse): Philox normals, correlation
// by the Cholesky factor, Hull-White rates with the quanto drift, lognormal FX,
// CIR intensities with full truncation (App. B), and the left-point integrals
// int r^0 (FP64) and Lambda^c (compensated FP32). At each pricing date it
// stores the state Y_j, int r^0 and the threshold 1 - exp(-Lambda_c(t_j)).
//
// price_kernel (one thread per outer path, pricing date and portfolio): the
// portfolio MtM per counterparty from the App. B swap formula, regrouped exactly by
// (counterparty, currency, reset date), and the exposure (1-R_c) beta_j MtM^+.
// It reads the state of date j and the short rates of the last reset date
// (Remark rem:pathdep) from the stored states; every (path, date) is
// independent, so the pricing runs at full occupancy.
//
// Outputs are structure-of-arrays with the path index fastest.
#pragma once
#include <algorithm>
#include <mutex>

#include "cva_internal.h"
#include "rng.cuh"
#include "umma.cuh"

namespace cva {
namespace {

static __constant__ SimConsts c_sim;
static __constant__ SimWeights c_w;

// expm1(x) by its Taylor series to degree 8 for |x| <= 1/4 (relative error below
// 2e-10 there, so the rounding of the FMAs dominates), library expm1f elsewhere.
__device__ __forceinline__ float expm1_small(float x)
{
    if (fabsf(x) > 0.25f) return expm1f(x);
    float p = 1.f / 40320.f;
    p = fmaf(p, x, 1.f / 5040.f);
    p = fmaf(p, x, 1.f / 720.f);
    p = fmaf(p, x, 1.f / 120.f);
    p = fmaf(p, x, 1.f / 24.f);
    p = fmaf(p, x, 1.f / 6.f);
    p = fmaf(p, x, 0.5f);
    p = fmaf(p, x, 1.f);
    return p * x;
}

struct OuterArgs {
    uint32_t M, k0, seed_lo, seed_hi;
    int branch_date;                   // steps j > branch_date draw with counter word `branch`
    uint32_t branch;
    const float4 *__restrict__ zc;     // [n+1][E][G] (lnA, B, dlnA, dB)
    const float2 *__restrict__ fix;    // [periods+1][E] (lnA, B)
    const int *__restrict__ date_p;    // [n+1]
    const float *__restrict__ drift;   // [n*S][E]
    float *features, *disc, *thr, *expo, *mtm;
    const float *w_glob;               // device copy of the date-bucketed weights: wA [kMaxW], then wK [kMaxW]
};

template <int E, int C, int CS>
__global__ void __launch_bounds__(128) sim_kernel(OuterArgs a)
{
    constexpr int F = 2 * E - 1 + CS;
    constexpr int NB = (F + 3) / 4;
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    if (kl >= a.M) return;
    const uint32_t k = a.k0 + kl;
    const size_t M = a.M;
    const int n = c_sim.n, S = c_sim.S;
    const float ds = c_sim.ds;
    const double ds_d = c_sim.ds_d;

    float r[E], lchi[E];
    float gam[C], lam[C], lamc[C];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        r[e] = c_sim.r0[e];
        lchi[e] = c_sim.lchi0[e];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        gam[c] = c_sim.gamma0[c];
        lam[c] = 0.f;
        lamc[c] = 0.f;
    }
    double I0 = 0.0;

    // date 0
#pragma unroll
    for (int e = 0; e < E; ++e) a.features[(size_t)e * M + kl] = r[e];
#pragma unroll
    for (int e = 1; e < E; ++e) a.features[(size_t)(E - 1 + e) * M + kl] = lchi[e];
#pragma unroll
    for (int c = 0; c < CS; ++c) a.features[(size_t)(2 * E - 1 + c) * M + kl] = gam[c];
    a.disc[kl] = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) a.thr[(size_t)c * M + kl] = 0.f;

    for (int j = 1; j <= n; ++j) {
        for (int s = 0; s < S; ++s) {
            const uint32_t q = (uint32_t)((j - 1) * S + s);
            // correlated increments W = L z, accumulated one Philox block (four
            // normals) at a time
            float W[F];
#pragma unroll
            for (int i = 0; i < F; ++i) W[i] = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint4 x = philox4x32_10(
                    make_uint4(k, q, j > a.branch_date ? a.branch : 0u, (kStreamOuter << 24) | (uint32_t)b), a.seed_lo,
                    a.seed_hi);
                float z[4];
                box_muller(x.x, x.y, z[0], z[1]);
                box_muller(x.z, x.w, z[2], z[3]);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int col = 4 * b + t;
                    if (col < F) {
#pragma unroll
                        for (int i = col; i < F; ++i) W[i] = fmaf(c_sim.L[i * (i + 1) / 2 + col], z[t], W[i]);
                    }
                }
            }
            const float r0 = r[0];
            // left-point integrals: int r^0 in FP64, Lambda^c compensated FP32 and
            // kept non-decreasing
            I0 = fma((double)r0, ds_d, I0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float gp = fmaxf(gam[c], 0.f);
                const float y = fmaf(gp, ds, -lamc[c]);
                const float t = lam[c] + y;
                lamc[c] = (t - lam[c]) - y;
                lam[c] = fmaxf(t, lam[c]);
                if (c < CS) {
                    constexpr int w0 = (CS > 0) ? 2 * E - 1 : 0;
                    gam[c] += c_sim.cir_ktds[c] - c_sim.cir_kds[c] * gp
                              + c_sim.cir_nu_sqds[c] * sqrtf(gp) * W[w0 + (c < CS ? c : 0)];
                }
            }
            const float *drow = a.drift + (size_t)q * E;
#pragma unroll
            for (int e = 1; e < E; ++e)
                lchi[e] += fmaf(r0 - r[e], ds, c_sim.fx_drift_ds[e]) + c_sim.fx_sig_sqds[e] * W[E - 1 + e];
#pragma unroll
            for (int e = 0; e < E; ++e)
                r[e] += (__ldg(drow + e) - c_sim.hw_a_ds[e] * r[e]) + c_sim.hw_sig_sqds[e] * W[e];
        }

        float *fe = a.features + (size_t)j * F * M + kl;
#pragma unroll
        for (int e = 0; e < E; ++e) fe[(size_t)e * M] = r[e];
#pragma unroll
        for (int e = 1; e < E; ++e) fe[(size_t)(E - 1 + e) * M] = lchi[e];
#pragma unroll
        for (int c = 0; c < CS; ++c) fe[(size_t)(2 * E - 1 + c) * M] = gam[c];
        a.disc[(size_t)j * M + kl] = (float)I0;
#pragma unroll
        for (int c = 0; c < C; ++c) a.thr[((size_t)j * C + c) * M + kl] = -expm1f(-lam[c]);
    }
}

// NPB portfolios per block (blockIdx.z picks the group): the bond prices of a
// (path, date) serve the group's portfolios, and the group's date-bucketed weights
// (NPB C E G pairs) must stay within the constant cache; the autotuner chooses NPB.
template <int E, int C, int CS, int G, int NPB>
__global__ void __launch_bounds__(256) price_kernel(OuterArgs a)
{
    constexpr int F = 2 * E - 1 + CS;
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, pf0 = blockIdx.z * NPB;
    if (kl >= a.M) return;
    const size_t M = a.M;
    const int n = c_sim.n, ppp = c_sim.ppp;
    if (j == 0) {   // no default at t_0: exposures of date 0 are never used
#pragma unroll
        for (int pb = 0; pb < NPB; ++pb)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                a.expo[((size_t)((pf0 + pb) * (n + 1)) * C + c) * M + kl] = 0.f;
                if (a.mtm) a.mtm[((size_t)((pf0 + pb) * (n + 1)) * C + c) * M + kl] = 0.f;
            }
        return;
    }
    const int p = __ldg(a.date_p + j);          // t_j in (p delta, (p+1) delta]
    const float *fe = a.features + (size_t)j * F * M + kl;
    const float *ffix = a.features + (size_t)(p * ppp) * F * M + kl;   // state at the last reset
    const float2 *fx = a.fix + (size_t)p * E;
    const float beta = expf(-__ldg(a.disc + (size_t)j * M + kl));

    float mt[NPB][C];
#pragma unroll
    for (int pb = 0; pb < NPB; ++pb)
#pragma unroll
        for (int c = 0; c < C; ++c) mt[pb][c] = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const float re = __ldg(fe + (size_t)e * M);
        // running floating coupon fixed at t_- = p delta: 1/ZC_{t_-}(t_+) - 1
        const float2 f2 = __ldg(fx + e);
        const float fixm1 = expm1f(fmaf(f2.y, __ldg(ffix + (size_t)e * M), -f2.x));
        const float4 *tab = a.zc + ((size_t)j * E + e) * G;
        // Z[g] = ZC_t((g+1) delta) for live reset dates (g >= p), chained from the
        // first one: Z[g] = Z[g-1] (1 + expm1(x_g)), x_g = ln ZC_t((g+1) delta) -
        // ln ZC_t(g delta). D[h] = ZC_t(h delta) - ZC_t((h+1) delta) = -Z[h-1] expm1(x_h)
        // keeps full relative accuracy of each bond-price difference; D[p] carries the
        // running floating coupon ZC_t(t_+) (1/ZC_{t_-}(t_+) - 1).
        const float4 tp = __ldg(tab + (p < G ? p : G - 1));   // p >= G: every swap has matured
        const float z_first = expf(fmaf(-tp.y, re, tp.x));
        float Z[G], D[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < p) {
                Z[g] = 0.f;
                D[g] = 0.f;
            } else if (g == p) {
                Z[g] = z_first;
                D[g] = z_first * fixm1;
            } else {
                const float4 t4 = __ldg(tab + g);
                const float zp = Z[g > 0 ? g - 1 : 0];
                const float em = expm1_small(fmaf(-t4.w, re, t4.z));
                D[g] = -zp * em;
                Z[g] = fmaf(zp, em, zp);
            }
        }
        const float chi = (e == 0) ? 1.f : expf(__ldg(fe + (size_t)(E - 1 + (e > 0 ? e : 1)) * M));
#pragma unroll
        for (int pb = 0; pb < NPB; ++pb)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int base = (((pf0 + pb) * C + c) * E + e) * G;
                float acc = 0.f;
#pragma unroll
                for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
#pragma unroll
                for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                mt[pb][c] = fmaf(chi, acc, mt[pb][c]);
            }
    }
#pragma unroll
    for (int pb = 0; pb < NPB; ++pb)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const size_t o = ((size_t)((pf0 + pb) * (n + 1) + j) * C + c) * M + kl;
            a.expo[o] = c_sim.lgd[c] * beta * fmaxf(mt[pb][c], 0.f);
            if (a.mtm) a.mtm[o] = mt[pb][c];
        }
}

// Every portfolio of the simulation priced by one thread, for PT outer paths of a
// pricing date at a time, with the date-bucketed weights staged once per block in
// shared memory: each (path, date) computes its bond prices once for all
// portfolios, and each weight, read with one broadcast load, feeds the thread's PT
// paths. The state of the next economy is requested while the current one is
// priced. The FMA order per path is price_kernel's, so the outputs are the same bits.
// Block: 256 / PT threads = paths [256 b, 256 b + 256) (thread t takes t + u 256/PT,
// u < PT), dates [dpb y, dpb y + dpb). Shared memory: NPF C E GP float2 (wA, wK)
// pairs, GP = G rounded up to even so that every row of pairs is 16-byte aligned.
template <int E, int C, int CS, int G, int NPF, int PT>
__global__ void __launch_bounds__(256 / PT, 2) price_smem_kernel(OuterArgs a, int dates_per_block)
{
    constexpr int F = 2 * E - 1 + CS, GP = (G + 1) / 2 * 2, NPAIR = NPF * C * E * GP, NT = 256 / PT;
    extern __shared__ float4 price_smem[];
    float2 *wsm = reinterpret_cast<float2 *>(price_smem);
    for (int i = threadIdx.x; i < NPAIR; i += blockDim.x) {
        const int h = i % GP, row = i / GP;   // row = (pf C + c) E + e
        wsm[i] = h < G ? make_float2(__ldg(a.w_glob + row * G + h), __ldg(a.w_glob + kMaxW + row * G + h))
                       : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const size_t M = a.M;
    const int n = c_sim.n, ppp = c_sim.ppp;
    uint32_t kk[PT];
    bool has[PT];
#pragma unroll
    for (int t = 0; t < PT; ++t) {
        const uint32_t k = blockIdx.x * 256u + (uint32_t)(t * NT) + threadIdx.x;
        has[t] = k < a.M;
        kk[t] = has[t] ? k : (blockIdx.x * 256u + threadIdx.x < a.M ? blockIdx.x * 256u + threadIdx.x : 0u);
    }
    if (!has[0]) return;
    const int j0 = (int)blockIdx.y * dates_per_block;
    for (int j = j0; j < j0 + dates_per_block && j <= n; ++j) {
        if (j == 0) {   // no default at t_0: exposures of date 0 are never used
#pragma unroll
            for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int t = 0; t < PT; ++t) {
                        if (!has[t]) continue;
                        const size_t o = ((size_t)(pf * (n + 1)) * C + c) * M + kk[t];
                        a.expo[o] = 0.f;
                        if (a.mtm) a.mtm[o] = 0.f;
                    }
            continue;
        }
        const int p = __ldg(a.date_p + j);          // t_j in (p delta, (p+1) delta]
        const float2 *fx = a.fix + (size_t)p * E;
        const float *fe = a.features + (size_t)j * F * M;
        const float *ffix = a.features + (size_t)(p * ppp) * F * M;   // state at the last reset
        float beta[PT], mt[PT][NPF][C];
        float nre[PT], nfix[PT], nchi[PT];   // the next economy's state, requested one economy ahead
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            beta[t] = expf(-__ldg(a.disc + (size_t)j * M + kk[t]));
            nre[t] = __ldg(fe + kk[t]);
            nfix[t] = __ldg(ffix + kk[t]);
            nchi[t] = 0.f;
#pragma unroll
            for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
                for (int c = 0; c < C; ++c) mt[t][pf][c] = 0.f;
        }
#pragma unroll 1
        for (int e = 0; e < E; ++e) {
            float re[PT], rfix[PT], lchi[PT];
#pragma unroll
            for (int t = 0; t < PT; ++t) {
                re[t] = nre[t];
                rfix[t] = nfix[t];
                lchi[t] = nchi[t];
                if (e + 1 < E) {
                    nre[t] = __ldg(fe + (size_t)(e + 1) * M + kk[t]);
                    nfix[t] = __ldg(ffix + (size_t)(e + 1) * M + kk[t]);
                    nchi[t] = __ldg(fe + (size_t)(E + e) * M + kk[t]);   // log chi^{e+1}
                }
            }
            const float2 f2 = __ldg(fx + e);
            const float4 *tab = a.zc + ((size_t)j * E + e) * G;
            const float4 tp = __ldg(tab + (p < G ? p : G - 1));   // p >= G: every swap has matured
            float Z[PT][G], D[PT][G], chi[PT];
#pragma unroll
            for (int t = 0; t < PT; ++t) {
                const float fixm1 = expm1f(fmaf(f2.y, rfix[t], -f2.x));
                const float z_first = expf(fmaf(-tp.y, re[t], tp.x));
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (g < p) {
                        Z[t][g] = 0.f;
                        D[t][g] = 0.f;
                    } else if (g == p) {
                        Z[t][g] = z_first;
                        D[t][g] = z_first * fixm1;
                    } else {
                        const float4 t4 = __ldg(tab + g);
                        const float zp = Z[t][g > 0 ? g - 1 : 0];
                        const float em = expm1_small(fmaf(-t4.w, re[t], t4.z));
                        D[t][g] = -zp * em;
                        Z[t][g] = fmaf(zp, em, zp);
                    }
                }
                chi[t] = (e == 0) ? 1.f : expf(lchi[t]);
            }
#pragma unroll
            for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 *wr = reinterpret_cast<const float4 *>(wsm + ((pf * C + c) * E + e) * GP);
                    float wa[GP], wk[GP];
#pragma unroll
                    for (int q = 0; q < GP / 2; ++q) {
                        const float4 w4 = wr[q];
                        wa[2 * q] = w4.x;
                        wk[2 * q] = w4.y;
                        wa[2 * q + 1] = w4.z;
                        wk[2 * q + 1] = w4.w;
                    }
#pragma unroll
                    for (int t = 0; t < PT; ++t) {
                        float acc = 0.f;
#pragma unroll
                        for (int h = 0; h < G; ++h) acc = fmaf(wa[h], D[t][h], acc);
#pragma unroll
                        for (int g = 0; g < G; ++g) acc = fmaf(-wk[g], Z[t][g], acc);
                        mt[t][pf][c] = fmaf(chi[t], acc, mt[t][pf][c]);
                    }
                }
        }
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            if (!has[t]) continue;
#pragma unroll
            for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const size_t o = ((size_t)(pf * (n + 1) + j) * C + c) * M + kk[t];
                    a.expo[o] = c_sim.lgd[c] * beta[t] * fmaxf(mt[t][pf][c], 0.f);
                    if (a.mtm) a.mtm[o] = mt[t][pf][c];
                }
        }
    }
}

#include "price_tc.cuh"

}  // namespace
}  // namespace cva

#include "adjoint.cuh"

namespace cva {
namespace {

// Constant-memory ownership of this translation unit: a launch for another
// simulation re-uploads the tables, and every launch first waits for the
// previous one (on whichever stream) before constant memory can change.
static std::mutex t_const_mu;
static const Sim *t_owner[64] = {};
static cudaEvent_t t_last[64] = {};

static cudaError_t upload_consts(const Sim &s, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyToSymbolAsync(c_sim, s.d_const_img, sizeof(SimConsts), 0, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_w, s.d_const_img + sizeof(SimConsts), sizeof(SimWeights), 0,
                                   cudaMemcpyDeviceToDevice, st);
}

static void outer_forget(const Sim *s)
{
    std::lock_guard<std::mutex> lk(t_const_mu);
    for (auto &o : t_owner)
        if (o == s) o = nullptr;
}

template <int E, int C, int CS, int G, int NPF>
cva_status outer_launch(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    OuterArgs args;
    args.M = (uint32_t)s.M;
    args.k0 = (uint32_t)k0;
    args.seed_lo = (uint32_t)seed;
    args.branch_date = s.branch_date;
    args.branch = s.branch;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.zc = s.d_zc;
    args.fix = s.d_fix;
    args.date_p = s.d_date_p;
    args.drift = s.d_drift;
    args.features = s.d_features;
    args.disc = s.d_disc;
    args.thr = s.d_thr;
    args.expo = s.d_expo;
    args.mtm = s.d_mtm;
    args.w_glob = reinterpret_cast<const float *>(s.d_const_img + sizeof(SimConsts));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CVA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lk(t_const_mu);
    if (capturing) {
        // a captured graph uploads its own tables every time it runs
        CVA_CUDA_TRY(upload_consts(s, st));
        t_owner[dev] = nullptr;
    } else {
        if (!t_last[dev]) CVA_CUDA_TRY(cudaEventCreateWithFlags(&t_last[dev], cudaEventDisableTiming));
        else CVA_CUDA_TRY(cudaStreamWaitEvent(st, t_last[dev], 0));
        if (t_owner[dev] != &s) {
            CVA_CUDA_TRY(upload_consts(s, st));
            t_owner[dev] = &s;
        }
    }
    const unsigned sb = (unsigned)(s.tune_sim_block > 0 && s.tune_sim_block <= 128 ? s.tune_sim_block : 128);
    const unsigned pb = (unsigned)(s.tune_price_block > 0 && s.tune_price_block <= 256 ? s.tune_price_block : 256);
    sim_kernel<E, C, CS><<<(args.M + sb - 1) / sb, sb, 0, st>>>(args);
    CVA_CUDA_TRY(cudaGetLastError());
    if (s.ev[1]) CVA_CUDA_TRY(cudaEventRecord(s.ev[1], st));
    if (s.tune_price_pf == 4) {   // every portfolio per 128-path tile on the tensor cores
        using PT = PriceTc<E, G, NPF, C>;
        static bool attr[64] = {};
        if (!attr[dev]) {
            if (capturing) return fail(CVA_EINVAL, "price: run once before capturing (kernel attribute)");
            CVA_CUDA_TRY(cudaFuncSetAttribute(price_tc_kernel<E, C, CS, G, NPF>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, PT::bytes));
            attr[dev] = true;
        }
        int sms = 0;
        CVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const uint32_t tiles = (args.M + 127u) / 128u;
        const uint64_t items = (uint64_t)tiles * (uint64_t)(s.n + 1);
        const unsigned grid =
            (unsigned)std::min<uint64_t>((items + kPriceSlots - 1) / kPriceSlots, (uint64_t)sms);
        price_tc_kernel<E, C, CS, G, NPF><<<grid, 128 * kPriceSlots, PT::bytes, st>>>(args, tiles);
        CVA_CUDA_TRY(cudaGetLastError());
        if (!capturing) CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
        return CVA_OK;
    }
    if (s.tune_price_pf == 0) {   // every portfolio per thread, weights in shared memory
        constexpr int GP = (G + 1) / 2 * 2;
        constexpr size_t smem = (size_t)NPF * C * E * GP * sizeof(float2);
        static_assert(smem <= 48 * 1024, "portfolio weights exceed the default shared-memory limit");
        const int dpb = 8;
        const dim3 sgrid((args.M + 255u) / 256u, (unsigned)((s.n + 1 + dpb - 1) / dpb));
        if (pb == 256) price_smem_kernel<E, C, CS, G, NPF, 1><<<sgrid, 256, smem, st>>>(args, dpb);
        else price_smem_kernel<E, C, CS, G, NPF, 2><<<sgrid, 128, smem, st>>>(args, dpb);
        CVA_CUDA_TRY(cudaGetLastError());
        if (!capturing) CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
        return CVA_OK;
    }
    const int ppb = ((s.tune_price_pf == 2 || s.tune_price_pf == 3) && NPF % s.tune_price_pf == 0) ? s.tune_price_pf : 1;
    const dim3 pgrid((args.M + pb - 1) / pb, (unsigned)s.n + 1u, (unsigned)(NPF / ppb));
    if constexpr (NPF % 3 == 0) {
        if (ppb == 3) price_kernel<E, C, CS, G, 3><<<pgrid, pb, 0, st>>>(args);
    }
    if constexpr (NPF % 2 == 0) {
        if (ppb == 2) price_kernel<E, C, CS, G, 2><<<pgrid, pb, 0, st>>>(args);
    }
    if (ppb == 1) price_kernel<E, C, CS, G, 1><<<pgrid, pb, 0, st>>>(args);
    CVA_CUDA_TRY(cudaGetLastError());
    if (!capturing) CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
    return CVA_OK;
}

template <int E, int C, int CS, int G>
cva_status adjoint_launch(Sim &s, const AdjBuffers &b, uint64_t seed, uint64_t k0, uint32_t M, cudaStream_t st)
{
    constexpr int KMAX = 16, SMAX = 4;
    if (b.K < 1 || b.K > KMAX || s.S > SMAX) return fail(CVA_ENOTSUP, "adjoint: checkpoint interval <= 16, sub-steps <= 4");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    AdjArgs a;
    a.M = M;
    a.k0 = (uint32_t)k0;
    a.seed_lo = (uint32_t)seed;
    a.seed_hi = (uint32_t)(seed >> 32);
    a.K = b.K;
    a.nseg = b.nseg;
    a.forward_only = b.forward_only;
    a.zc = s.d_zc;
    a.fix = s.d_fix;
    a.date_p = s.d_date_p;
    a.drift = s.d_drift;
    a.dzc = b.dzc;
    a.dfix = b.dfix;
    a.ddrift = b.ddrift;
    a.rho = b.rho;
    a.sig = b.sig;
    a.ckpt = b.ckpt;
    a.ckpt_I0 = b.ckpt_I0;
    a.fixr = b.fixr;
    a.part = b.part;
    std::lock_guard<std::mutex> lk(t_const_mu);
    if (!t_last[dev]) CVA_CUDA_TRY(cudaEventCreateWithFlags(&t_last[dev], cudaEventDisableTiming));
    else CVA_CUDA_TRY(cudaStreamWaitEvent(st, t_last[dev], 0));
    if (t_owner[dev] != &s) {
        CVA_CUDA_TRY(upload_consts(s, st));
        t_owner[dev] = &s;
    }
    adjoint_kernel<E, C, CS, G, KMAX, SMAX><<<(M + 127u) / 128u, 128, 0, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
    return CVA_OK;
}

}  // namespace
}  // namespace cva
