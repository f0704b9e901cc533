// Outer-path and inner-default kernels of the hierarchical CVA simulation.
//
// Outer kernel (one thread per outer path k, Sec. 3.2): Euler-Maruyama steps of
// the Hull-White rates, lognormal FX and CIR intensities (App. B, Remark
// rem:finecoarse), the left-point integrals int r^0 (FP64) and Lambda^c
// (compensated FP32), and at every pricing date the portfolio MtM per
// counterparty (App. B swap formula, regrouped exactly by currency and reset
// date), the exposure (1-R_c) beta_j MtM^+ and the default threshold
// 1 - exp(-Lambda_c(t_j)). All outputs are structure-of-arrays with the path
// index fastest, so each warp stores 128 contiguous bytes per field.
//
// Inner kernel (one warp per outer path, Sec. 3.2 / eq. (e:tau)): N default
// clocks per counterparty; tau^{k,l} falls in (t_{j-1}, t_j] when the uniform w
// (epsilon = -log(1 - w)) satisfies T(j-1) < w <= T(j), T = 1 - e^{-Lambda};
// the default step is the lower bound of w in the monotone thresholds. Counts
// per (counterparty, step) are integers, so the averaged target of eq.
// (eq:CVA_portfolio),
//   xi_bar_i = beta_i^{-1} (1/N) sum_{j>i} sum_c V_c(j) count_c(j),
// does not depend on the order of the draws.
#include <mutex>

#include "cva_internal.h"
#include "rng.cuh"

namespace cva {

__constant__ SimConsts c_sim;
__constant__ SimWeights c_w;

namespace {

struct OuterArgs {
    uint32_t M, k0, seed_lo, seed_hi;
    const float2 *__restrict__ zc;     // [n+1][E][G] (lnA, B)
    const float2 *__restrict__ fix;    // [periods+1][E] (lnA, B)
    const int *__restrict__ date_p;    // [n+1]
    const float *__restrict__ drift;   // [n*S][E]
    float *features, *disc, *thr, *expo, *mtm;
};

template <int E, int C, int CS, int G, int NPF>
__global__ void __launch_bounds__(128) outer_kernel(OuterArgs a)
{
    constexpr int F = 2 * E - 1 + CS;
    constexpr int NB = (F + 3) / 4;
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    if (kl >= a.M) return;
    const uint32_t k = a.k0 + kl;
    const size_t M = a.M;
    const int n = c_sim.n, S = c_sim.S, ppp = c_sim.ppp;
    const float ds = c_sim.ds;
    const double ds_d = (double)c_sim.ds_d;

    float r[E], lchi[E], fixm1[E];
    float gam[C], lam[C], lamc[C], thr_prev[C];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        r[e] = c_sim.r0[e];
        lchi[e] = c_sim.lchi0[e];
        fixm1[e] = c_sim.fix0_m1[e];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        gam[c] = c_sim.gamma0[c];
        lam[c] = 0.f;
        lamc[c] = 0.f;
        thr_prev[c] = 0.f;
    }
    double I0 = 0.0;

    // date 0
    {
#pragma unroll
        for (int e = 0; e < E; ++e) a.features[(size_t)e * M + kl] = r[e];
#pragma unroll
        for (int e = 1; e < E; ++e) a.features[(size_t)(E - 1 + e) * M + kl] = lchi[e];
#pragma unroll
        for (int c = 0; c < CS; ++c) a.features[(size_t)(2 * E - 1 + c) * M + kl] = gam[c];
        a.disc[kl] = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) a.thr[(size_t)c * M + kl] = 0.f;
#pragma unroll
        for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                a.expo[((size_t)(pf * (n + 1)) * C + c) * M + kl] = 0.f;
                if (a.mtm) a.mtm[((size_t)(pf * (n + 1)) * C + c) * M + kl] = 0.f;
            }
    }

    for (int j = 1; j <= n; ++j) {
        for (int s = 0; s < S; ++s) {
            const uint32_t q = (uint32_t)((j - 1) * S + s);
            float z[4 * NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint4 x = philox4x32_10(make_uint4(k, q, 0u, (kStreamOuter << 24) | (uint32_t)b),
                                              a.seed_lo, a.seed_hi);
                box_muller(x.x, x.y, z[4 * b], z[4 * b + 1]);
                box_muller(x.z, x.w, z[4 * b + 2], z[4 * b + 3]);
            }
            float W[F];
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int b = 0; b <= i; ++b) acc = fmaf(c_sim.L[i * (i + 1) / 2 + b], z[b], acc);
                W[i] = acc;
            }
            const float r0 = r[0];
            // left-point integrals: int r^0 in FP64, Lambda^c compensated FP32
            I0 = fma((double)r0, ds_d, I0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float gp = fmaxf(gam[c], 0.f);
                const float y = fmaf(gp, ds, -lamc[c]);
                const float t = lam[c] + y;
                lamc[c] = (t - lam[c]) - y;
                lam[c] = t;
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

        // ---- pricing date t_j ----
        const float I0f = (float)I0;
        const float beta = expf(-I0f);
        const int p = __ldg(a.date_p + j);
        float mt[NPF][C];
#pragma unroll
        for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
            for (int c = 0; c < C; ++c) mt[pf][c] = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float re = r[e];
            const float2 *tab = a.zc + ((size_t)j * E + e) * G;
            float Z[G], D[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float2 t2 = __ldg(tab + g);
                Z[g] = (g >= p) ? expf(fmaf(-t2.y, re, t2.x)) : 0.f;   // ZC_t((g+1) delta)
            }
            // D[h]: h == p -> ZC_t(t_+) (1/ZC_{t_-}(t_+) - 1); h > p -> ZC_t(h delta) - ZC_t((h+1) delta)
#pragma unroll
            for (int h = 0; h < G; ++h)
                D[h] = (h == p) ? Z[h] * fixm1[e] : ((h > p) ? Z[h - 1 >= 0 ? h - 1 : 0] - Z[h] : 0.f);
            const float chi = (e == 0) ? 1.f : expf(lchi[e]);
#pragma unroll
            for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int base = ((pf * C + c) * E + e) * G;
                    float acc = 0.f;
#pragma unroll
                    for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
#pragma unroll
                    for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                    mt[pf][c] = fmaf(chi, acc, mt[pf][c]);
                }
        }
        if (j % ppp == 0) {   // reset date: fix the next floating coupon at today's rate
            const float2 *fx = a.fix + (size_t)(j / ppp) * E;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float2 f2 = __ldg(fx + e);
                fixm1[e] = expm1f(fmaf(f2.y, r[e], -f2.x));
            }
        }

        float *fe = a.features + (size_t)j * F * M + kl;
#pragma unroll
        for (int e = 0; e < E; ++e) fe[(size_t)e * M] = r[e];
#pragma unroll
        for (int e = 1; e < E; ++e) fe[(size_t)(E - 1 + e) * M] = lchi[e];
#pragma unroll
        for (int c = 0; c < CS; ++c) fe[(size_t)(2 * E - 1 + c) * M] = gam[c];
        a.disc[(size_t)j * M + kl] = I0f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float T = fmaxf(-expm1f(-lam[c]), thr_prev[c]);
            thr_prev[c] = T;
            a.thr[((size_t)j * C + c) * M + kl] = T;
        }
#pragma unroll
        for (int pf = 0; pf < NPF; ++pf)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const size_t o = ((size_t)(pf * (n + 1) + j) * C + c) * M + kl;
                a.expo[o] = c_sim.lgd[c] * beta * fmaxf(mt[pf][c], 0.f);
                if (a.mtm) a.mtm[o] = mt[pf][c];
            }
    }
}

struct InnerArgs {
    uint32_t M, k0, seed_lo, seed_hi, N;
    int n, NPF, P;
    const float *__restrict__ thr;    // [n+1][C][M]
    const float *__restrict__ expo;   // [NPF][n+1][C][M]
    const float *__restrict__ disc;   // [n+1][M]
    float *targets;                   // [NPF][n][M]
    uint8_t *idx;                     // [M][N][C] or null
};

template <int C>
__global__ void __launch_bounds__(256) inner_kernel(InnerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int P = a.P, n = a.n, np1 = n + 1;
    float *thr_s = reinterpret_cast<float *>(smem);                 // [P][C][n+1]
    uint32_t *cnt_s = reinterpret_cast<uint32_t *>(thr_s + P * C * np1);  // [P][C][n+1]
    float *red_s = reinterpret_cast<float *>(cnt_s + P * C * np1);  // [P][n+1]
    const uint32_t M = a.M, tile0 = blockIdx.x * (uint32_t)P;
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = nthr >> 5;

    for (int i = tid; i < n * C * P; i += nthr) {
        const int pk = i % P, jc = i / P, c = jc % C, j = 1 + jc / C;
        const uint32_t kl = tile0 + pk;
        thr_s[(pk * C + c) * np1 + j] = (kl < M) ? __ldg(a.thr + ((size_t)j * C + c) * M + kl) : 2.f;
    }
    for (int i = tid; i < P * C * np1; i += nthr) cnt_s[i] = 0u;
    __syncthreads();

    for (int pk = warp; pk < P; pk += nwarps) {
        const uint32_t kl = tile0 + pk;
        if (kl >= M) continue;
        const uint32_t k = a.k0 + kl;
        for (uint32_t l = lane; l < a.N; l += 32) {
#pragma unroll
            for (int cb = 0; cb < (C + 3) / 4; ++cb) {
                const uint4 x = philox4x32_10(make_uint4(k, l, 0u, (kStreamInner << 24) | (uint32_t)cb),
                                              a.seed_lo, a.seed_hi);
                const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * cb + i;
                    if (c < C) {
                        const float w = uniform23(xs[i]);
                        const float *T = thr_s + (pk * C + c) * np1;
                        int lo = 1, len = n;      // first j in [1, n] with T[j] >= w, else n+1
                        while (len > 0) {
                            const int half = len >> 1;
                            if (T[lo + half] < w) {
                                lo += half + 1;
                                len -= half + 1;
                            } else {
                                len = half;
                            }
                        }
                        if (a.idx) a.idx[((size_t)kl * a.N + l) * C + c] = (uint8_t)lo;
                        if (lo <= n) atomicAdd(&cnt_s[(pk * C + c) * np1 + lo], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();

    const float invN = 1.0f / (float)a.N;
    for (int pf = 0; pf < a.NPF; ++pf) {
        // H[pk][j] = sum_c V_c(j) count_c(j); loads of 8 consecutive paths share a sector
        for (int i = tid; i < n * P; i += nthr) {
            const int pk = i % P, j = 1 + i / P;
            const uint32_t kl = tile0 + pk;
            float h = 0.f;
            if (kl < M) {
#pragma unroll
                for (int c = 0; c < C; ++c)
                    h = fmaf(__ldg(a.expo + ((size_t)(pf * np1 + j) * C + c) * M + kl),
                             (float)cnt_s[(pk * C + c) * np1 + j], h);
            }
            red_s[pk * np1 + j] = h;
        }
        __syncthreads();
        // suffix sums S(i) = sum_{j > i} H(j), stored at position i+1
        const int per = (n + 31) / 32;
        for (int pk = warp; pk < P; pk += nwarps) {
            float loc = 0.f;
            for (int t = 0; t < per; ++t) {
                const int j = 1 + lane * per + t;
                if (j <= n) loc += red_s[pk * np1 + j];
            }
            __syncwarp();
            float suf = loc;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float v = __shfl_down_sync(0xffffffffu, suf, off);
                if (lane + off < 32) suf += v;
            }
            float acc = suf - loc;
            for (int t = per - 1; t >= 0; --t) {
                const int j = 1 + lane * per + t;
                if (j <= n) {
                    acc += red_s[pk * np1 + j];
                    red_s[pk * np1 + j] = acc;    // = S(j-1)
                }
            }
        }
        __syncthreads();
        for (int i2 = tid; i2 < n * P; i2 += nthr) {
            const int pk = i2 % P, i = i2 / P;
            const uint32_t kl = tile0 + pk;
            if (kl < M) {
                const float disc = __ldg(a.disc + (size_t)i * M + kl);
                a.targets[((size_t)pf * n + i) * M + kl] = red_s[pk * np1 + i + 1] * expf(disc) * invN;
            }
        }
        __syncthreads();
    }
}

// Constant-memory ownership: the outer kernel reads c_sim / c_w, so a launch
// for another simulation re-uploads them, and every launch waits for the
// previous one (on whichever stream) before touching constant memory.
std::mutex g_const_mu;
const Sim *g_owner[64] = {};
cudaEvent_t g_last[64] = {};

template <int E, int C, int CS, int G, int NPF>
cudaError_t launch_outer_t(const OuterArgs &args, cudaStream_t st)
{
    const unsigned blocks = (args.M + 127u) / 128u;
    outer_kernel<E, C, CS, G, NPF><<<blocks, 128, 0, st>>>(args);
    return cudaGetLastError();
}

typedef cudaError_t (*outer_fn)(const OuterArgs &, cudaStream_t);

struct OuterInst {
    int E, C, CS, G, NPF;
    outer_fn fn;
};

const OuterInst kOuter[] = {
    {1, 2, 0, 5, 1, launch_outer_t<1, 2, 0, 5, 1>},
    {1, 2, 0, 10, 1, launch_outer_t<1, 2, 0, 10, 1>},
    {10, 8, 8, 10, 1, launch_outer_t<10, 8, 8, 10, 1>},
    {10, 8, 8, 10, 6, launch_outer_t<10, 8, 8, 10, 6>},
};

const OuterInst *find_outer(int E, int C, int CS, int G, int NPF)
{
    const OuterInst *best = nullptr;
    for (const auto &o : kOuter)
        if (o.E == E && o.C == C && o.CS == CS && o.NPF == NPF && o.G >= G && (!best || o.G < best->G))
            best = &o;
    return best;
}

}  // namespace

bool outer_supported(int E, int C, int CS, int G, int NPF, int *Ginst)
{
    const OuterInst *o = find_outer(E, C, CS, G, NPF);
    if (o && Ginst) *Ginst = o->G;
    return o != nullptr;
}

void forget_const_owner(const Sim *s)
{
    std::lock_guard<std::mutex> lk(g_const_mu);
    for (auto &o : g_owner)
        if (o == s) o = nullptr;
}

cva_status launch_outer(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    const OuterInst *o = find_outer(s.E, s.C, s.CS, s.G, s.NPF);
    if (!o || o->G != s.Ginst) return fail(CVA_ENOTSUP, "no outer kernel for this model shape");
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    OuterArgs args;
    args.M = (uint32_t)s.M;
    args.k0 = (uint32_t)k0;
    args.seed_lo = (uint32_t)seed;
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

    std::lock_guard<std::mutex> lk(g_const_mu);
    if (!g_last[dev]) CVA_CUDA_TRY(cudaEventCreateWithFlags(&g_last[dev], cudaEventDisableTiming));
    else CVA_CUDA_TRY(cudaStreamWaitEvent(st, g_last[dev], 0));
    if (g_owner[dev] != &s) {
        CVA_CUDA_TRY(cudaMemcpyToSymbolAsync(c_sim, &s.consts, sizeof(SimConsts), 0,
                                             cudaMemcpyHostToDevice, st));
        CVA_CUDA_TRY(cudaMemcpyToSymbolAsync(c_w, &s.weights, sizeof(SimWeights), 0,
                                             cudaMemcpyHostToDevice, st));
        g_owner[dev] = &s;
    }
    CVA_CUDA_TRY(o->fn(args, st));
    CVA_CUDA_TRY(cudaEventRecord(g_last[dev], st));
    return CVA_OK;
}

static size_t inner_smem(int P, int C, int n) { return (size_t)P * (n + 1) * 4 * (2 * C + 1); }

template <int C>
static cudaError_t launch_inner_t(const InnerArgs &args, size_t smem, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(inner_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned blocks = (args.M + args.P - 1) / args.P;
    inner_kernel<C><<<blocks, 32 * args.P, smem, st>>>(args);
    return cudaGetLastError();
}

cva_status launch_inner(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    InnerArgs args;
    args.M = (uint32_t)s.M;
    args.k0 = (uint32_t)k0;
    args.seed_lo = (uint32_t)seed;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.N = s.N;
    args.n = s.n;
    args.NPF = s.NPF;
    int P = 8;
    while (P > 1 && inner_smem(P, s.C, s.n) > 160 * 1024) P >>= 1;
    args.P = P;
    args.thr = s.d_thr;
    args.expo = s.d_expo;
    args.disc = s.d_disc;
    args.targets = s.d_targets;
    args.idx = s.d_idx;
    const size_t smem = inner_smem(P, s.C, s.n);
    cudaError_t e;
    switch (s.C) {
    case 1: e = launch_inner_t<1>(args, smem, st); break;
    case 2: e = launch_inner_t<2>(args, smem, st); break;
    case 4: e = launch_inner_t<4>(args, smem, st); break;
    case 8: e = launch_inner_t<8>(args, smem, st); break;
    case 16: e = launch_inner_t<16>(args, smem, st); break;
    default: return fail(CVA_ENOTSUP, "inner kernel compiled for C in {1, 2, 4, 8, 16}");
    }
    if (e != cudaSuccess) return cuda_fail(e, "inner_kernel launch");
    return CVA_OK;
}

}  // namespace cva
