// Outer-path kernels for any model shape within the library's limits (E <= 16
// economies, C <= 16 counterparties with CIR and constant intensities in any order,
// up to 6 portfolios): the model's sizes are run-time values and the per-path
// state lives in arrays sized at those limits. The arithmetic, and its order, is
// that of sim_kernel and price_kernel (outer.cuh), so a shape that also has a
// compiled instantiation gives the same bits on either; the compiled ones stay the
// fast paths. The stochastic intensity of counterparty c is state factor
// c_sim.gpos[c] (the factors are r^0..r^{E-1}, log chi^1..log chi^{E-1}, then the
// CIR intensities in counterparty order), or -1 for a constant intensity.
#include "outer.cuh"

namespace cva {
namespace {

__global__ void __launch_bounds__(128) sim_generic_kernel(OuterArgs a)
{
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    if (kl >= a.M) return;
    const uint32_t k = a.k0 + kl;
    const size_t M = a.M;
    const int E = c_sim.E, C = c_sim.C, F = c_sim.F, n = c_sim.n, S = c_sim.S;
    const int NB = (F + 3) / 4;
    const float ds = c_sim.ds;
    const double ds_d = c_sim.ds_d;

    float r[kMaxE], lchi[kMaxE], W[kMaxF];
    float gam[kMaxC], lam[kMaxC], lamc[kMaxC];
    for (int e = 0; e < E; ++e) {
        r[e] = c_sim.r0[e];
        lchi[e] = c_sim.lchi0[e];
    }
    for (int c = 0; c < C; ++c) {
        gam[c] = c_sim.gamma0[c];
        lam[c] = 0.f;
        lamc[c] = 0.f;
    }
    double I0 = 0.0;

    auto store_state = [&](int j) {
        float *fe = a.features + (size_t)j * F * M + kl;
        for (int e = 0; e < E; ++e) fe[(size_t)e * M] = r[e];
        for (int e = 1; e < E; ++e) fe[(size_t)(E - 1 + e) * M] = lchi[e];
        for (int c = 0; c < C; ++c)
            if (c_sim.gpos[c] >= 0) fe[(size_t)c_sim.gpos[c] * M] = gam[c];
    };
    store_state(0);
    a.disc[kl] = 0.f;
    for (int c = 0; c < C; ++c) a.thr[(size_t)c * M + kl] = 0.f;

    for (int j = 1; j <= n; ++j) {
        for (int s = 0; s < S; ++s) {
            const uint32_t q = (uint32_t)((j - 1) * S + s);
            // correlated increments W = L z, one Philox block (four normals) at a time
            for (int i = 0; i < F; ++i) W[i] = 0.f;
            for (int b = 0; b < NB; ++b) {
                const uint4 x = philox4x32_10(
                    make_uint4(k, q, j > a.branch_date ? a.branch : 0u, (kStreamOuter << 24) | (uint32_t)b), a.seed_lo,
                    a.seed_hi);
                float z[4];
                box_muller(x.x, x.y, z[0], z[1]);
                box_muller(x.z, x.w, z[2], z[3]);
                for (int t = 0; t < 4; ++t) {
                    const int col = 4 * b + t;
                    if (col < F)
                        for (int i = col; i < F; ++i) W[i] = fmaf(c_sim.L[i * (i + 1) / 2 + col], z[t], W[i]);
                }
            }
            const float r0 = r[0];
            // left-point integrals: int r^0 in FP64, Lambda^c compensated FP32, non-decreasing
            I0 = fma((double)r0, ds_d, I0);
            for (int c = 0; c < C; ++c) {
                const float gp = fmaxf(gam[c], 0.f);
                const float y = fmaf(gp, ds, -lamc[c]);
                const float t = lam[c] + y;
                lamc[c] = (t - lam[c]) - y;
                lam[c] = fmaxf(t, lam[c]);
                const int w = c_sim.gpos[c];
                if (w >= 0)
                    gam[c] += c_sim.cir_ktds[c] - c_sim.cir_kds[c] * gp + c_sim.cir_nu_sqds[c] * sqrtf(gp) * W[w];
            }
            const float *drow = a.drift + (size_t)q * E;
            for (int e = 1; e < E; ++e)
                lchi[e] += fmaf(r0 - r[e], ds, c_sim.fx_drift_ds[e]) + c_sim.fx_sig_sqds[e] * W[E - 1 + e];
            for (int e = 0; e < E; ++e)
                r[e] += (__ldg(drow + e) - c_sim.hw_a_ds[e] * r[e]) + c_sim.hw_sig_sqds[e] * W[e];
        }
        store_state(j);
        a.disc[(size_t)j * M + kl] = (float)I0;
        for (int c = 0; c < C; ++c) a.thr[((size_t)j * C + c) * M + kl] = -expm1f(-lam[c]);
    }
}

// One thread per (path, date, portfolio): blockIdx.z is the portfolio.
__global__ void __launch_bounds__(256) price_generic_kernel(OuterArgs a)
{
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, pf = blockIdx.z;
    if (kl >= a.M) return;
    const size_t M = a.M;
    const int E = c_sim.E, C = c_sim.C, F = c_sim.F, G = c_sim.G, n = c_sim.n, ppp = c_sim.ppp;
    if (j == 0) {   // no default at t_0: exposures of date 0 are never used
        for (int c = 0; c < C; ++c) {
            a.expo[((size_t)(pf * (n + 1)) * C + c) * M + kl] = 0.f;
            if (a.mtm) a.mtm[((size_t)(pf * (n + 1)) * C + c) * M + kl] = 0.f;
        }
        return;
    }
    const int p = __ldg(a.date_p + j);          // t_j in (p delta, (p+1) delta]
    const float *fe = a.features + (size_t)j * F * M + kl;
    const float *ffix = a.features + (size_t)(p * ppp) * F * M + kl;   // state at the last reset
    const float2 *fx = a.fix + (size_t)p * E;
    const float beta = expf(-__ldg(a.disc + (size_t)j * M + kl));

    float mt[kMaxC];
    for (int c = 0; c < C; ++c) mt[c] = 0.f;
    for (int e = 0; e < E; ++e) {
        const float re = __ldg(fe + (size_t)e * M);
        const float2 f2 = __ldg(fx + e);
        const float fixm1 = expm1f(fmaf(f2.y, __ldg(ffix + (size_t)e * M), -f2.x));
        const float4 *tab = a.zc + ((size_t)j * E + e) * G;
        const float4 tp = __ldg(tab + (p < G ? p : G - 1));   // p >= G: every swap has matured
        const float z_first = expf(fmaf(-tp.y, re, tp.x));
        float Z[kMaxG], D[kMaxG];
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
        for (int c = 0; c < C; ++c) {
            const int base = ((pf * C + c) * E + e) * G;
            float acc = 0.f;
            for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
            for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
            mt[c] = fmaf(chi, acc, mt[c]);
        }
    }
    for (int c = 0; c < C; ++c) {
        const size_t o = ((size_t)(pf * (n + 1) + j) * C + c) * M + kl;
        a.expo[o] = c_sim.lgd[c] * beta * fmaxf(mt[c], 0.f);
        if (a.mtm) a.mtm[o] = mt[c];
    }
}

cva_status outer_generic_launch(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CVA_EINVAL, "device index out of range");
    OuterArgs args;
    args.M = (uint32_t)s.M;
    args.k0 = (uint32_t)k0;
    args.seed_lo = (uint32_t)seed;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.branch_date = s.branch_date;
    args.branch = s.branch;
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
    sim_generic_kernel<<<(args.M + 127u) / 128u, 128, 0, st>>>(args);
    CVA_CUDA_TRY(cudaGetLastError());
    if (s.ev[1]) CVA_CUDA_TRY(cudaEventRecord(s.ev[1], st));
    price_generic_kernel<<<dim3((args.M + 255u) / 256u, (unsigned)s.n + 1u, (unsigned)s.NPF), 256, 0, st>>>(args);
    CVA_CUDA_TRY(cudaGetLastError());
    if (!capturing) CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
    return CVA_OK;
}

}  // namespace

int outer_insts_generic(const OuterInst **out)
{
    // E, C, CS, NPF of -1: any shape within the limits; G: the schedules' longest
    static const OuterInst insts[] = {
        {-1, -1, -1, kMaxG, -1, outer_generic_launch, outer_forget, nullptr},
    };
    *out = insts;
    return (int)(sizeof(insts) / sizeof(insts[0]));
}

}  // namespace cva
