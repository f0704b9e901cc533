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

// ---- adjoint of the smooth CVA_0 for run-time shapes ----
// adjoint_kernel (adjoint.cuh) with the model's sizes as run-time values: the same
// forward sweep with checkpoints every K dates, the same segment recompute and
// reverse of the pricing and of the Euler sub-steps, in the same order, so a shape
// with a compiled adjoint gives its bits. The stochastic intensity of counterparty c
// is state factor c_sim.gpos[c] (-1: constant, whose kappa, theta, nu receive
// nothing). Per-thread arrays are sized at the library's limits (local memory); the
// parameter adjoints live in dynamic shared memory, NPAR x 128 floats.
constexpr int kAdjKMax = 16, kAdjSMax = 4;

// bond prices Z and their differences D (and the expm1 factors EM) of economy e at
// date j for one path: the chained form of price_kernel
__device__ __forceinline__ void bonds_generic(const AdjArgs &a, int j, int e, int p, float re, float fixm1,
                                              float (&Z)[kMaxG], float (&D)[kMaxG], float (&EM)[kMaxG])
{
    const int E = c_sim.E, G = c_sim.G;
    const float4 *tab = a.zc + ((size_t)j * E + e) * G;
    const float4 tp = __ldg(tab + (p < G ? p : G - 1));
    const float z_first = expf(fmaf(-tp.y, re, tp.x));
    for (int g = 0; g < G; ++g) {
        EM[g] = 0.f;
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
            EM[g] = em;
            D[g] = -zp * em;
            Z[g] = fmaf(zp, em, zp);
        }
    }
}

// correlated increments W = L z of fine step q for path k
__device__ __forceinline__ void increments_generic(const AdjArgs &a, uint32_t k, uint32_t q, float (&W)[kMaxF])
{
    const int F = c_sim.F, NB = (F + 3) / 4;
    for (int i = 0; i < F; ++i) W[i] = 0.f;
    for (int b = 0; b < NB; ++b) {
        const uint4 x = philox4x32_10(make_uint4(k, q, 0u, (kStreamOuter << 24) | (uint32_t)b), a.seed_lo, a.seed_hi);
        float z[4];
        box_muller(x.x, x.y, z[0], z[1]);
        box_muller(x.z, x.w, z[2], z[3]);
        for (int t = 0; t < 4; ++t) {
            const int col = 4 * b + t;
            if (col < F)
                for (int i = col; i < F; ++i) W[i] = fmaf(c_sim.L[i * (i + 1) / 2 + col], z[t], W[i]);
        }
    }
}

__global__ void __launch_bounds__(128) adjoint_generic_kernel(AdjArgs a)
{
    const int E = c_sim.E, C = c_sim.C, G = c_sim.G;
    const int NV = 2 * E + 3 * C, NPAR = 3 * E - 1 + 3 * C;
    const int PF = 0, PSR = E, PSX = 2 * E - 1, PK = 3 * E - 1, PT = PK + C, PN = PT + C;
    extern __shared__ float pb_s[];                    // [NPAR][128]
    __shared__ double red_s[128];
    const int tid = threadIdx.x;
    const uint32_t kl = blockIdx.x * blockDim.x + tid;
    const bool active = kl < a.M;
    const uint32_t k = a.k0 + kl;
    const size_t M = a.M;
    const int n = c_sim.n, S = c_sim.S, ppp = c_sim.ppp, K = a.K;
    const float ds = c_sim.ds, sqds = c_sim.sqds;
    const double ds_d = c_sim.ds_d;
    float *pb = pb_s + tid;
    for (int i = 0; i < NPAR; ++i) pb[i * 128] = 0.f;
    double J = 0.0;

    if (active) {
        float r[kMaxE], lchi[kMaxE], gam[kMaxC], lam[kMaxC], lamc[kMaxC], lam_prev[kMaxC];
        float W[kMaxF], Z[kMaxG], D[kMaxG], EM[kMaxG], mt[kMaxC];
        for (int e = 0; e < E; ++e) {
            r[e] = c_sim.r0[e];
            lchi[e] = c_sim.lchi0[e];
        }
        for (int c = 0; c < C; ++c) {
            gam[c] = c_sim.gamma0[c];
            lam[c] = lamc[c] = lam_prev[c] = 0.f;
        }
        double I0 = 0.0;
        // one Euler sub-step of the state (sim_kernel's order)
        auto step = [&](uint32_t q) {
            increments_generic(a, k, q, W);
            const float r0 = r[0];
            I0 = fma((double)r0, ds_d, I0);
            for (int c = 0; c < C; ++c) {
                const float gp = fmaxf(gam[c], 0.f);
                const float y = fmaf(gp, ds, -lamc[c]);
                const float t = lam[c] + y;
                lamc[c] = (t - lam[c]) - y;
                lam[c] = fmaxf(t, lam[c]);
                const int w = c_sim.gpos[c];
                if (w >= 0) gam[c] += c_sim.cir_ktds[c] - c_sim.cir_kds[c] * gp + c_sim.cir_nu_sqds[c] * sqrtf(gp) * W[w];
            }
            const float *drow = a.drift + (size_t)q * E;
            for (int e = 1; e < E; ++e)
                lchi[e] += fmaf(r0 - r[e], ds, c_sim.fx_drift_ds[e]) + c_sim.fx_sig_sqds[e] * W[E - 1 + e];
            for (int e = 0; e < E; ++e) r[e] += (__ldg(drow + e) - c_sim.hw_a_ds[e] * r[e]) + c_sim.hw_sig_sqds[e] * W[e];
        };
        // the MtM of every counterparty at date j from the rates and FX levels given
        auto mtm = [&](int j, int p, const float *rr, const float *ll) {
            for (int c = 0; c < C; ++c) mt[c] = 0.f;
            for (int e = 0; e < E; ++e) {
                const float2 f2 = __ldg(a.fix + (size_t)p * E + e);
                const float fixm1 = expm1f(fmaf(f2.y, a.fixr[((size_t)p * E + e) * M + kl], -f2.x));
                bonds_generic(a, j, e, p, rr[e], fixm1, Z, D, EM);
                const float chi = (e == 0) ? 1.f : expf(ll[e]);
                for (int c = 0; c < C; ++c) {
                    const int base = (c * E + e) * G;
                    float acc = 0.f;
                    for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
                    for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                    mt[c] = fmaf(chi, acc, mt[c]);
                }
            }
        };

        // ---------------- forward sweep: checkpoints and fixings ----------------
        for (int j = 0; j <= n; ++j) {
            if (j > 0)
                for (int s = 0; s < S; ++s) step((uint32_t)((j - 1) * S + s));
            if (j % ppp == 0)
                for (int e = 0; e < E; ++e) a.fixr[((size_t)(j / ppp) * E + e) * M + kl] = r[e];
            if (a.forward_only && j > 0) {
                const int p = __ldg(a.date_p + j);
                const float beta = expf(-(float)I0);
                mtm(j, p, r, lchi);
                for (int c = 0; c < C; ++c) {
                    const float V = c_sim.lgd[c] * beta * fmaxf(mt[c], 0.f);
                    J += (double)V * (double)(expf(-lam_prev[c]) - expf(-lam[c]));
                }
            }
            for (int c = 0; c < C; ++c) lam_prev[c] = lam[c];
            if (j % K == 0 && j / K < a.nseg) {
                float *cp = a.ckpt + (size_t)(j / K) * NV * M + kl;
                int v = 0;
                for (int e = 0; e < E; ++e) cp[(size_t)(v++) * M] = r[e];
                for (int e = 0; e < E; ++e) cp[(size_t)(v++) * M] = lchi[e];
                for (int c = 0; c < C; ++c) cp[(size_t)(v++) * M] = gam[c];
                for (int c = 0; c < C; ++c) cp[(size_t)(v++) * M] = lam[c];
                for (int c = 0; c < C; ++c) cp[(size_t)(v++) * M] = lamc[c];
                a.ckpt_I0[(size_t)(j / K) * M + kl] = I0;
            }
        }

        if (!a.forward_only) {
            // ---------------- reverse sweep ----------------
            float rb[kMaxE], lb[kMaxE], rfb[kMaxE], gb[kMaxC], Lb[kMaxC], Vnext[kMaxC], mtb[kMaxC];
            for (int e = 0; e < E; ++e) rb[e] = lb[e] = rfb[e] = 0.f;
            for (int c = 0; c < C; ++c) gb[c] = Lb[c] = Vnext[c] = 0.f;
            float Ib = 0.f;
            float st_g[kAdjKMax * kAdjSMax][kMaxC];
            float dt_r[kAdjKMax + 1][kMaxE], dt_l[kAdjKMax + 1][kMaxE], dt_lam[kAdjKMax + 1][kMaxC];
            double dt_I0[kAdjKMax + 1];
            for (int seg = a.nseg - 1; seg >= 0; --seg) {
                const int d0 = seg * K, d1 = min(d0 + K, n);
                {
                    const float *cp = a.ckpt + (size_t)seg * NV * M + kl;
                    int v = 0;
                    for (int e = 0; e < E; ++e) r[e] = cp[(size_t)(v++) * M];
                    for (int e = 0; e < E; ++e) lchi[e] = cp[(size_t)(v++) * M];
                    for (int c = 0; c < C; ++c) gam[c] = cp[(size_t)(v++) * M];
                    for (int c = 0; c < C; ++c) lam[c] = cp[(size_t)(v++) * M];
                    for (int c = 0; c < C; ++c) lamc[c] = cp[(size_t)(v++) * M];
                    I0 = a.ckpt_I0[(size_t)seg * M + kl];
                }
                for (int e = 0; e < E; ++e) {
                    dt_r[0][e] = r[e];
                    dt_l[0][e] = lchi[e];
                }
                for (int c = 0; c < C; ++c) dt_lam[0][c] = lam[c];
                dt_I0[0] = I0;
                for (int j = d0 + 1; j <= d1; ++j) {
                    for (int s = 0; s < S; ++s) {
                        const int qs = (j - d0 - 1) * S + s;
                        for (int c = 0; c < C; ++c) st_g[qs][c] = gam[c];
                        step((uint32_t)((j - 1) * S + s));
                    }
                    for (int e = 0; e < E; ++e) {
                        dt_r[j - d0][e] = r[e];
                        dt_l[j - d0][e] = lchi[e];
                    }
                    for (int c = 0; c < C; ++c) dt_lam[j - d0][c] = lam[c];
                    dt_I0[j - d0] = I0;
                }

                for (int j = d1; j > d0; --j) {
                    const int jj = j - d0;
                    const int p = __ldg(a.date_p + j);
                    const float beta = expf(-(float)dt_I0[jj]);
                    mtm(j, p, dt_r[jj], dt_l[jj]);
                    // ---- survival terms and exposure adjoints ----
                    for (int c = 0; c < C; ++c) {
                        const float V = c_sim.lgd[c] * beta * fmaxf(mt[c], 0.f);
                        const float Sp = expf(-dt_lam[jj - 1][c]), Sc = expf(-dt_lam[jj][c]);
                        J += (double)V * (double)(Sp - Sc);
                        const float Vb = Sp - Sc;
                        Lb[c] += Sc * (V - Vnext[c]);
                        Vnext[c] = V;
                        mtb[c] = mt[c] > 0.f ? Vb * c_sim.lgd[c] * beta : 0.f;
                        Ib -= Vb * V;
                    }
                    // ---- pricing at t_j: reverse, economy by economy ----
                    for (int e = 0; e < E; ++e) {
                        const float re = dt_r[jj][e];
                        const float2 f2 = __ldg(a.fix + (size_t)p * E + e);
                        const float rfix = a.fixr[((size_t)p * E + e) * M + kl];
                        const float fixm1 = expm1f(fmaf(f2.y, rfix, -f2.x));
                        const float4 *tab = a.zc + ((size_t)j * E + e) * G;
                        const float4 *dtab = a.dzc + ((size_t)j * E + e) * G;
                        bonds_generic(a, j, e, p, re, fixm1, Z, D, EM);
                        const float4 tp = __ldg(tab + (p < G ? p : G - 1));
                        const float chi = (e == 0) ? 1.f : expf(dt_l[jj][e]);
                        float Db[kMaxG], Zb[kMaxG];
                        for (int g = 0; g < G; ++g) Db[g] = Zb[g] = 0.f;
                        float chib = 0.f;
                        for (int c = 0; c < C; ++c) {
                            const int base = (c * E + e) * G;
                            float acc = 0.f;
                            for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
                            for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                            chib = fmaf(mtb[c], acc, chib);
                            const float accb = mtb[c] * chi;
                            for (int h = 0; h < G; ++h) Db[h] = fmaf(accb, c_w.wA[base + h], Db[h]);
                            for (int g = 0; g < G; ++g) Zb[g] = fmaf(-accb, c_w.wK[base + g], Zb[g]);
                        }
                        if (e > 0) lb[e] += chib * chi;
                        float rbe = 0.f, pf = 0.f, ps = 0.f;
                        for (int g = G - 1; g >= 0; --g) {
                            if (g > p) {
                                const int gm = g - 1 >= 0 ? g - 1 : 0;
                                const float zp = Z[gm];
                                const float em = EM[g];
                                Zb[gm] += Zb[g] * (1.f + em) - Db[g] * em;
                                const float xb = (Zb[g] - Db[g]) * zp * (1.f + em);
                                const float4 t4 = __ldg(tab + g);
                                const float4 d4 = __ldg(dtab + g);
                                rbe -= xb * t4.w;
                                pf += xb * d4.z;
                                ps += xb * d4.w;
                            } else if (g == p) {
                                Zb[g] += Db[g] * fixm1;
                                const float fixb = Db[g] * Z[g];
                                const float yb = Zb[g] * Z[g];
                                const float4 d4 = __ldg(dtab + g);
                                rbe -= yb * tp.y;
                                pf += yb * d4.x;
                                ps += yb * d4.y;
                                const float ub = fixb * (1.f + fixm1);
                                const float2 df2 = __ldg(a.dfix + (size_t)p * E + e);
                                rfb[e] += ub * f2.y;
                                pf -= ub * df2.x;
                                ps -= ub * df2.y;
                            }
                        }
                        rb[e] += rbe;
                        pb[(PF + e) * 128] += pf;
                        pb[(PSR + e) * 128] += ps;
                    }
                    // ---- Euler sub-steps of (t_{j-1}, t_j], in reverse ----
                    for (int s = S - 1; s >= 0; --s) {
                        const int qs = (jj - 1) * S + s;
                        const uint32_t q = (uint32_t)((j - 1) * S + s);
                        increments_generic(a, k, q, W);
                        const float2 *dd = a.ddrift + (size_t)q * E;
                        for (int e = 0; e < E; ++e) {
                            const float2 d2 = __ldg(dd + e);
                            pb[(PF + e) * 128] += rb[e] * d2.x;
                            pb[(PSR + e) * 128] += rb[e] * fmaf(sqds, W[e], d2.y);
                        }
                        for (int e = 1; e < E; ++e) {
                            const float sx = __ldg(a.sig + E + e), sr = __ldg(a.sig + e);
                            pb[(PSX + e) * 128] += lb[e] * fmaf(sqds, W[E - 1 + e], -sx * ds)
                                                   - rb[e] * __ldg(a.rho + e) * sr * ds;
                        }
                        float rb0_extra = Ib * ds;
                        for (int e = 1; e < E; ++e) rb0_extra = fmaf(lb[e], ds, rb0_extra);
                        for (int e = 0; e < E; ++e) {
                            float v = rb[e] - rb[e] * c_sim.hw_a_ds[e];
                            if (e > 0) v -= lb[e] * ds;
                            else v += rb0_extra;
                            rb[e] = v;
                        }
                        for (int c = 0; c < C; ++c) {
                            const float g = st_g[qs][c];
                            const float gp = fmaxf(g, 0.f);
                            float gbn = gb[c];
                            const int w = c_sim.gpos[c];
                            if (w >= 0) {
                                const float Wc = W[w];
                                const float kap = __ldg(a.sig + 2 * E + c), th = __ldg(a.sig + 2 * E + C + c);
                                pb[(PK + c) * 128] += gb[c] * (th - gp) * ds;
                                pb[(PT + c) * 128] += gb[c] * kap * ds;
                                pb[(PN + c) * 128] += gb[c] * sqrtf(gp) * sqds * Wc;
                                if (g > 0.f)
                                    gbn = gb[c] * (1.f - c_sim.cir_kds[c] + c_sim.cir_nu_sqds[c] * Wc * 0.5f * rsqrtf(g));
                            }
                            if (g > 0.f) gbn += Lb[c] * ds;
                            gb[c] = gbn;
                        }
                    }
                    // the state at t_{j-1}: a reset date receives the adjoint of its fixing
                    if ((j - 1) % ppp == 0)
                        for (int e = 0; e < E; ++e) {
                            rb[e] += rfb[e];
                            rfb[e] = 0.f;
                        }
                }
            }
            // r_0 = f
            for (int e = 0; e < E; ++e) pb[(PF + e) * 128] += rb[e];
        }
    }

    // ---- block reduction of the parameter adjoints and of J (FP64, fixed order) ----
    __syncthreads();
    double *out = a.part + (size_t)blockIdx.x * (NPAR + 1);
    for (int i = 0; i <= NPAR; ++i) {
        red_s[tid] = (i < NPAR) ? (double)pb_s[i * 128 + tid] : J;
        __syncthreads();
        for (int s = 64; s > 0; s >>= 1) {
            if (tid < s) red_s[tid] += red_s[tid + s];
            __syncthreads();
        }
        if (tid == 0) out[i] = red_s[0];
        __syncthreads();
    }
}

cva_status adjoint_generic_launch(Sim &s, const AdjBuffers &b, uint64_t seed, uint64_t k0, uint32_t M, cudaStream_t st)
{
    if (b.K < 1 || b.K > kAdjKMax || s.S > kAdjSMax)
        return fail(CVA_ENOTSUP, "adjoint: checkpoint interval <= 16, sub-steps <= 4");
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
    const int npar = 3 * s.E - 1 + 3 * s.C;
    const size_t smem = (size_t)npar * 128 * sizeof(float);
    static bool attr = false;
    if (!attr) {
        CVA_CUDA_TRY(cudaFuncSetAttribute(adjoint_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)((3 * kMaxE - 1 + 3 * kMaxC) * 128 * sizeof(float))));
        attr = true;
    }
    std::lock_guard<std::mutex> lk(t_const_mu);
    if (!t_last[dev]) CVA_CUDA_TRY(cudaEventCreateWithFlags(&t_last[dev], cudaEventDisableTiming));
    else CVA_CUDA_TRY(cudaStreamWaitEvent(st, t_last[dev], 0));
    if (t_owner[dev] != &s) {
        CVA_CUDA_TRY(upload_consts(s, st));
        t_owner[dev] = &s;
    }
    adjoint_generic_kernel<<<(M + 127u) / 128u, 128, smem, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    CVA_CUDA_TRY(cudaEventRecord(t_last[dev], st));
    return CVA_OK;
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
        {-1, -1, -1, kMaxG, -1, outer_generic_launch, outer_forget, adjoint_generic_launch},
    };
    *out = insts;
    return (int)(sizeof(insts) / sizeof(insts[0]));
}

}  // namespace cva
