// Adjoint (reverse-mode) sensitivities of the smooth CVA_0 (one thread per outer
// path), included by outer.cuh so that it reads the same constant-memory tables.
//
// The sampled default indicators have zero pathwise derivative, so the kernel
// differentiates the smooth functional the oversimulated average estimates: the
// exact discrete conditional default probabilities e^{-Lambda(t_{j-1})} -
// e^{-Lambda(t_j)} (the intensity form of eq. (eq:CVAint)):
//   J_k = sum_c sum_{j=1..n} V_c(j) (e^{-Lambda_c(j-1)} - e^{-Lambda_c(j)}),
//   V_c(j) = (1 - R_c) beta_j MtM_c(j)^+,  CVA_0 = mean_k J_k.
// Parameters: flat curve levels f_e, rate volatilities sigma^r_e, FX volatilities
// sigma^chi_e (e >= 1), CIR kappa_c, theta_c, nu_c (gamma_0 held fixed; fixed
// rates of the swaps held at their base-curve par values).
//
// Forward sweep: the Euler scheme of the simulation kernel, storing the full
// state every K pricing dates and the short rates at every reset date. Reverse
// sweep, segment by segment from the last: restore the checkpoint, recompute the
// segment's sub-steps (the Philox counters regenerate the normals), then walk
// the dates backwards: the adjoint of the pricing at t_j (App. B swap formula in
// its date-bucketed form, bond prices, FX conversion, exposure and survival
// terms) followed by the adjoint of every Euler sub-step of (t_{j-1}, t_j].
#pragma once

namespace cva {
namespace {

struct AdjArgs {
    uint32_t M, k0, seed_lo, seed_hi;
    int K, nseg;
    int forward_only;                   // 1: the smooth CVA_0 of the forward sweep only
    const float4 *__restrict__ zc;      // [n+1][E][G] (lnA, B, dlnA, dB)
    const float2 *__restrict__ fix;     // [periods+1][E] (lnA, B)
    const int *__restrict__ date_p;     // [n+1]
    const float *__restrict__ drift;    // [n*S][E]
    const float4 *__restrict__ dzc;     // [n+1][E][G] d/df, d/dsigma of (lnA, dlnA)
    const float2 *__restrict__ dfix;    // [periods+1][E] d/df, d/dsigma of lnA at the fixing
    const float2 *__restrict__ ddrift;  // [n*S][E] d drift/df, d drift/dsigma^r (quanto included)
    const float *__restrict__ rho;      // [E] correlation of r^e and log chi^e (entry 0 unused)
    const float *__restrict__ sig;      // [E] sigma^r, [E] sigma^chi, [C] kappa, [C] theta, [C] nu
    float *ckpt;                        // [nseg][2E+3C][M]
    double *ckpt_I0;                    // [nseg][M]
    float *fixr;                        // [periods+1][E][M]
    double *part;                       // [blocks][npar + 1]
};

template <int E, int C, int CS, int G, int KMAX, int SMAX>
__global__ void __launch_bounds__(128) adjoint_kernel(AdjArgs a)
{
    constexpr int F = 2 * E - 1 + CS;
    constexpr int NB = (F + 3) / 4;
    constexpr int NV = 2 * E + 3 * C;          // checkpointed floats: r, lchi, gam, lam, lamc
    constexpr int NPAR = 3 * E - 1 + 3 * C;
    constexpr int PF = 0, PSR = E, PSX = 2 * E - 1, PK = 3 * E - 1, PT = PK + C, PN = PT + C;   // PSX + e for e >= 1
    __shared__ float pb_s[NPAR * 128];
    __shared__ double red_s[128];
    const int tid = threadIdx.x;
    const uint32_t kl = blockIdx.x * blockDim.x + tid;
    const bool active = kl < a.M;
    const uint32_t k = a.k0 + kl;
    const size_t M = a.M;
    const int n = c_sim.n, S = c_sim.S, ppp = c_sim.ppp, K = a.K;
    const float ds = c_sim.ds, sqds = c_sim.sqds;
    const double ds_d = c_sim.ds_d;
    float *pb = pb_s + tid;                    // this thread's parameter adjoints, stride 128
    for (int i = 0; i < NPAR; ++i) pb[i * 128] = 0.f;
    double J = 0.0;

    if (active) {
        // ---------------- forward sweep: checkpoints and fixings ----------------
        float r[E], lchi[E], gam[C], lam[C], lamc[C];
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
        float lam_prev[C];
        for (int c = 0; c < C; ++c) lam_prev[c] = 0.f;
        for (int j = 0; j <= n; ++j) {
            if (j > 0) {
                for (int s = 0; s < S; ++s) {
                    const uint32_t q = (uint32_t)((j - 1) * S + s);
                    float W[F];
#pragma unroll
                    for (int i = 0; i < F; ++i) W[i] = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const uint4 x = philox4x32_10(make_uint4(k, q, 0u, (kStreamOuter << 24) | (uint32_t)b),
                                                      a.seed_lo, a.seed_hi);
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
            }
            if (j % ppp == 0)
                for (int e = 0; e < E; ++e) a.fixr[((size_t)(j / ppp) * E + e) * M + kl] = r[e];
            if (a.forward_only && j > 0) {
                // smooth CVA_0 term of date j: V_c(j) (e^{-Lambda_c(j-1)} - e^{-Lambda_c(j)})
                const int p = __ldg(a.date_p + j);
                const float beta = expf(-(float)I0);
                float mt[C];
                for (int c = 0; c < C; ++c) mt[c] = 0.f;
                for (int e = 0; e < E; ++e) {
                    const float re = r[e];
                    const float2 f2 = __ldg(a.fix + (size_t)p * E + e);
                    const float fixm1 = expm1f(fmaf(f2.y, a.fixr[((size_t)p * E + e) * M + kl], -f2.x));
                    const float4 *tab = a.zc + ((size_t)j * E + e) * G;
                    float Z[G], D[G];
                    const float4 tp = __ldg(tab + (p < G ? p : G - 1));
                    const float z_first = expf(fmaf(-tp.y, re, tp.x));
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
                    const float chi = (e == 0) ? 1.f : expf(lchi[e]);
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const int base = (c * E + e) * G;
                        float acc = 0.f;
#pragma unroll
                        for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
#pragma unroll
                        for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                        mt[c] = fmaf(chi, acc, mt[c]);
                    }
                }
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
        float rb[E], lb[E], gb[C], Lb[C], rfb[E], Vnext[C];
        for (int e = 0; e < E; ++e) rb[e] = lb[e] = rfb[e] = 0.f;
        for (int c = 0; c < C; ++c) gb[c] = Lb[c] = Vnext[c] = 0.f;
        float Ib = 0.f;
        // segment storage (local memory): pre-states of every sub-step, states of every date
        float st_g[KMAX * SMAX][C];
        float dt_r[KMAX + 1][E], dt_l[KMAX + 1][E], dt_lam[KMAX + 1][C];
        double dt_I0[KMAX + 1];
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
                    const uint32_t q = (uint32_t)((j - 1) * S + s);
                    float W[F];
#pragma unroll
                    for (int i = 0; i < F; ++i) W[i] = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const uint4 x = philox4x32_10(make_uint4(k, q, 0u, (kStreamOuter << 24) | (uint32_t)b),
                                                      a.seed_lo, a.seed_hi);
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
                for (int e = 0; e < E; ++e) {
                    dt_r[j - d0][e] = r[e];
                    dt_l[j - d0][e] = lchi[e];
                }
                for (int c = 0; c < C; ++c) dt_lam[j - d0][c] = lam[c];
                dt_I0[j - d0] = I0;
            }

            for (int j = d1; j > d0; --j) {
                const int jj = j - d0;
                // ---- pricing at t_j: forward ----
                const int p = __ldg(a.date_p + j);
                const float beta = expf(-(float)dt_I0[jj]);
                float mt[C];
                for (int c = 0; c < C; ++c) mt[c] = 0.f;
                for (int e = 0; e < E; ++e) {
                    const float re = dt_r[jj][e];
                    const float2 f2 = __ldg(a.fix + (size_t)p * E + e);
                    const float rfix = a.fixr[((size_t)p * E + e) * M + kl];
                    const float fixm1 = expm1f(fmaf(f2.y, rfix, -f2.x));
                    const float4 *tab = a.zc + ((size_t)j * E + e) * G;
                    float Z[G], D[G];
                    const float4 tp = __ldg(tab + (p < G ? p : G - 1));
                    const float z_first = expf(fmaf(-tp.y, re, tp.x));
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
                    const float chi = (e == 0) ? 1.f : expf(dt_l[jj][e]);
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const int base = (c * E + e) * G;
                        float acc = 0.f;
#pragma unroll
                        for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
#pragma unroll
                        for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                        mt[c] = fmaf(chi, acc, mt[c]);
                    }
                }
                // ---- survival terms and exposure adjoints ----
                float mtb[C];
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
                    float Z[G], D[G], EM[G];
                    const int pc = p < G ? p : G - 1;
                    const float4 tp = __ldg(tab + pc);
                    const float z_first = expf(fmaf(-tp.y, re, tp.x));
#pragma unroll
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
                    const float chi = (e == 0) ? 1.f : expf(dt_l[jj][e]);
                    float Db[G], Zb[G];
#pragma unroll
                    for (int g = 0; g < G; ++g) Db[g] = Zb[g] = 0.f;
                    float chib = 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const int base = (c * E + e) * G;
                        float acc = 0.f;
#pragma unroll
                        for (int h = 0; h < G; ++h) acc = fmaf(c_w.wA[base + h], D[h], acc);
#pragma unroll
                        for (int g = 0; g < G; ++g) acc = fmaf(-c_w.wK[base + g], Z[g], acc);
                        chib = fmaf(mtb[c], acc, chib);
                        const float accb = mtb[c] * chi;
#pragma unroll
                        for (int h = 0; h < G; ++h) Db[h] = fmaf(accb, c_w.wA[base + h], Db[h]);
#pragma unroll
                        for (int g = 0; g < G; ++g) Zb[g] = fmaf(-accb, c_w.wK[base + g], Zb[g]);
                    }
                    if (e > 0) lb[e] += chib * chi;
                    float rbe = 0.f, pf = 0.f, ps = 0.f;
#pragma unroll
                    for (int g = G - 1; g >= 0; --g) {
                        if (g > p) {
                            const float zp = Z[g - 1 >= 0 ? g - 1 : 0];
                            const float em = EM[g];
                            Zb[g - 1 >= 0 ? g - 1 : 0] += Zb[g] * (1.f + em) - Db[g] * em;
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
                    float W[F];
#pragma unroll
                    for (int i = 0; i < F; ++i) W[i] = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const uint4 x = philox4x32_10(make_uint4(k, q, 0u, (kStreamOuter << 24) | (uint32_t)b),
                                                      a.seed_lo, a.seed_hi);
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
                    const float2 *dd = a.ddrift + (size_t)q * E;
                    // parameter adjoints of this sub-step
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const float2 d2 = __ldg(dd + e);
                        pb[(PF + e) * 128] += rb[e] * d2.x;
                        pb[(PSR + e) * 128] += rb[e] * fmaf(sqds, W[e], d2.y);
                    }
#pragma unroll
                    for (int e = 1; e < E; ++e) {
                        const float sx = __ldg(a.sig + E + e), sr = __ldg(a.sig + e);
                        pb[(PSX + e) * 128] += lb[e] * fmaf(sqds, W[E - 1 + e], -sx * ds)
                                               - rb[e] * __ldg(a.rho + e) * sr * ds;
                    }
                    float rb0_extra = Ib * ds;
#pragma unroll
                    for (int e = 1; e < E; ++e) rb0_extra = fmaf(lb[e], ds, rb0_extra);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        float v = rb[e] - rb[e] * c_sim.hw_a_ds[e];
                        if (e > 0) v -= lb[e] * ds;
                        else v += rb0_extra;
                        rb[e] = v;
                    }
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const float g = st_g[qs][c];
                        const float gp = fmaxf(g, 0.f);
                        float gbn = gb[c];
                        if (c < CS) {
                            constexpr int w0 = (CS > 0) ? 2 * E - 1 : 0;
                            const float Wc = W[w0 + (c < CS ? c : 0)];
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

}  // namespace
}  // namespace cva
