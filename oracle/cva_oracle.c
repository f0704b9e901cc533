/*
 * FP64 CPU oracle for the hierarchical ("oversimulated") pathwise CVA scheme
 * of Abbas-Turki, Crepey and Saadeddine, "Pathwise CVA Regressions With
 * Oversimulated Defaults" (arXiv 2211.17005).
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so, which only
 * the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark load. The product path never calls it, and it shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * It is deliberately plain and slow: one outer path at a time, every swap
 * priced on its own by the three-case formula of App. B, every inner default
 * clock compared with the integrated intensity as in eq. (e:tau), and the
 * pathwise target assembled term by term as in eq. (eq:CVA_portfolio).
 * Floating point is binary64 throughout; the only shared inputs with the GPU
 * path are the random-number counters (Philox4x32-10, Salmon et al., SC'11),
 * re-implemented here from the published definition.
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository):
 *  - short rates follow Hull-White fitted to a flat curve f_e (the paper writes
 *    Vasicek, App. B eq. (e:sde1); Vasicek is the constant-theta special case);
 *  - the quanto drift of r^e under Q^0 is -rho_e sigma^chi_e sigma^r_e (App. B,
 *    Girsanov step; the printed drift drops the sigma^r factor);
 *  - the pathwise CVA is multiplied by the loss-given-default (1 - R_c), and
 *    defaults are counted in (t_i, t_n] (eq. (eq:CVA_portfolio) with j = i..n-1);
 *  - integrals of r^0 and gamma^c use the left point of each Euler sub-step
 *    (Remark rem:finecoarse);
 *  - CIR intensities use full truncation (gamma^+ in drift, diffusion, integral);
 *  - a default clock is E = -log(1 - w) with w the uniform below, and
 *    tau in (t_{j-1}, t_j] iff Lambda(t_{j-1}) < E <= Lambda(t_j) (eq. (e:tau)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ---------------- Philox4x32-10 (Salmon et al., SC'11) ------------------ */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Counter layout: (path k, fine step q or inner index l, copy, stream<<24 | block);
 * copy = 0 for the simulation itself, b >= 1 for twin copy b of the twin Monte
 * Carlo validation (Sec. ss:twin) after its branch date. */
#define STREAM_OUTER 1u
#define STREAM_INNER 2u

/* Uniform on (0,1) from the top 23 bits: (m + 1/2) 2^-23. */
double oracle_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

static void draw(uint64_t seed, uint32_t k, uint32_t c1, uint32_t c2, uint32_t stream, uint32_t blk,
                 uint32_t out[4])
{
    const uint32_t ctr[4] = {k, c1, c2, (stream << 24) | blk};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* F standard normals for path k at fine step q (copy word c2): Box-Muller on
 * consecutive pairs. */
static void normals_c(uint64_t seed, uint32_t k, uint32_t q, uint32_t c2, int F, double *z)
{
    for (int b = 0; 4 * b < F; ++b) {
        uint32_t x[4];
        draw(seed, k, q, c2, STREAM_OUTER, (uint32_t)b, x);
        for (int p = 0; p < 2; ++p) {
            const double u1 = oracle_uniform(x[2 * p]);
            const double u2 = oracle_uniform(x[2 * p + 1]);
            const double rad = sqrt(-2.0 * log(u1));
            const int i0 = 4 * b + 2 * p;
            if (i0 < F) z[i0] = rad * cos(2.0 * OR_PI * u2);
            if (i0 + 1 < F) z[i0 + 1] = rad * sin(2.0 * OR_PI * u2);
        }
    }
}

void oracle_normals(uint64_t seed, uint32_t k, uint32_t q, int F, double *z) { normals_c(seed, k, q, 0u, F, z); }

/* Standard exponential clock epsilon^{c} of inner draw l of path k (eq. (e:tau)),
 * copy word c2. */
double oracle_exp_clock_copy(uint64_t seed, uint32_t k, uint32_t l, uint32_t c2, int c)
{
    uint32_t x[4];
    draw(seed, k, l, c2, STREAM_INNER, (uint32_t)(c / 4), x);
    const double w = oracle_uniform(x[c % 4]);
    return -log1p(-w);
}

double oracle_exp_clock(uint64_t seed, uint32_t k, uint32_t l, int c) { return oracle_exp_clock_copy(seed, k, l, 0u, c); }

/* All default clocks of paths [k0, k1) with copy word c2: out[(k-k0)][l][c], for
 * tie accounting. */
void oracle_exp_clocks_copy(uint64_t seed, uint64_t k0, uint64_t k1, uint32_t N, int C, uint32_t c2, double *out)
{
    for (uint64_t k = k0; k < k1; ++k)
        for (uint32_t l = 0; l < N; ++l)
            for (int c = 0; c < C; ++c)
                out[((k - k0) * N + l) * (uint64_t)C + c] = oracle_exp_clock_copy(seed, (uint32_t)k, l, c2, c);
}

void oracle_exp_clocks(uint64_t seed, uint64_t k0, uint64_t k1, uint32_t N, int C, double *out)
{
    oracle_exp_clocks_copy(seed, k0, k1, N, C, 0u, out);
}

/* ---------------- model, portfolio, grid --------------------------------- */

typedef struct {
    int E, C;
    const double *a, *sigma_r, *f;          /* [E] Hull-White, flat curve level */
    const double *sigma_chi, *chi0;         /* [E], entry 0 unused */
    const double *kappa, *theta, *nu, *gamma0, *recovery; /* [C] */
    const double *corr;                     /* [F*F] row-major */
} om_model;

typedef struct {
    int n_swaps;
    const int *ccy, *cpty, *omega, *n_periods;
    const double *notional;
    double delta;
    const double *fixed_rate;   /* [n_swaps] or NULL: par at t = 0 */
} om_portfolio;

typedef struct {
    double horizon;
    int n_steps, substeps;
} om_grid;

typedef struct {
    double *features;   /* [n+1][F][Mloc]  r^e, log chi^e, stochastic gamma^c      */
    double *I0;         /* [n+1][Mloc]     int_0^{t_j} r^0 (so beta_j = exp(-I0)) */
    double *Lambda;     /* [n+1][C][Mloc]  int_0^{t_j} gamma^c                    */
    double *mtm;        /* [n+1][C][Mloc]  MtM^c_j in reference currency           */
    double *swap_pv;    /* [n+1][S][Mloc]  P^sw of each swap in its own currency   */
    uint16_t *idx;      /* [Mloc][N][C]    default step, n+1 = no default by t_n  */
    double *xi_bar;     /* [n][Mloc]       averaged pathwise CVA target, i=0..n-1 */
    double *smooth;     /* [n][Mloc]       intensity form: conditional default probs */
} om_out;

static int n_factors(const om_model *m)
{
    int F = m->E + (m->E - 1);
    for (int c = 0; c < m->C; ++c)
        if (m->nu[c] > 0.0) ++F;
    return F;
}

int oracle_n_factors(const om_model *m) { return n_factors(m); }

/* Lower Cholesky factor L of the correlation matrix, L L^T = corr. */
static int cholesky(int F, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)F * F);
    for (int i = 0; i < F; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * F + j];
            for (int p = 0; p < j; ++p) s -= L[i * F + p] * L[j * F + p];
            if (i == j) {
                if (s <= 0.0) return -1;
                L[i * F + i] = sqrt(s);
            } else {
                L[i * F + j] = s / L[j * F + j];
            }
        }
    }
    return 0;
}

/* Hull-White zero-coupon bond ZC_t(T) of economy e given r_t, for a flat initial
 * curve f: P(0,T)/P(0,t) exp(B f - sigma^2/(4a) (1 - e^{-2at}) B^2 - B r_t),
 * B = (1 - e^{-a(T-t)})/a (App. B footnote: closed form in the affine model). */
double oracle_zc(const om_model *m, int e, double t, double T, double r)
{
    const double a = m->a[e], s = m->sigma_r[e], f = m->f[e];
    const double B = (1.0 - exp(-a * (T - t))) / a;
    const double lnA = -f * (T - t) + B * f - s * s / (4.0 * a) * (1.0 - exp(-2.0 * a * t)) * B * B;
    return exp(lnA - B * r);
}

/* theta_e(t) of Hull-White fitted to a flat curve: a f + sigma^2/(2a) (1 - e^{-2at}). */
static double hw_theta(const om_model *m, int e, double t)
{
    const double a = m->a[e], s = m->sigma_r[e];
    return a * m->f[e] + s * s / (2.0 * a) * (1.0 - exp(-2.0 * a * t));
}

/* Par swap rate Sigma from P^sw_0 = 0 (third case of the App. B formula). */
double oracle_par_rate(const om_model *m, int e, int n_periods, double delta)
{
    double annuity = 0.0;
    for (int g = 1; g <= n_periods; ++g) annuity += oracle_zc(m, e, 0.0, g * delta, m->f[e]);
    return (1.0 - oracle_zc(m, e, 0.0, n_periods * delta, m->f[e])) / (delta * annuity);
}

/* Price of a spot-starting payer swap (pay delta*Sigma, receive floating) at
 * t = t_j, App. B. Reset dates are 0, delta, ..., n_periods*delta = tbar.
 * r_t is today's short rate, r_fix the short rate at the last reset date
 * t_- (Remark rem:pathdep). on_reset says whether t is a reset date, q is the
 * number of periods elapsed (t_- = q delta when t is not a reset date, t = q
 * delta when it is). Returns 0 after maturity. */
static double swap_price(const om_model *m, int e, int n_periods, double delta,
                         double Sigma, double t, int on_reset, int q,
                         double r_t, double r_fix)
{
    const double tbar = n_periods * delta;
    if (on_reset && q == 0) {
        double ann = 0.0;
        for (int g = 1; g <= n_periods; ++g) ann += oracle_zc(m, e, 0.0, g * delta, r_t);
        return 1.0 - oracle_zc(m, e, 0.0, tbar, r_t) - delta * Sigma * ann;
    }
    if (on_reset) {
        if (q > n_periods) return 0.0;
        const double t_minus = (q - 1) * delta;
        double ann = 1.0;   /* ZC_t(t) = 1 for the coupon paid today */
        for (int g = q + 1; g <= n_periods; ++g) ann += oracle_zc(m, e, t, g * delta, r_t);
        return 1.0 / oracle_zc(m, e, t_minus, t, r_fix) - oracle_zc(m, e, t, tbar, r_t)
               - delta * Sigma * ann;
    }
    if (q + 1 > n_periods) return 0.0;
    const double t_minus = q * delta, t_plus = (q + 1) * delta;
    double ann = 0.0;
    for (int g = q + 1; g <= n_periods; ++g) ann += oracle_zc(m, e, t, g * delta, r_t);
    return oracle_zc(m, e, t, t_plus, r_t) / oracle_zc(m, e, t_minus, t_plus, r_fix)
           - oracle_zc(m, e, t, tbar, r_t) - delta * Sigma * ann;
}

/* Steps of length Delta per reset period delta; 0 if delta is not a whole
 * number of pricing steps (the swap schedules must lie on the pricing grid). */
static int steps_per_period(double Delta, double delta)
{
    const double p = delta / Delta;
    const long pr = lround(p);
    if (pr < 1 || fabs(p - (double)pr) > 1e-9 * p) return 0;
    return (int)pr;
}

/*
 * Simulate outer paths k in [k0, k1) and, for each, N inner default draws per
 * counterparty; fill whichever outputs are non-NULL. Returns 0 on success.
 * With copy >= 1 the run is twin copy `copy` branching at date branch_date: the
 * Euler increments of steps j > branch_date and all inner clocks draw with copy
 * as the third counter word (copy 0: the simulation itself).
 */
int oracle_simulate_copy(const om_model *m, const om_portfolio *pf, const om_grid *g,
                         uint64_t k0, uint64_t k1, uint32_t N, uint64_t seed,
                         int branch_date, uint32_t copy, int n_threads, const om_out *out)
{
    const int E = m->E, C = m->C, F = n_factors(m), n = g->n_steps, S = g->substeps;
    const int NS = pf->n_swaps;
    const size_t Mloc = (size_t)(k1 - k0);
    const double Delta = g->horizon / n, ds = Delta / S, sqds = sqrt(ds);
    const int ppp = steps_per_period(Delta, pf->delta);
    if (n < 1 || S < 1 || k1 <= k0 || ppp == 0 || C > 64) return -1;

    double *L = (double *)malloc(sizeof(double) * (size_t)F * F);
    if (cholesky(F, m->corr, L) != 0) { free(L); return -2; }

    /* factor positions in the correlated normal vector */
    int *pos_r = (int *)malloc(sizeof(int) * E), *pos_x = (int *)malloc(sizeof(int) * E);
    int *pos_g = (int *)malloc(sizeof(int) * C);
    {
        int p = 0;
        for (int e = 0; e < E; ++e) pos_r[e] = p++;
        pos_x[0] = -1;
        for (int e = 1; e < E; ++e) pos_x[e] = p++;
        for (int c = 0; c < C; ++c) pos_g[c] = (m->nu[c] > 0.0) ? p++ : -1;
    }
    double *Sigma = (double *)malloc(sizeof(double) * (NS > 0 ? NS : 1));
    for (int s = 0; s < NS; ++s)
        Sigma[s] = pf->fixed_rate ? pf->fixed_rate[s] : oracle_par_rate(m, pf->ccy[s], pf->n_periods[s], pf->delta);

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double *r = malloc(sizeof(double) * E), *lchi = malloc(sizeof(double) * E);
        double *gam = malloc(sizeof(double) * C), *Lam = malloc(sizeof(double) * (size_t)C * (n + 1));
        double *rfix = malloc(sizeof(double) * E), *z = malloc(sizeof(double) * F);
        double *W = malloc(sizeof(double) * F), *dr = malloc(sizeof(double) * E);
        double *dl = malloc(sizeof(double) * E), *dg = malloc(sizeof(double) * C);
        double *I0 = malloc(sizeof(double) * (n + 1));
        double *V = malloc(sizeof(double) * (size_t)C * (n + 1));   /* (1-R) beta MtM^+ */

#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (long long kk = 0; kk < (long long)Mloc; ++kk) {
            const uint32_t k = (uint32_t)(k0 + (uint64_t)kk);
            for (int e = 0; e < E; ++e) { r[e] = m->f[e]; lchi[e] = log(m->chi0[e]); rfix[e] = r[e]; }
            for (int c = 0; c < C; ++c) { gam[c] = m->gamma0[c]; Lam[c * (n + 1)] = 0.0; }
            I0[0] = 0.0;
            double Iacc = 0.0;

            for (int j = 0; j <= n; ++j) {
                if (j > 0) {
                    /* Euler-Maruyama sub-steps from t_{j-1} to t_j (Remark rem:finecoarse) */
                    for (int s = 0; s < S; ++s) {
                        const int q = (j - 1) * S + s;
                        const double t = q * ds;
                        normals_c(seed, k, (uint32_t)q, j > branch_date ? copy : 0u, F, z);
                        for (int a = 0; a < F; ++a) {
                            double acc = 0.0;
                            for (int b = 0; b <= a; ++b) acc += L[a * F + b] * z[b];
                            W[a] = acc;
                        }
                        for (int e = 0; e < E; ++e) {
                            double drift = hw_theta(m, e, t) - m->a[e] * r[e];
                            if (e > 0) /* quanto adjustment: Q^e -> Q^0 (App. B) */
                                drift -= m->corr[pos_r[e] * F + pos_x[e]] * m->sigma_chi[e] * m->sigma_r[e];
                            dr[e] = drift * ds + m->sigma_r[e] * sqds * W[pos_r[e]];
                        }
                        for (int e = 1; e < E; ++e) {
                            const double sx = m->sigma_chi[e];
                            dl[e] = (r[0] - r[e] - 0.5 * sx * sx) * ds + sx * sqds * W[pos_x[e]];
                        }
                        for (int c = 0; c < C; ++c) {
                            if (pos_g[c] < 0) { dg[c] = 0.0; continue; }
                            const double gp = gam[c] > 0.0 ? gam[c] : 0.0;
                            dg[c] = m->kappa[c] * (m->theta[c] - gp) * ds + m->nu[c] * sqrt(gp) * sqds * W[pos_g[c]];
                        }
                        /* left-point integrals of r^0 and gamma^+ */
                        Iacc += r[0] * ds;
                        for (int c = 0; c < C; ++c) {
                            const double gp = gam[c] > 0.0 ? gam[c] : 0.0;
                            Lam[c * (n + 1) + j] = (s == 0 ? Lam[c * (n + 1) + j - 1] : Lam[c * (n + 1) + j]) + gp * ds;
                        }
                        for (int e = 0; e < E; ++e) r[e] += dr[e];
                        for (int e = 1; e < E; ++e) lchi[e] += dl[e];
                        for (int c = 0; c < C; ++c) gam[c] += dg[c];
                    }
                    I0[j] = Iacc;
                }

                /* pricing date t_j */
                const double t = j * Delta;
                const int on_reset = (j % ppp) == 0;
                const int q = j / ppp;
                double mtm_c[64];
                for (int c = 0; c < C; ++c) mtm_c[c] = 0.0;
                for (int sw = 0; sw < NS; ++sw) {
                    const int e = pf->ccy[sw];
                    const double pv = swap_price(m, e, pf->n_periods[sw], pf->delta, Sigma[sw], t,
                                                 on_reset, q, r[e], rfix[e]);
                    if (out->swap_pv) out->swap_pv[((size_t)j * NS + sw) * Mloc + kk] = pv;
                    const double chi = (e == 0) ? 1.0 : exp(lchi[e]);
                    mtm_c[pf->cpty[sw]] += pf->omega[sw] * pf->notional[sw] * chi * pv;
                }
                if (on_reset)
                    for (int e = 0; e < E; ++e) rfix[e] = r[e];
                for (int c = 0; c < C; ++c) {
                    const double mp = mtm_c[c] > 0.0 ? mtm_c[c] : 0.0;
                    V[c * (n + 1) + j] = (1.0 - m->recovery[c]) * exp(-I0[j]) * mp;
                    if (out->mtm) out->mtm[((size_t)j * C + c) * Mloc + kk] = mtm_c[c];
                    if (out->Lambda) out->Lambda[((size_t)j * C + c) * Mloc + kk] = Lam[c * (n + 1) + j];
                }
                if (out->I0) out->I0[(size_t)j * Mloc + kk] = I0[j];
                if (out->features) {
                    double *fe = out->features + (size_t)j * F * Mloc + kk;
                    int p = 0;
                    for (int e = 0; e < E; ++e) fe[(size_t)(p++) * Mloc] = r[e];
                    for (int e = 1; e < E; ++e) fe[(size_t)(p++) * Mloc] = lchi[e];
                    for (int c = 0; c < C; ++c)
                        if (pos_g[c] >= 0) fe[(size_t)(p++) * Mloc] = gam[c];
                }
            }

            /* Inner defaults and the averaged target, eq. (eq:CVA_portfolio):
             * xi_i = sum_c sum_{j=i}^{n-1} beta_i^{-1} beta_{j+1} (1-R_c) (MtM^c_{j+1})^+ 1{t_j < tau^c <= t_{j+1}},
             * where the indicator picks the single j with tau in (t_j, t_{j+1}]. */
            if (out->xi_bar)
                for (int i = 0; i < n; ++i) out->xi_bar[(size_t)i * Mloc + kk] = 0.0;
            for (uint32_t l = 0; l < N; ++l) {
                for (int c = 0; c < C; ++c) {
                    const double eps = oracle_exp_clock_copy(seed, k, l, copy, c);
                    int idx = n + 1;
                    for (int j = 1; j <= n; ++j)
                        if (Lam[c * (n + 1) + j] >= eps) { idx = j; break; }
                    if (out->idx) out->idx[((size_t)kk * N + l) * C + c] = (uint16_t)idx;
                    if (out->xi_bar && idx <= n)
                        for (int i = 0; i < idx; ++i)
                            out->xi_bar[(size_t)i * Mloc + kk] += exp(I0[i]) * V[c * (n + 1) + idx] / N;
                }
            }
            /* Smooth form: E over the default clocks given Y of the same sum,
             * sum_c sum_{j>i} beta_i^{-1} V_c(j) (e^{-(Lam_{j-1}-Lam_i)} - e^{-(Lam_j-Lam_i)}) times
             * the survival to t_i, i.e. the Y-conditional mean of xi_i. */
            if (out->smooth)
                for (int i = 0; i < n; ++i) {
                    double acc = 0.0;
                    for (int c = 0; c < C; ++c)
                        for (int j = i + 1; j <= n; ++j)
                            acc += V[c * (n + 1) + j] * (exp(-Lam[c * (n + 1) + j - 1]) - exp(-Lam[c * (n + 1) + j]));
                    out->smooth[(size_t)i * Mloc + kk] = exp(I0[i]) * acc;
                }
        }
        free(r); free(lchi); free(gam); free(Lam); free(rfix); free(z); free(W);
        free(dr); free(dl); free(dg); free(I0); free(V);
    }
    free(L); free(pos_r); free(pos_x); free(pos_g); free(Sigma);
    return 0;
}

int oracle_simulate(const om_model *m, const om_portfolio *pf, const om_grid *g,
                    uint64_t k0, uint64_t k1, uint32_t N, uint64_t seed,
                    int n_threads, const om_out *out)
{
    return oracle_simulate_copy(m, pf, g, k0, k1, N, seed, 1 << 30, 0u, n_threads, out);
}
