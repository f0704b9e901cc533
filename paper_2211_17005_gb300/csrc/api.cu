// C ABI of the library (include/cva.h): input validation, host-side tables
// and device buffers of a simulation, and the entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cva_internal.h"

namespace cva {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string &msg) { g_err = msg; }

cva_status fail(cva_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

cva_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CVA_ENOMEM : CVA_ECUDA;
}

namespace {

bool is_fin(double x) { return std::isfinite(x); }

// Hull-White bond ZC_t(T) = exp(lnA(t,T) - B(t,T) r_t) for a flat initial curve f:
// B = (1 - e^{-a(T-t)})/a, lnA = -f (T-t) + B f - sigma^2/(4a) (1 - e^{-2at}) B^2.
struct HW {
    double a, s, f;
    double B(double t, double T) const { return (1.0 - std::exp(-a * (T - t))) / a; }
    double lnA(double t, double T) const
    {
        const double b = B(t, T);
        return -f * (T - t) + b * f - s * s / (4.0 * a) * (1.0 - std::exp(-2.0 * a * t)) * b * b;
    }
    // theta(t) of the fit to the flat curve: a f + sigma^2/(2a) (1 - e^{-2at})
    double theta(double t) const { return a * f + s * s / (2.0 * a) * (1.0 - std::exp(-2.0 * a * t)); }
};

// Lower Cholesky factor of an SPD matrix (FP64); false if not positive definite.
bool cholesky(int F, const double *A, std::vector<double> &L)
{
    L.assign((size_t)F * F, 0.0);
    for (int i = 0; i < F; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * F + j];
            for (int p = 0; p < j; ++p) s -= L[i * F + p] * L[j * F + p];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * F + i] = std::sqrt(s);
            } else {
                L[i * F + j] = s / L[j * F + j];
            }
        }
    return true;
}

template <class T>
cva_status dev_alloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return CVA_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(CVA_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return CVA_OK;
}

void free_sim(Sim *s)
{
    if (!s) return;
    forget_const_owner(s);
    cudaFree(s->d_zc);
    cudaFree(s->d_fix);
    cudaFree(s->d_date_p);
    cudaFree(s->d_drift);
    cudaFree(s->d_features);
    cudaFree(s->d_disc);
    cudaFree(s->d_thr);
    cudaFree(s->d_expo);
    cudaFree(s->d_mtm);
    cudaFree(s->d_targets);
    cudaFree(s->d_idx);
    cudaFree(s->d_cnt);
    cudaFree(s->d_const_img);
    cudaFree(s->d_lsq);
    cudaFree(s->d_alive_stats);
    cudaFree(s->d_alive);
    for (cudaEvent_t &e : s->ev)
        if (e) cudaEventDestroy(e);
    delete s;
}

cva_status validate_model(const cva_model_desc *m, int *F_out, int *CS_out, std::vector<double> &L)
{
    if (!m) return fail(CVA_EINVAL, "model is NULL");
    if (m->E < 1 || m->E > kMaxE) return fail(CVA_EINVAL, "model: E must be in [1, 16]");
    if (m->C < 1 || m->C > kMaxC) return fail(CVA_EINVAL, "model: C must be in [1, 16]");
    if (!m->hw_a || !m->hw_sigma || !m->curve || !m->fx_vol || !m->fx0 || !m->cir_kappa ||
        !m->cir_theta || !m->cir_nu || !m->gamma0 || !m->recovery || !m->corr)
        return fail(CVA_EINVAL, "model: NULL parameter array");
    for (int e = 0; e < m->E; ++e) {
        if (!(m->hw_a[e] > 0.0) || !is_fin(m->hw_a[e])) return fail(CVA_EINVAL, "model: hw_a must be > 0");
        if (!(m->hw_sigma[e] >= 0.0) || !is_fin(m->hw_sigma[e])) return fail(CVA_EINVAL, "model: hw_sigma must be >= 0");
        if (!is_fin(m->curve[e])) return fail(CVA_EINVAL, "model: curve must be finite");
        if (e > 0 && (!(m->fx_vol[e] >= 0.0) || !is_fin(m->fx_vol[e])))
            return fail(CVA_EINVAL, "model: fx_vol must be >= 0");
        if (e > 0 && (!(m->fx0[e] > 0.0) || !is_fin(m->fx0[e]))) return fail(CVA_EINVAL, "model: fx0 must be > 0");
    }
    int CS = 0;
    for (int c = 0; c < m->C; ++c) {
        if (!(m->cir_kappa[c] >= 0.0) || !(m->cir_theta[c] >= 0.0) || !(m->cir_nu[c] >= 0.0) ||
            !(m->gamma0[c] >= 0.0) || !is_fin(m->cir_kappa[c]) || !is_fin(m->cir_theta[c]) ||
            !is_fin(m->cir_nu[c]) || !is_fin(m->gamma0[c]))
            return fail(CVA_EINVAL, "model: CIR parameters must be finite and >= 0");
        if (!(m->recovery[c] >= 0.0 && m->recovery[c] <= 1.0)) return fail(CVA_EINVAL, "model: recovery must be in [0, 1]");
        if (m->cir_nu[c] > 0.0) ++CS;
    }
    const int F = m->E + (m->E - 1) + CS;
    for (int i = 0; i < F; ++i) {
        if (std::fabs(m->corr[i * F + i] - 1.0) > 1e-12) return fail(CVA_EINVAL, "model: corr diagonal must be 1");
        for (int j = 0; j < F; ++j) {
            const double v = m->corr[i * F + j];
            if (!is_fin(v) || std::fabs(v - m->corr[j * F + i]) > 1e-12 || std::fabs(v) > 1.0)
                return fail(CVA_EINVAL, "model: corr must be a symmetric correlation matrix");
        }
    }
    if (!cholesky(F, m->corr, L)) return fail(CVA_EINVAL, "model: corr is not positive definite");
    *F_out = F;
    *CS_out = CS;
    return CVA_OK;
}

}  // namespace
}  // namespace cva

using namespace cva;

extern "C" {

const char *cva_last_error(void) { return g_err.c_str(); }

const char *cva_version(void) { return "sm_103a 0.1.0"; }

cva_status cva_sim_create(const cva_model_desc *model, const cva_portfolio_desc *pfs, int n_pf,
                          const cva_grid *grid, uint64_t M, uint32_t N, uint32_t flags, cva_sim **out)
{
    if (!out) return fail(CVA_EINVAL, "out is NULL");
    *out = nullptr;
    int F = 0, CS = 0;
    std::vector<double> L;
    cva_status st = validate_model(model, &F, &CS, L);
    if (st != CVA_OK) return st;
    if (!pfs || n_pf < 1 || n_pf > kMaxPF) return fail(CVA_EINVAL, "n_pf must be in [1, 6]");
    if (!grid || !(grid->horizon > 0.0) || !is_fin(grid->horizon) || grid->n_steps < 1 || grid->n_steps > 254 ||
        grid->substeps < 1 || (int64_t)grid->n_steps * grid->substeps > (1 << 24))
        return fail(CVA_EINVAL, "grid: need horizon > 0, 1 <= n_steps <= 254, substeps >= 1");
    if (M < 1 || M > 0x7fffffffull) return fail(CVA_EINVAL, "M must be in [1, 2^31)");
    if (N < 1 || N > (1u << 24)) return fail(CVA_EINVAL, "N must be in [1, 2^24]");
    const int E = model->E, C = model->C, n = grid->n_steps, S = grid->substeps;
    const double Delta = grid->horizon / n;
    const double delta = pfs[0].delta;
    if (!(delta > 0.0)) return fail(CVA_EINVAL, "portfolio: delta must be > 0");
    const double pr = delta / Delta;
    const long ppp = std::lround(pr);
    if (ppp < 1 || std::fabs(pr - (double)ppp) > 1e-9 * pr)
        return fail(CVA_EINVAL, "portfolio: delta must be a whole number of pricing steps");
    int G = 1;
    for (int p = 0; p < n_pf; ++p) {
        const cva_portfolio_desc &d = pfs[p];
        if (d.n_swaps < 0) return fail(CVA_EINVAL, "portfolio: n_swaps < 0");
        if (d.n_swaps > 0 && (!d.ccy || !d.cpty || !d.omega || !d.n_periods || !d.notional))
            return fail(CVA_EINVAL, "portfolio: NULL swap array");
        if (std::fabs(d.delta - delta) > 1e-12) return fail(CVA_EINVAL, "portfolios must share delta");
        for (int s = 0; s < d.n_swaps; ++s) {
            if (d.ccy[s] < 0 || d.ccy[s] >= E) return fail(CVA_EINVAL, "swap: currency out of range");
            if (d.cpty[s] < 0 || d.cpty[s] >= C) return fail(CVA_EINVAL, "swap: counterparty out of range");
            if (d.omega[s] != 1 && d.omega[s] != -1) return fail(CVA_EINVAL, "swap: omega must be +1 or -1");
            if (d.n_periods[s] < 1 || d.n_periods[s] > kMaxG)
                return fail(CVA_EINVAL, "swap: n_periods must be in [1, 10]");
            if (!is_fin(d.notional[s])) return fail(CVA_EINVAL, "swap: notional must be finite");
            if (d.fixed_rate && !is_fin(d.fixed_rate[s])) return fail(CVA_EINVAL, "swap: fixed rate must be finite");
            G = std::max(G, (int)d.n_periods[s]);
        }
    }
    // the compiled instantiation of this shape if there is one (and its stochastic
    // intensities are the first counterparties), else the run-time-shape kernels
    bool cir_first = true;
    for (int c = 0; c < C; ++c)
        if ((model->cir_nu[c] > 0.0) != (c < CS)) cir_first = false;
    int Ginst = 0;
    const bool generic = (flags & CVA_GENERIC_KERNELS) || !cir_first || !outer_supported(E, C, CS, G, n_pf, &Ginst);
    if (generic) Ginst = G;
    if ((size_t)n_pf * C * E * Ginst > (size_t)kMaxW)
        return fail(CVA_ENOTSUP, "portfolio weights exceed constant memory: n_pf C E (longest schedule) must be <= " +
                                     std::to_string(kMaxW));

    Sim *s = new Sim();
    s->generic = generic;
    s->E = E; s->C = C; s->CS = CS; s->F = F; s->G = G; s->Ginst = Ginst; s->NPF = n_pf;
    s->n = n; s->S = S; s->ppp = (int)ppp; s->M = M; s->N = N; s->flags = flags;
    s->horizon = grid->horizon; s->delta = delta;

    // ---- constants ----
    SimConsts &k = s->consts;
    memset(&k, 0, sizeof(k));
    k.E = E; k.C = C; k.CS = CS; k.F = F; k.G = Ginst; k.NPF = n_pf; k.n = n; k.S = S; k.ppp = (int)ppp;
    const double ds = Delta / S;
    k.ds_d = ds;
    k.ds = (float)ds;
    k.sqds = (float)std::sqrt(ds);
    for (int i = 0; i < F; ++i)
        for (int j = 0; j <= i; ++j) k.L[i * (i + 1) / 2 + j] = (float)L[i * F + j];
    std::vector<HW> hw(E);
    for (int e = 0; e < E; ++e) {
        hw[e] = HW{model->hw_a[e], model->hw_sigma[e], model->curve[e]};
        k.hw_a_ds[e] = (float)(model->hw_a[e] * ds);
        k.hw_sig_sqds[e] = (float)(model->hw_sigma[e] * std::sqrt(ds));
        k.fx_drift_ds[e] = e ? (float)(-0.5 * model->fx_vol[e] * model->fx_vol[e] * ds) : 0.f;
        k.fx_sig_sqds[e] = e ? (float)(model->fx_vol[e] * std::sqrt(ds)) : 0.f;
        k.r0[e] = (float)model->curve[e];
        k.lchi0[e] = e ? (float)std::log(model->fx0[e]) : 0.f;
        k.fix0_m1[e] = (float)std::expm1(model->curve[e] * delta);   // 1/ZC_0(delta) - 1
    }
    for (int c = 0, pos = 2 * E - 1; c < C; ++c) {
        const bool stoch = model->cir_nu[c] > 0.0;
        k.gpos[c] = stoch ? pos++ : -1;
        k.cir_kds[c] = stoch ? (float)(model->cir_kappa[c] * ds) : 0.f;
        k.cir_ktds[c] = stoch ? (float)(model->cir_kappa[c] * model->cir_theta[c] * ds) : 0.f;
        k.cir_nu_sqds[c] = stoch ? (float)(model->cir_nu[c] * std::sqrt(ds)) : 0.f;
        k.gamma0[c] = (float)model->gamma0[c];
        k.lgd[c] = (float)(1.0 - model->recovery[c]);
    }
    // quanto drift of r^e under the reference measure: -rho_e sigma^chi_e sigma^r_e
    std::vector<double> quanto(E, 0.0);
    for (int e = 1; e < E; ++e) {
        const int pr_ = e, px = E - 1 + e;
        quanto[e] = model->corr[pr_ * F + px] * model->fx_vol[e] * model->hw_sigma[e];
    }

    // ---- tables ----
    std::vector<float> drift((size_t)n * S * E);
    for (int q = 0; q < n * S; ++q)
        for (int e = 0; e < E; ++e)
            drift[(size_t)q * E + e] = (float)((hw[e].theta(q * ds) - quanto[e]) * ds);
    // bond tables: for T = (g+1) delta >= t_j, (lnA(t_j, T), B(t_j, T)) and the
    // increments from T - delta (log-ratio of consecutive bond prices is
    // dlnA - dB r), all in FP64 before rounding
    std::vector<float4> zc((size_t)(n + 1) * E * Ginst, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<int> date_p(n + 1, 0);
    for (int j = 1; j <= n; ++j) date_p[j] = (j - 1) / (int)ppp;
    for (int j = 0; j <= n; ++j) {
        const double t = j * Delta;
        for (int e = 0; e < E; ++e)
            for (int g = 0; g < Ginst; ++g) {
                const double T = (g + 1) * delta;
                if (T + 1e-12 < t) continue;
                const double lnA = hw[e].lnA(t, T), B = hw[e].B(t, T);
                double dlnA = 0.0, dB = 0.0;
                if (T - delta + 1e-12 >= t) {
                    dlnA = lnA - hw[e].lnA(t, T - delta);
                    dB = B - hw[e].B(t, T - delta);
                }
                zc[((size_t)j * E + e) * Ginst + g] = make_float4((float)lnA, (float)B, (float)dlnA, (float)dB);
            }
    }
    const int n_periods = n / (int)ppp + 1;
    std::vector<float2> fix((size_t)(n_periods + 1) * E);
    for (int p = 0; p <= n_periods; ++p)
        for (int e = 0; e < E; ++e)
            fix[(size_t)p * E + e] = make_float2((float)hw[e].lnA(p * delta, (p + 1) * delta),
                                                 (float)hw[e].B(p * delta, (p + 1) * delta));
    // date-bucketed weights, App. B formula regrouped by (counterparty, currency, reset date)
    memset(&s->weights, 0, sizeof(SimWeights));
    {
        // accumulate in FP64, then round once
        std::vector<double> wA((size_t)n_pf * C * E * Ginst, 0.0), wK(wA.size(), 0.0);
        for (int p = 0; p < n_pf; ++p) {
            const cva_portfolio_desc &d = pfs[p];
            for (int sw = 0; sw < d.n_swaps; ++sw) {
                const int e = d.ccy[sw], c = d.cpty[sw], m = d.n_periods[sw];
                double ann = 0.0;
                for (int g = 1; g <= m; ++g) ann += std::exp(-model->curve[e] * g * delta);
                const double Sigma = d.fixed_rate ? d.fixed_rate[sw]
                                                  : (1.0 - std::exp(-model->curve[e] * m * delta)) / (delta * ann);
                const double wN = d.omega[sw] * d.notional[sw];
                const size_t base = (((size_t)p * C + c) * E + e) * Ginst;
                for (int h = 0; h < m; ++h) wA[base + h] += wN;                  // float notional, period h
                for (int g = 1; g <= m; ++g) wK[base + g - 1] += delta * wN * Sigma;   // fixed coupon at g
            }
        }
        for (size_t i = 0; i < wA.size(); ++i) {
            s->weights.wA[i] = (float)wA[i];
            s->weights.wK[i] = (float)wK[i];
        }
    }
    s->recovery.assign(model->recovery, model->recovery + C);

    // ---- device buffers ----
    const size_t Mz = (size_t)M;
#define TRY_ALLOC(p, n_)                           \
    do {                                           \
        cva_status _s = dev_alloc(&(p), (n_));     \
        if (_s != CVA_OK) {                        \
            free_sim(s);                           \
            return _s;                             \
        }                                          \
    } while (0)
    TRY_ALLOC(s->d_zc, zc.size());
    TRY_ALLOC(s->d_fix, fix.size());
    TRY_ALLOC(s->d_date_p, date_p.size());
    TRY_ALLOC(s->d_drift, drift.size());
    TRY_ALLOC(s->d_features, (size_t)(n + 1) * F * Mz);
    TRY_ALLOC(s->d_disc, (size_t)(n + 1) * Mz);
    TRY_ALLOC(s->d_thr, (size_t)(n + 1) * C * Mz);
    TRY_ALLOC(s->d_expo, (size_t)n_pf * (n + 1) * C * Mz);
    if (flags & CVA_KEEP_EXPOSURES) TRY_ALLOC(s->d_mtm, (size_t)n_pf * (n + 1) * C * Mz);
    TRY_ALLOC(s->d_targets, (size_t)n_pf * n * Mz);
    if (flags & CVA_KEEP_DEFAULTS) TRY_ALLOC(s->d_idx, Mz * N * C);
    if (N <= 65535u) {
        uint16_t *cnt = nullptr;
        TRY_ALLOC(cnt, (size_t)(n + 1) * C * Mz);
        s->d_cnt = cnt;
    } else {
        uint32_t *cnt = nullptr;
        TRY_ALLOC(cnt, (size_t)(n + 1) * C * Mz);
        s->d_cnt = cnt;
    }
    TRY_ALLOC(s->d_const_img, sizeof(SimConsts) + sizeof(SimWeights));
#undef TRY_ALLOC
    cudaError_t e1 = cudaMemcpy(s->d_zc, zc.data(), zc.size() * sizeof(float4), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(s->d_fix, fix.data(), fix.size() * sizeof(float2), cudaMemcpyHostToDevice);
    cudaError_t e3 = cudaMemcpy(s->d_date_p, date_p.data(), date_p.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaError_t e4 = cudaMemcpy(s->d_drift, drift.data(), drift.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaError_t e5 = cudaMemcpy(s->d_const_img, &s->consts, sizeof(SimConsts), cudaMemcpyHostToDevice);
    cudaError_t e6 = cudaMemcpy(s->d_const_img + sizeof(SimConsts), &s->weights, sizeof(SimWeights), cudaMemcpyHostToDevice);
    for (cudaError_t e : {e1, e2, e3, e4, e5, e6})
        if (e != cudaSuccess) {
            free_sim(s);
            return cuda_fail(e, "table upload");
        }
    if (flags & CVA_PROFILE)
        for (cudaEvent_t &ev : s->ev)
            if (cudaEventCreate(&ev) != cudaSuccess) {
                free_sim(s);
                return fail(CVA_ECUDA, "event creation failed");
            }
    *out = reinterpret_cast<cva_sim *>(s);
    return CVA_OK;
}

cva_status cva_simulate(cva_sim *sim, uint64_t seed, uint64_t k0, void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    if (k0 + s.M > 0xffffffffull) return fail(CVA_EINVAL, "k0 + M must fit in 32 bits");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (s.ev[0]) CVA_CUDA_TRY(cudaEventRecord(s.ev[0], st));
    cva_status r = launch_outer(s, seed, k0, st);   // records ev[1] between its two kernels
    if (r != CVA_OK) return r;
    if (s.ev[2]) CVA_CUDA_TRY(cudaEventRecord(s.ev[2], st));
    r = launch_inner(s, seed, k0, st);
    if (r != CVA_OK) return r;
    if (s.ev[3]) CVA_CUDA_TRY(cudaEventRecord(s.ev[3], st));
    return CVA_OK;
}

cva_status cva_simulate_twin(cva_sim *sim, uint64_t seed, uint64_t k0, int date, uint32_t copy, void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    if (date < 0 || date > s.n) return fail(CVA_EINVAL, "twin: branch date outside [0, n]");
    if (copy < 1 || copy >= (1u << 24)) return fail(CVA_EINVAL, "twin: copy must be in [1, 2^24)");
    s.branch_date = date;
    s.branch = copy;
    const cva_status r = cva_simulate(sim, seed, k0, stream);
    s.branch_date = 1 << 30;
    s.branch = 0;
    return r;
}

cva_status cva_twin_l2(const float *phi_dev, const float *xi1_dev, const float *xi2_dev, uint64_t M, double *out2,
                       void *stream)
{
    return twin_l2_fp64(phi_dev, xi1_dev, xi2_dev, M, out2, reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_nested_reference(cva_sim *sim, uint64_t seed, uint64_t k0, int pf, int date, int copies,
                                float *out_dev, void *stream)
{
    if (!sim || !out_dev) return fail(CVA_EINVAL, "nested: NULL argument");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "portfolio index out of range");
    if (date < 0 || date >= s.n) return fail(CVA_EINVAL, "nested: date outside [0, n)");
    if (copies < 1 || copies >= (1 << 24)) return fail(CVA_EINVAL, "nested: copies must be in [1, 2^24)");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float *row = s.d_targets + ((size_t)pf * s.n + date) * s.M;
    for (int b = 1; b <= copies; ++b) {
        cva_status r = cva_simulate_twin(sim, seed, k0, date, (uint32_t)b, stream);
        if (r == CVA_OK) r = accumulate_mean(out_dev, row, s.M, b == 1, b == copies, copies, st);
        if (r != CVA_OK) return r;
    }
    return CVA_OK;
}

cva_status cva_relative_rmse(const float *phi_dev, const float *ref_dev, uint64_t M, double *out2, void *stream)
{
    return relative_rmse_fp64(phi_dev, ref_dev, M, out2, reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_cva0_partials(const float *xi0_dev, uint64_t M, double *out3_host, void *stream)
{
    if (!out3_host) return fail(CVA_EINVAL, "cva0_partials: NULL output");
    double h[2];
    cva_status r = sums_fp64(xi0_dev, M, h, reinterpret_cast<cudaStream_t>(stream));
    if (r != CVA_OK) return r;
    out3_host[0] = (double)M;
    out3_host[1] = h[0];
    out3_host[2] = h[1];
    return CVA_OK;
}

cva_status cva_cva0_combine(const double *parts_host, int n_parts, double *out2_host)
{
    if (!parts_host || !out2_host || n_parts < 1) return fail(CVA_EINVAL, "cva0_combine: bad arguments");
    double m = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < n_parts; ++i) {   // in part order
        m += parts_host[3 * i];
        s1 += parts_host[3 * i + 1];
        s2 += parts_host[3 * i + 2];
    }
    if (!(m > 0.0)) return fail(CVA_EINVAL, "cva0_combine: no paths");
    mean_se_from_sums(m, s1, s2, out2_host);
    return CVA_OK;
}

cva_status cva_regress_partial(const float *targets_dev, const float *features_dev, int F, uint64_t M, int basis,
                               const float *centre_dev, double *gram_host, void *stream)
{
    return lsq_normal_partial(targets_dev, features_dev, F, M, basis, centre_dev, gram_host,
                              reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_regress_solve(const double *gram_host, int F, int basis, const double *centre_host,
                             double *coef_centred_host, double *coef_raw_host, int *dropped_host)
{
    return lsq_solve_normal_host(gram_host, F, basis, centre_host, coef_centred_host, coef_raw_host, dropped_host);
}

cva_status cva_regress_predict(const float *features_dev, int F, uint64_t M, int basis, const float *centre_dev,
                               const double *coef_centred_host, float *pred_dev, void *stream)
{
    return lsq_predict_centred(features_dev, F, M, basis, centre_dev, coef_centred_host, pred_dev,
                               reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_inner_cost_ratio(double t1, uint32_t N1, double t2, uint32_t N2, double *kappa_out)
{
    if (!kappa_out) return fail(CVA_EINVAL, "cost_ratio: NULL output");
    if (!is_fin(t1) || !is_fin(t2) || !(t1 > 0.0) || !(t2 > 0.0) || N1 == N2)
        return fail(CVA_EINVAL, "cost_ratio: need two positive timings at different N");
    // t = c M (kappa + N) at both N: two equations in c M and kappa (eq. (l:ratio))
    const double kappa = (t1 * (double)N2 - t2 * (double)N1) / (t2 - t1);
    if (!is_fin(kappa)) return fail(CVA_EINVAL, "cost_ratio: equal timings");
    *kappa_out = kappa;
    return CVA_OK;
}

cva_status cva_oversim_choice(const double *qr_host, int n, double kappa, double budget, double *Ni_host,
                              double *N_out, double *M_out)
{
    if (!qr_host || !Ni_host || !N_out || n < 1) return fail(CVA_EINVAL, "oversim_choice: bad arguments");
    if (!is_fin(kappa) || !(kappa >= 0.0)) return fail(CVA_EINVAL, "oversim_choice: kappa must be >= 0");
    // Prop. 1: at a fixed budget M (N + kappa) the variance of the empirical loss,
    // (R + Q / N) (N + kappa) / budget, is smallest at N_i = sqrt(Q_i kappa / R_i)
    // (eq. (e:optom)); Heuristic 1 takes the mean of the N_i over the dates and
    // spends the budget on M = budget / (N + kappa) outer paths.
    double sum = 0.0;
    int used = 0;
    for (int i = 0; i < n; ++i) {
        const double Q = qr_host[2 * i], R = qr_host[2 * i + 1];
        if (is_fin(Q) && is_fin(R) && R > 0.0 && Q >= 0.0) {
            Ni_host[i] = std::sqrt(Q * kappa / R);
            sum += Ni_host[i];
            ++used;
        } else {
            Ni_host[i] = std::nan("");   // no optimum: R <= 0 or Q < 0 (estimates at a degenerate date)
        }
    }
    *N_out = used > 0 ? sum / used : std::nan("");
    if (M_out) *M_out = (used > 0 && budget > 0.0) ? budget / (*N_out + kappa) : std::nan("");
    return used > 0 ? CVA_OK : fail(CVA_ENUMERIC, "oversim_choice: no date with R > 0 and Q >= 0");
}

cva_status cva_oversim_stats(const cva_sim *sim, int pf, const float *pred_dev, uint64_t seed, double *qr_host,
                             void *stream)
{
    if (!sim || !pred_dev || !qr_host) return fail(CVA_EINVAL, "oversim: NULL argument");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "portfolio index out of range");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((s.M + 255) / 256);
    const int cols = 3 * s.n;
    double *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * ((size_t)blocks * cols + cols)) != cudaSuccess)
        return fail(CVA_ENOMEM, "oversim: scratch allocation failed");
    cva_status r = launch_oversim(s, pf, pred_dev, seed, buf, blocks, st);
    if (r == CVA_OK) r = sum_columns_fp64(buf, (int)blocks, cols, buf + (size_t)blocks * cols, st);
    std::vector<double> h(cols, 0.0);
    if (r == CVA_OK) {
        cudaError_t e = cudaMemcpyAsync(h.data(), buf + (size_t)blocks * cols, sizeof(double) * cols,
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "oversim: copy back");
    }
    cudaFree(buf);
    if (r != CVA_OK) return r;
    const double M = (double)s.M;
    for (int i = 0; i < s.n; ++i) {
        const double m1 = h[3 * i] / M, m2 = h[3 * i + 1] / M, m12 = h[3 * i + 2] / M;
        qr_host[2 * i] = m2 - m12;           // Q_i = E[g^2] - E[g0 g1] = E[Var(g | Y)]
        qr_host[2 * i + 1] = m12 - m1 * m1;  // R_i = E[g0 g1] - E[g]^2 = Var(E[g | Y])
    }
    return CVA_OK;
}

cva_status cva_sim_kernel_ms(const cva_sim *sim, float out_ms[3])
{
    if (!sim || !out_ms) return fail(CVA_EINVAL, "NULL argument");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    if (!s.ev[0]) return fail(CVA_EINVAL, "sim was not created with CVA_PROFILE");
    CVA_CUDA_TRY(cudaEventSynchronize(s.ev[3]));
    CVA_CUDA_TRY(cudaEventElapsedTime(&out_ms[0], s.ev[0], s.ev[1]));
    CVA_CUDA_TRY(cudaEventElapsedTime(&out_ms[1], s.ev[1], s.ev[2]));
    CVA_CUDA_TRY(cudaEventElapsedTime(&out_ms[2], s.ev[2], s.ev[3]));
    return CVA_OK;
}

cva_status cva_sim_view(const cva_sim *sim, int what, void **dev_ptr, size_t *bytes)
{
    if (!sim || !dev_ptr || !bytes) return fail(CVA_EINVAL, "NULL argument");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    const size_t M = s.M, n = s.n;
    void *p = nullptr;
    size_t b = 0;
    switch (what) {
    case CVA_VIEW_FEATURES: p = s.d_features; b = (n + 1) * s.F * M * 4; break;
    case CVA_VIEW_TARGETS: p = s.d_targets; b = (size_t)s.NPF * n * M * 4; break;
    case CVA_VIEW_DISCOUNT: p = s.d_disc; b = (n + 1) * M * 4; break;
    case CVA_VIEW_THRESHOLD: p = s.d_thr; b = (n + 1) * s.C * M * 4; break;
    case CVA_VIEW_EXPOSURE: p = s.d_expo; b = (size_t)s.NPF * (n + 1) * s.C * M * 4; break;
    case CVA_VIEW_MTM: p = s.d_mtm; b = (size_t)s.NPF * (n + 1) * s.C * M * 4; break;
    case CVA_VIEW_DEFAULTS: p = s.d_idx; b = M * s.N * s.C; break;
    default: return fail(CVA_EINVAL, "unknown view");
    }
    if (!p) return fail(CVA_EINVAL, "view not kept (see the flags of cva_sim_create)");
    *dev_ptr = p;
    *bytes = b;
    return CVA_OK;
}

cva_status cva_sim_shape(const cva_sim *sim, int64_t out[6])
{
    if (!sim || !out) return fail(CVA_EINVAL, "NULL argument");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    out[0] = (int64_t)s.M;
    out[1] = s.N;
    out[2] = s.n;
    out[3] = s.F;
    out[4] = s.C;
    out[5] = s.NPF;
    return CVA_OK;
}

void cva_sim_destroy(cva_sim *sim) { free_sim(reinterpret_cast<Sim *>(sim)); }

cva_status cva_cva0(const float *xi0_dev, uint64_t M, double *out2_host, void *stream)
{
    return mean_fp64(xi0_dev, M, out2_host, reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_regress(const float *targets_dev, const float *features_dev, int F, uint64_t M, int basis,
                       float *pred_dev, double *coef_host, void *stream)
{
    return lsq_grouped_strided(features_dev, 0, targets_dev, 0, pred_dev, 0, F, M, basis, 1, coef_host,
                               reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_regress_all(const cva_sim *sim, int pf, int basis, float *pred_dev, double *coef_host,
                           void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "portfolio index out of range");
    if (s.n < 2) return fail(CVA_EINVAL, "need at least two pricing steps");
    const size_t M = s.M;
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : s.F + 1;
    const float *feat1 = s.d_features + (size_t)s.F * M;                 // date 1
    const float *targ1 = s.d_targets + ((size_t)pf * s.n + 1) * M;        // date 1
    float *pred1 = pred_dev ? pred_dev + M : nullptr;
    return lsq_grouped_strided(feat1, (size_t)s.F * M, targ1, M, pred1, M, s.F, M, basis, s.n - 1,
                               coef_host ? coef_host + m : nullptr, reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_regress_batched_static(const float *targets_dev, const float *features_dev, int groups, int F,
                                      uint64_t M, int basis, float *pred_dev, double *coef_host, void *stream)
{
    return lsq_batched_static(targets_dev, features_dev, groups, F, M, basis, pred_dev, coef_host,
                              reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_regress_portfolios(cva_sim *sim, int basis, float *pred_dev, double *coef_host, void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    if (s.n < 2) return fail(CVA_EINVAL, "need at least two pricing steps");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const size_t M = s.M;
    const int m = (basis == CVA_BASIS_POLY2) ? 3 : s.F + 1;
    LsqJob j;
    j.feat0 = s.d_features + (size_t)s.F * M;       // date 1
    j.feat_stride = (size_t)s.F * M;
    j.targ0 = s.d_targets + M;                       // portfolio 0, date 1
    j.targ_stride = M;
    j.targ_tstride = (size_t)s.n * M;
    j.pred0 = pred_dev ? pred_dev + M : nullptr;
    j.pred_stride = M;
    j.pred_tstride = (size_t)s.n * M;
    j.F = s.F;
    j.M = M;
    j.basis = basis;
    j.groups = s.n - 1;
    j.nt = s.NPF;
    j.chunk_target = s.tune_lsq_chunks;
    const size_t need = lsq_scratch_need(j);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CVA_CUDA_TRY(cudaStreamIsCapturing(cs, &cap));
    if (s.lsq_cap < need) {
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CVA_EINVAL, "regress_portfolios: call once before capturing so that the scratch exists");
        CVA_CUDA_TRY(cudaStreamSynchronize(cs));
        cudaFree(s.d_lsq);
        s.d_lsq = nullptr;
        s.lsq_cap = 0;
        if (dev_alloc(&s.d_lsq, need) != CVA_OK) return CVA_ENOMEM;
        s.lsq_cap = need;
    }
    if (!coef_host) return lsq_launch(j, s.d_lsq, s.lsq_cap, nullptr, cs);
    std::vector<double> tmp((size_t)j.groups * j.nt * m);
    cva_status r = lsq_launch(j, s.d_lsq, s.lsq_cap, tmp.data(), cs);
    if (r != CVA_OK) return r;
    for (int g = 0; g < j.groups; ++g)          // [date][portfolio][m] -> [portfolio][date][m]
        for (int t = 0; t < j.nt; ++t)
            for (int i = 0; i < m; ++i)
                coef_host[((size_t)t * s.n + (g + 1)) * m + i] = tmp[((size_t)g * j.nt + t) * m + i];
    return CVA_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::string, std::array<int, 5>> g_tune_cache;

float time_once(cudaStream_t st, const std::function<cva_status()> &f, cva_status *err)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    *err = f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}
}  // namespace

cva_status cva_autotune(cva_sim *sim, uint64_t seed, int basis, char *report, size_t report_len, void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    CVA_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CVA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    char key[512];
    snprintf(key, sizeof(key), "%s|E%d C%d CS%d G%d P%d n%d S%d M%llu N%u b%d", prop.name, s.E, s.C, s.CS, s.Ginst,
             s.NPF, s.n, s.S, (unsigned long long)s.M, s.N, basis);
    std::array<int, 5> best = {s.tune_sim_block, s.tune_price_block, s.tune_inner_P, s.tune_lsq_chunks, s.tune_price_pf};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        cva_status err = CVA_OK;
        auto measure = [&](int which, int value) -> float {
            std::array<int, 5> save = {s.tune_sim_block, s.tune_price_block, s.tune_inner_P, s.tune_lsq_chunks,
                                       s.tune_price_pf};
            int *slot[5] = {&s.tune_sim_block, &s.tune_price_block, &s.tune_inner_P, &s.tune_lsq_chunks,
                            &s.tune_price_pf};
            *slot[which] = value;
            auto run = [&]() -> cva_status {
                if (which == 3) return cva_regress_portfolios(sim, basis, nullptr, nullptr, cs);
                if (which == 2) return launch_inner(s, seed, 0, cs);
                return launch_outer(s, seed, 0, cs);
            };
            time_once(cs, run, &err);              // warm-up
            float t = 1e30f;
            for (int rep = 0; rep < 2 && err == CVA_OK; ++rep) t = fminf(t, time_once(cs, run, &err));
            s.tune_sim_block = save[0];
            s.tune_price_block = save[1];
            s.tune_inner_P = save[2];
            s.tune_lsq_chunks = save[3];
            s.tune_price_pf = save[4];
            return err == CVA_OK ? t : 1e30f;
        };
        // portfolios per pricing block: the divisors of n_pf among 1, 2, 3 (weights in
        // constant memory), or 0 (every portfolio per thread, weights in shared memory)
        std::vector<int> ppf = {4, 0, 1};
        for (int v : {2, 3})
            if (s.NPF % v == 0) ppf.push_back(v);
        const std::vector<std::vector<int>> cand = {{64, 128}, {128, 256}, {2, 4, 8}, {1216, 2432, 4864, 9728}, ppf};
        // the first pass needs valid outputs of the earlier kernels: simulate once
        cva_status r = cva_simulate(sim, seed, 0, stream);
        if (r != CVA_OK) return r;
        // the pricing form (portfolios per block) before its block size: the best block
        // size differs between the constant-memory and the shared-memory forms
        for (int w : {0, 4, 1, 2, 3}) {
            float tb = 1e30f;
            for (int v : cand[w]) {
                const float t = measure(w, v);
                if (t < tb) {
                    tb = t;
                    best[w] = v;
                }
            }
            int *slot[5] = {&s.tune_sim_block, &s.tune_price_block, &s.tune_inner_P, &s.tune_lsq_chunks,
                            &s.tune_price_pf};
            *slot[w] = best[w];
        }
        if (err != CVA_OK) return err;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    s.tune_sim_block = best[0];
    s.tune_price_block = best[1];
    s.tune_inner_P = best[2];
    s.tune_lsq_chunks = best[3];
    s.tune_price_pf = best[4];
    if (report && report_len)
        snprintf(report, report_len, "{\"sim_block\": %d, \"price_block\": %d, \"inner_paths_per_block\": %d, "
                                     "\"lsq_chunk_target\": %d, \"portfolios_per_price_block\": %d, \"cached\": %s}",
                 best[0], best[1], best[2], best[3], best[4], cached ? "true" : "false");
    return CVA_OK;
}

cva_status cva_regress_alive(cva_sim *sim, int pf, float *pred_dev, double *coef_host, int *dropped_host,
                             void *stream)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    return alive_regress(*reinterpret_cast<Sim *>(sim), pf, pred_dev, coef_host, dropped_host,
                         reinterpret_cast<cudaStream_t>(stream));
}

cva_status cva_set_tiles(cva_sim *sim, int sim_block, int price_block, int inner_paths_per_block,
                         int lsq_chunk_target, int portfolios_per_price_block)
{
    if (!sim) return fail(CVA_EINVAL, "sim is NULL");
    Sim &s = *reinterpret_cast<Sim *>(sim);
    if (sim_block != 64 && sim_block != 128) return fail(CVA_EINVAL, "sim_block must be 64 or 128");
    if (price_block != 128 && price_block != 256) return fail(CVA_EINVAL, "price_block must be 128 or 256");
    if (inner_paths_per_block != 0 && inner_paths_per_block != 2 && inner_paths_per_block != 4 &&
        inner_paths_per_block != 8)
        return fail(CVA_EINVAL, "inner_paths_per_block must be 0, 2, 4 or 8");
    if (lsq_chunk_target < 152 || lsq_chunk_target > (1 << 20))
        return fail(CVA_EINVAL, "lsq_chunk_target must lie in [152, 2^20]");
    if (portfolios_per_price_block < 0 || portfolios_per_price_block > 4 ||
        (portfolios_per_price_block >= 1 && portfolios_per_price_block <= 3 &&
         s.NPF % portfolios_per_price_block != 0))
        return fail(CVA_EINVAL, "pricing form must be 0 (shared memory), 1, 2 or 3 dividing the number of portfolios "
                                "(constant memory) or 4 (tensor cores)");
    s.tune_sim_block = sim_block;
    s.tune_price_block = price_block;
    s.tune_inner_P = inner_paths_per_block;
    s.tune_lsq_chunks = lsq_chunk_target;
    s.tune_price_pf = portfolios_per_price_block;
    return CVA_OK;
}

int cva_mlp_num_params(int hidden) { return mlp_num_params(hidden); }

cva_status cva_mlp_set_wait_limit(uint32_t grid_polls)
{
    mlp_wide_set_grid_polls(grid_polls);
    return CVA_OK;
}

cva_status cva_mlp_kernel_timing(int on, double *ms_host, uint64_t *launches_host)
{
    mlp_kernel_timing(on != 0, ms_host, launches_host);
    return CVA_OK;
}

cva_status cva_mlp_plan(uint64_t M, int hidden, int n_batches, int32_t *out4_host)
{
    if (!out4_host) return fail(CVA_EINVAL, "mlp_plan: NULL output");
    return mlp_plan(M, hidden, n_batches, out4_host);
}

cva_status cva_mlp_fit(const float *targets_dev, const float *features_dev, int F, uint64_t M, int hidden,
                       int n_batches, int epochs, float lr, float *params_dev, float *pred_dev, float *loss_dev,
                       void *stream)
{
    if (!targets_dev || !features_dev || !params_dev) return fail(CVA_EINVAL, "mlp: NULL pointer");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cva_status r = mlp_begin(st);
    if (r == CVA_OK)
        r = mlp_fit_dates(features_dev, 0, targets_dev, 0, 1, F, M, hidden, n_batches, epochs, lr, 0, params_dev,
                          pred_dev, nullptr, loss_dev, st);
    return r == CVA_OK ? mlp_finish(st) : r;
}

cva_status cva_mlp_first_gradient(const float *targets_dev, const float *features_dev, int F, uint64_t M,
                                  int hidden, int n_batches, float lr, float *params_dev, float *grad_dev,
                                  void *stream)
{
    if (!targets_dev || !features_dev || !params_dev || !grad_dev) return fail(CVA_EINVAL, "mlp: NULL pointer");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cva_status r = mlp_begin(st);
    if (r == CVA_OK)
        r = mlp_fit_dates(features_dev, 0, targets_dev, 0, 1, F, M, hidden, n_batches, 1, lr, 1, params_dev, nullptr,
                          grad_dev, nullptr, st);
    return r == CVA_OK ? mlp_finish(st) : r;
}

cva_status cva_mlp_regress_all(const cva_sim *sim, int pf, int hidden, int n_batches, int epochs, float lr,
                               float *params_dev, float *pred_dev, void *stream)
{
    if (!sim || !params_dev) return fail(CVA_EINVAL, "mlp: NULL pointer");
    const Sim &s = *reinterpret_cast<const Sim *>(sim);
    if (pf < 0 || pf >= s.NPF) return fail(CVA_EINVAL, "portfolio index out of range");
    const size_t M = s.M;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cva_status r = mlp_begin(st);
    if (r == CVA_OK && s.n >= 2)   // dates n-1 .. 1
        r = mlp_fit_dates(s.d_features + (size_t)s.F * M, (size_t)s.F * M, s.d_targets + ((size_t)pf * s.n + 1) * M, M,
                          s.n - 1, s.F, M, hidden, n_batches, epochs, lr, 0, params_dev,
                          pred_dev ? pred_dev + M : nullptr, nullptr, nullptr, st);
    return r == CVA_OK ? mlp_finish(st) : r;
}

int cva_grad_num_params(int E, int C) { return 3 * E - 1 + 3 * C; }

cva_status cva_par_rates(const cva_model_desc *model, const cva_portfolio_desc *pf, double *rates_host)
{
    int F = 0, CS = 0;
    std::vector<double> L;
    cva_status st = validate_model(model, &F, &CS, L);
    if (st != CVA_OK) return st;
    if (!pf || !rates_host || pf->n_swaps < 0 || !(pf->delta > 0.0)) return fail(CVA_EINVAL, "par_rates: bad portfolio");
    for (int s = 0; s < pf->n_swaps; ++s) {
        const int e = pf->ccy[s], m = pf->n_periods[s];
        if (e < 0 || e >= model->E || m < 1) return fail(CVA_EINVAL, "par_rates: bad swap");
        double ann = 0.0;
        for (int g = 1; g <= m; ++g) ann += std::exp(-model->curve[e] * g * pf->delta);
        rates_host[s] = (1.0 - std::exp(-model->curve[e] * m * pf->delta)) / (pf->delta * ann);
    }
    return CVA_OK;
}

cva_status cva_grad_cva0(const cva_model_desc *model, const cva_portfolio_desc *pf, const cva_grid *grid,
                         uint64_t M, uint64_t seed, uint64_t k0, int ckpt_every, int forward_only,
                         double *grad_host, double *cva0_host, void *stream)
{
    if (!cva0_host || (!forward_only && !grad_host)) return fail(CVA_EINVAL, "grad: NULL output");
    if (M < 1 || M > 0x7fffffffull || k0 + M > 0xffffffffull) return fail(CVA_EINVAL, "grad: bad path range");
    cva_sim *hs = nullptr;
    cva_status st = cva_sim_create(model, pf, 1, grid, 1, 1, 0, &hs);   // tables only
    if (st != CVA_OK) return st;
    Sim &s = *reinterpret_cast<Sim *>(hs);
    const int E = s.E, C = s.C, n = s.n, S = s.S, G = s.Ginst, F = s.F;
    const int NPAR = 3 * E - 1 + 3 * C, NV = 2 * E + 3 * C;
    const int K = ckpt_every > 0 ? ckpt_every : 10;
    const double Delta = s.horizon / n, ds = Delta / S, delta = s.delta;
    const int ppp = s.ppp, periods = n / ppp + 1;
    std::vector<HW> hw(E);
    for (int e = 0; e < E; ++e) hw[e] = HW{model->hw_a[e], model->hw_sigma[e], model->curve[e]};
    // derivatives of ln A(t, T) of the flat-curve Hull-White bond with respect to f and sigma:
    //   d/df = -(T - t) + B(t, T),  d/dsigma = -sigma/(2a) (1 - e^{-2at}) B(t, T)^2
    auto dA = [&](int e, double t, double T, double &df, double &dsg) {
        const double b = hw[e].B(t, T), a = hw[e].a, sg = hw[e].s;
        df = -(T - t) + b;
        dsg = -sg / (2.0 * a) * (1.0 - std::exp(-2.0 * a * t)) * b * b;
    };
    std::vector<float4> dzc((size_t)(n + 1) * E * G, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int j = 0; j <= n; ++j) {
        const double t = j * Delta;
        for (int e = 0; e < E; ++e)
            for (int g = 0; g < G; ++g) {
                const double T = (g + 1) * delta;
                if (T + 1e-12 < t) continue;
                double df, dsg, df0 = 0.0, dsg0 = 0.0;
                dA(e, t, T, df, dsg);
                if (T - delta + 1e-12 >= t) dA(e, t, T - delta, df0, dsg0);
                else df0 = df, dsg0 = dsg;
                dzc[((size_t)j * E + e) * G + g] = make_float4((float)df, (float)dsg, (float)(df - df0), (float)(dsg - dsg0));
            }
    }
    std::vector<float2> dfix((size_t)(periods + 1) * E);
    for (int p = 0; p <= periods; ++p)
        for (int e = 0; e < E; ++e) {
            double df, dsg;
            dA(e, p * delta, (p + 1) * delta, df, dsg);
            dfix[(size_t)p * E + e] = make_float2((float)df, (float)dsg);
        }
    std::vector<float> rho(E, 0.f), sig(2 * E + 3 * C, 0.f);
    std::vector<float2> ddrift((size_t)n * S * E);
    for (int e = 1; e < E; ++e) rho[e] = (float)model->corr[e * F + (E - 1 + e)];
    for (int q = 0; q < n * S; ++q)
        for (int e = 0; e < E; ++e) {
            const double a = hw[e].a, sg = hw[e].s, t = q * ds;
            const double dq = e ? rho[e] * model->fx_vol[e] : 0.0;   // d quanto / d sigma^r
            ddrift[(size_t)q * E + e] = make_float2((float)(a * ds),
                                                    (float)((sg / a * (1.0 - std::exp(-2.0 * a * t)) - dq) * ds));
        }
    for (int e = 0; e < E; ++e) {
        sig[e] = (float)model->hw_sigma[e];
        sig[E + e] = e ? (float)model->fx_vol[e] : 0.f;
    }
    for (int c = 0; c < C; ++c) {
        sig[2 * E + c] = (float)model->cir_kappa[c];
        sig[2 * E + C + c] = (float)model->cir_theta[c];
        sig[2 * E + 2 * C + c] = (float)model->cir_nu[c];
    }
    AdjBuffers b;
    b.K = K;
    b.nseg = (n + K - 1) / K;
    b.forward_only = forward_only ? 1 : 0;
    const size_t Mz = M;
    const unsigned blocks = (unsigned)((M + 127) / 128);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    auto cleanup = [&]() {
        cudaFree(b.dzc);
        cudaFree(b.dfix);
        cudaFree(b.ddrift);
        cudaFree(b.rho);
        cudaFree(b.sig);
        cudaFree(b.ckpt);
        cudaFree(b.ckpt_I0);
        cudaFree(b.fixr);
        cudaFree(b.part);
        cudaFree(b.sum);
        cva_sim_destroy(hs);
    };
    if (dev_alloc(&b.dzc, dzc.size()) != CVA_OK || dev_alloc(&b.dfix, dfix.size()) != CVA_OK ||
        dev_alloc(&b.ddrift, ddrift.size()) != CVA_OK || dev_alloc(&b.rho, rho.size()) != CVA_OK ||
        dev_alloc(&b.sig, sig.size()) != CVA_OK || dev_alloc(&b.ckpt, (size_t)b.nseg * NV * Mz) != CVA_OK ||
        dev_alloc(&b.ckpt_I0, (size_t)b.nseg * Mz) != CVA_OK ||
        dev_alloc(&b.fixr, (size_t)(periods + 1) * E * Mz) != CVA_OK ||
        dev_alloc(&b.part, (size_t)blocks * (NPAR + 1)) != CVA_OK || dev_alloc(&b.sum, (size_t)NPAR + 1) != CVA_OK) {
        cleanup();
        return CVA_ENOMEM;
    }
    cudaError_t e1 = cudaMemcpyAsync(b.dzc, dzc.data(), dzc.size() * sizeof(float4), cudaMemcpyHostToDevice, cs);
    cudaError_t e2 = cudaMemcpyAsync(b.dfix, dfix.data(), dfix.size() * sizeof(float2), cudaMemcpyHostToDevice, cs);
    cudaError_t e3 = cudaMemcpyAsync(b.ddrift, ddrift.data(), ddrift.size() * sizeof(float2), cudaMemcpyHostToDevice, cs);
    cudaError_t e4 = cudaMemcpyAsync(b.rho, rho.data(), rho.size() * sizeof(float), cudaMemcpyHostToDevice, cs);
    cudaError_t e5 = cudaMemcpyAsync(b.sig, sig.data(), sig.size() * sizeof(float), cudaMemcpyHostToDevice, cs);
    for (cudaError_t e : {e1, e2, e3, e4, e5})
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "grad: table upload");
        }
    st = launch_adjoint(s, b, seed, k0, (uint32_t)M, cs);
    if (st == CVA_OK) st = sum_columns_fp64(b.part, (int)blocks, NPAR + 1, b.sum, cs);
    std::vector<double> h(NPAR + 1);
    if (st == CVA_OK) {
        cudaError_t e = cudaMemcpyAsync(h.data(), b.sum, h.size() * sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "grad: read-back");
    }
    if (st == CVA_OK) {
        *cva0_host = h[NPAR] / (double)M;
        if (grad_host && !forward_only)
            for (int i = 0; i < NPAR; ++i) grad_host[i] = h[i] / (double)M;
    }
    cleanup();
    return st;
}

cva_status cva_philox4x32_10(const uint32_t *ctr_dev, uint32_t *out_dev, uint64_t n, uint64_t seed,
                             void *stream)
{
    return philox_blocks(ctr_dev, out_dev, n, seed, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
