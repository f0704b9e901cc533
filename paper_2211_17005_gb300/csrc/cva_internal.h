// Internal declarations shared by the library's translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cva.h"

namespace cva {

constexpr int kMaxE = 16;
constexpr int kMaxC = 16;
constexpr int kMaxF = 2 * kMaxE - 1 + kMaxC;
constexpr int kMaxG = 10;        // reset dates per swap schedule (periods)
constexpr int kMaxPF = 6;        // portfolios simulated together
constexpr int kMaxW = 5120;     // NPF*C*E*G weights of each kind held in constant memory

// Per-thread error message of the C ABI.
void set_error(const std::string &msg);
cva_status fail(cva_status st, const std::string &msg);
cva_status cuda_fail(cudaError_t e, const char *what);

#define CVA_CUDA_TRY(expr)                                                   \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) return ::cva::cuda_fail(_e, #expr);           \
    } while (0)

// Scalars and small tables of a simulation, uploaded to __constant__ memory
// before each launch of the outer-path kernel.
struct SimConsts {
    int E, C, CS, F, G, NPF, n, S, ppp;
    double ds_d;                           // sub-step length in FP64 (discount integral)
    float ds, sqds;
    float L[kMaxF * (kMaxF + 1) / 2];      // packed lower Cholesky factor, row-major
    float hw_a_ds[kMaxE];                  // a_e * ds
    float hw_sig_sqds[kMaxE];              // sigma^r_e * sqrt(ds)
    float fx_drift_ds[kMaxE];              // -sigma^chi_e^2 / 2 * ds
    float fx_sig_sqds[kMaxE];              // sigma^chi_e * sqrt(ds)
    float r0[kMaxE], lchi0[kMaxE];         // initial state
    float fix0_m1[kMaxE];                  // 1/ZC_0(delta) - 1 (first fixing)
    float cir_kds[kMaxC], cir_ktds[kMaxC], cir_nu_sqds[kMaxC];
    float gamma0[kMaxC], lgd[kMaxC];
    int gpos[kMaxC];                       // state factor of gamma^c (CIR), -1 for a constant intensity
};

// Date-bucketed portfolio weights, [pf][c][e][g] with compile-time strides
// (C, E, G of the kernel instantiation):
//   wA[..][h]  = sum over live swaps of (c, e) with n_periods >= h+1 of omega*N
//                (floating notional of period h, h = 0..G-1)
//   wK[..][g-1] = delta * sum over swaps of (c, e) with n_periods >= g of omega*N*Sigma
//                (fixed coupon paid at reset g, g = 1..G)
struct SimWeights {
    float wA[kMaxW];
    float wK[kMaxW];
};

struct Sim {
    // shape
    int E, C, CS, F, G, NPF, n, S, ppp, Ginst;
    uint64_t M;
    uint32_t N;
    uint32_t flags;
    bool generic = false;          // the run-time-shape kernels (outer_generic.cu)
    double horizon, delta;
    // host tables
    SimConsts consts;
    SimWeights weights;
    std::vector<double> recovery;
    // device tables
    float4 *d_zc = nullptr;        // [n+1][E][Ginst]  (lnA, B, dlnA, dB) of ZC_{t_j}((g+1) delta)
    float2 *d_fix = nullptr;       // [n_periods+1][E] (lnA, B) of ZC_{p delta}((p+1) delta)
    int *d_date_p = nullptr;       // [n+1] period index of t_j
    float *d_drift = nullptr;      // [n*S][E] (theta_e(t_q) - quanto_e) * ds
    // device outputs / scratch
    float *d_features = nullptr;   // [n+1][F][M]
    float *d_disc = nullptr;       // [n+1][M]
    float *d_thr = nullptr;        // [n+1][C][M]
    float *d_expo = nullptr;       // [NPF][n+1][C][M]
    float *d_mtm = nullptr;        // [NPF][n+1][C][M] (optional)
    float *d_targets = nullptr;    // [NPF][n][M]
    uint8_t *d_idx = nullptr;      // [M][N][C] (optional)
    void *d_cnt = nullptr;         // [n+1][C][M] default counts per step: uint16 (N <= 65535) or uint32
    // device image of consts + weights (constant uploads are device-to-device, so
    // they can be captured in a CUDA graph)
    unsigned char *d_const_img = nullptr;
    // tile shapes, set by cva_autotune
    int tune_sim_block = 128, tune_price_block = 256, tune_inner_P = 0, tune_lsq_chunks = 2432;
    int tune_price_pf = 1;         // portfolios per pricing block (1, 2 or 3, dividing n_pf; 0: all, from shared memory)
    // scratch of the portfolio-grouped regression, owned by the simulation
    double *d_lsq = nullptr;
    size_t lsq_cap = 0;
    // scratch of the regression on (default indicators, state), owned by the simulation
    float *d_alive_stats = nullptr;   // [n][2C + C(C-1)/2][M] per-path sums over the inner draws
    size_t alive_stats_cap = 0;
    double *d_alive = nullptr;        // Gram partials, coefficients, status
    size_t alive_cap = 0;
    // profiling events: before the simulation kernel, after it, after the pricing
    // kernel, after the inner-default kernel
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // twin copy being simulated (Sec. ss:twin): outer normals of the steps after
    // branch_date and all inner clocks draw with the copy id as the third counter
    // word; 0 (and no branch date) for the simulation itself
    int branch_date = 1 << 30;
    uint32_t branch = 0;
};

// Device buffers of the adjoint sweep (adjoint.cuh).
struct AdjBuffers {
    int K, nseg, forward_only;
    float4 *dzc = nullptr;      // [n+1][E][G] d/df, d/dsigma of (lnA, dlnA)
    float2 *dfix = nullptr;     // [periods+1][E] d/df, d/dsigma of lnA(p delta, (p+1) delta)
    float2 *ddrift = nullptr;   // [n*S][E] d drift/df, d drift/dsigma^r
    float *rho = nullptr;       // [E]
    float *sig = nullptr;       // [2E + 3C]
    float *ckpt = nullptr;      // [nseg][2E+3C][M]
    double *ckpt_I0 = nullptr;  // [nseg][M]
    float *fixr = nullptr;      // [periods+1][E][M]
    double *part = nullptr;     // [blocks][npar+1]
    double *sum = nullptr;      // [npar+1]
};

// One compiled shape of the outer-path kernel (outer_*.cu).
struct OuterInst {
    int E, C, CS, G, NPF;
    cva_status (*launch)(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st);
    void (*forget)(const Sim *s);
    cva_status (*adjoint)(Sim &s, const AdjBuffers &b, uint64_t seed, uint64_t k0, uint32_t M, cudaStream_t st);
};

// Kernel launchers (sim.cu).
cva_status launch_outer(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st);
cva_status launch_inner(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st);
void forget_const_owner(const Sim *s);
bool outer_supported(int E, int C, int CS, int G, int NPF, int *Ginst);
cva_status launch_adjoint(Sim &s, const AdjBuffers &b, uint64_t seed, uint64_t k0, uint32_t M, cudaStream_t st);
cva_status sum_columns_fp64(const double *part, int rows, int cols, double *out, cudaStream_t st);
// Block sums of the Prop. 1 statistics (sim.cu): part [blocks][n][3].
cva_status launch_oversim(const Sim &s, int pf, const float *pred, uint64_t seed, double *part, unsigned blocks,
                          cudaStream_t st);

// One grouped least-squares job: group g reads features feat0 + g*feat_stride ([F][M])
// and target t of it at targ0 + g*targ_stride + t*targ_tstride (nt targets share
// the normal matrix); predictions go to pred0 + g*pred_stride + t*pred_tstride.
struct LsqJob {
    const float *feat0 = nullptr;
    size_t feat_stride = 0;
    const float *targ0 = nullptr;
    size_t targ_stride = 0, targ_tstride = 0;
    float *pred0 = nullptr;
    size_t pred_stride = 0, pred_tstride = 0;
    int F = 0, basis = 0, groups = 1, nt = 1, chunk_target = 0;
    uint64_t M = 0;
};
cva_status lsq_launch(const LsqJob &j, double *scratch, size_t scratch_cap, double *coef_host, cudaStream_t st);
size_t lsq_scratch_need(const LsqJob &j);

// Regression (lsq.cu): least squares for `groups` dates at once; group g reads
// features feat0 + g*feat_stride ([F][M]) and targets targ0 + g*targ_stride.
cva_status lsq_grouped_strided(const float *feat0, size_t feat_stride, const float *targ0,
                               size_t targ_stride, float *pred0, size_t pred_stride, int F,
                               uint64_t M, int basis, int groups, double *coef_host, cudaStream_t st);

// The same regression for `groups` dates, scratch in a static device array (lsq.cu).
cva_status lsq_batched_static(const float *targ0, const float *feat0, int groups, int F, uint64_t M,
                              int basis, float *pred0, double *coef_host, cudaStream_t st);

// Neural regression (mlp.cu). mlp_fit_dates enqueues Algorithm 2 over n_dates
// consecutive dates of date-major arrays (Algorithm 1 when n_dates = 1) on `st`;
// mlp_begin clears the device status before it and mlp_finish synchronises `st`
// and reports a bounded wait that gave up.
int mlp_num_params(int U);
// Launch shape of the trainer (cva_mlp_plan); mlp_wide_plan is the width-128 one.
cva_status mlp_plan(uint64_t M, int U, int n_batches, int32_t out[4]);
cva_status mlp_wide_plan(int tiles_per_batch, int32_t out[4]);
void mlp_wide_set_grid_polls(uint32_t polls);
cva_status mlp_begin(cudaStream_t st);
cva_status mlp_finish(cudaStream_t st);
// Kernel timing of the train launches: mlp_kernel_timing returns and clears the
// totals and switches timing on or off; mlp_timing_pair hands out the event pair
// to record around one train launch (false when timing is off); mlp_finish adds
// the durations of the pairs recorded since mlp_begin.
void mlp_kernel_timing(bool on, double *ms, uint64_t *launches);
bool mlp_timing_pair(int dev, cudaEvent_t *a, cudaEvent_t *b);
cva_status mlp_fit_dates(const float *feat0, size_t feat_stride, const float *targ0, size_t targ_stride, int n_dates,
                         int F, uint64_t M, int U, int n_batches, int epochs, float lr, int max_steps,
                         float *params_dev, float *pred0, float *grad_out_dev, float *loss_out_dev, cudaStream_t st);
// The same at hidden width 128 on a cooperative grid (mlp_wide.cu); count and err
// are the device counters and status word that mlp_begin cleared.
cva_status mlp_wide_fit_dates(const float *feat0, size_t feat_stride, const float *targ0, size_t targ_stride,
                              int n_dates, int F, uint64_t M, int n_batches, int epochs, float lr, int max_steps,
                              float *params_dev, float *pred0, float *grad_out_dev, float *loss_out_dev,
                              unsigned *count, int *err, cudaStream_t st);

// Least squares on (default indicators, state) over the M N hierarchical sample
// of portfolio pf at dates 1..n-1 (alive.cu).
cva_status alive_regress(Sim &s, int pf, float *pred_dev, double *coef_host, int *dropped_host, cudaStream_t st);

// CVA_0 reduction (reduce.cu).
cva_status philox_blocks(const uint32_t *ctr, uint32_t *out, uint64_t n, uint64_t seed, cudaStream_t st);
cva_status mean_fp64(const float *x, uint64_t M, double *out2, cudaStream_t st);
cva_status sums_fp64(const float *x, uint64_t M, double *sum2_host, cudaStream_t st);
void mean_se_from_sums(double M, double s1, double s2, double *out2);
// Least squares split over path ranges (lsq.cu): the augmented normal matrix of one
// range with a given centring, its solution on the host, the predictions of a range.
cva_status lsq_normal_partial(const float *targ, const float *feat, int F, uint64_t M, int basis, const float *centre,
                              double *gram_host, cudaStream_t st);
cva_status lsq_solve_normal_host(const double *gram, int F, int basis, const double *centre, double *coef_centred,
                                 double *coef_raw, int *dropped);
cva_status lsq_predict_centred(const float *feat, int F, uint64_t M, int basis, const float *centre,
                               const double *coef_centred_host, float *pred, cudaStream_t st);
cva_status twin_l2_fp64(const float *phi, const float *xi1, const float *xi2, uint64_t M, double *out2,
                        cudaStream_t st);
cva_status accumulate_mean(float *acc, const float *x, uint64_t M, int first, int last, int copies, cudaStream_t st);
cva_status relative_rmse_fp64(const float *phi, const float *ref, uint64_t M, double *out2, cudaStream_t st);

}  // namespace cva
