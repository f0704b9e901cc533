/*
 * cva.h -- C ABI of the GB300 (sm_103a) hierarchical pathwise-CVA library.
 *
 * The library implements the data-parallel hot path of Abbas-Turki, Crepey and
 * Saadeddine, "Pathwise CVA Regressions With Oversimulated Defaults"
 * (arXiv 2211.17005):
 *
 *   simulate  M outer paths Y^k of the market/credit factors (App. B: Hull-White
 *             short rates eq. (e:sde1), lognormal FX, CIR intensities eq. (e:sde2)),
 *             price the swap portfolio at every pricing date (App. B swap formula),
 *             draw N inner default scenarios X^{k,l} per outer path (Sec. 3.2,
 *             default clocks of eq. (e:tau)) and form the averaged pathwise CVA
 *             target of eq. (eq:CVA_portfolio);
 *   regress   the target on the state at each date by least squares (eq. (e:forw));
 *   cva0      CVA_0 as the mean of the date-0 targets.
 *
 * Conventions (every entry point):
 *  - all functions return a cva_status; nothing throws across the ABI; on error
 *    cva_last_error() returns a message for the calling thread;
 *  - "dev" pointers are CUDA device pointers on the current device, "host"
 *    pointers are host memory; all work is enqueued on the caller's stream
 *    (a cudaStream_t passed as void*, NULL = legacy default stream) and is
 *    asynchronous unless the comment says the call synchronises;
 *  - arrays are row-major, the outer-path index k is always the fastest
 *    (innermost) index of device arrays so that warps access consecutive paths;
 *  - objects created by the library are owned by the library and released by
 *    the matching _destroy call; pointers returned by cva_sim_view are borrowed
 *    and valid until cva_sim_destroy.
 */
#ifndef CVA_H
#define CVA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CVA_API __attribute__((visibility("default")))
#else
#define CVA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CVA_OK = 0,
    CVA_EINVAL = 1,     /* bad argument (shape, range, non-SPD correlation, ...) */
    CVA_ENOMEM = 2,     /* device or host allocation failed                      */
    CVA_ECUDA = 3,      /* a CUDA runtime call failed                            */
    CVA_ETIMEOUT = 4,   /* a bounded device-side wait gave up                    */
    CVA_ENOTSUP = 5,    /* shape not supported by the compiled kernels           */
    CVA_ENUMERIC = 6    /* numerical failure (e.g. singular normal equations)    */
} cva_status;

/* Market and credit model (Sec. 4.1 and App. B). E economies, economy 0 is the
 * reference currency; C counterparties. The stochastic factors, in this order,
 * are r^0..r^{E-1}, log chi^1..log chi^{E-1}, then gamma^c of every
 * counterparty with cir_nu[c] > 0; F is their count and corr is their F x F
 * correlation matrix (row-major, symmetric positive definite).
 * Short rates are Hull-White fitted to a flat curve curve[e] (Vasicek is the
 * constant-theta special case of eq. (e:sde1)); r^e for e >= 1 carries the
 * quanto drift -rho_e fx_vol[e] hw_sigma[e] under the reference measure, rho_e
 * being the correlation of r^e and log chi^e. cir_nu[c] = 0 makes gamma^c the
 * constant gamma0[c]. All arrays are host memory, copied at creation. */
typedef struct {
    int E, C;
    const double *hw_a, *hw_sigma, *curve;       /* [E] */
    const double *fx_vol, *fx0;                  /* [E], entry 0 ignored */
    const double *cir_kappa, *cir_theta, *cir_nu, *gamma0, *recovery; /* [C] */
    const double *corr;                          /* [F*F] */
} cva_model_desc;

/* Spot-starting interest-rate swaps with regular resets every delta years
 * (App. B): the bank pays delta*Sigma and receives the floating coupon at each
 * reset date; omega = +1 (payer) or -1 (receiver) from the bank's point of
 * view. fixed_rate gives Sigma per swap; when it is NULL every swap is at par
 * at t = 0 (P^sw_0 = 0, computed by the library from the model's curve).
 * delta must be a whole number of pricing steps. Host memory. */
typedef struct {
    int n_swaps;
    const int32_t *ccy, *cpty, *omega, *n_periods;   /* [n_swaps] */
    const double *notional;                          /* [n_swaps] */
    double delta;
    const double *fixed_rate;                        /* [n_swaps] or NULL (par) */
} cva_portfolio_desc;

/* Pricing grid t_j = j*horizon/n_steps, j = 0..n_steps, with `substeps`
 * Euler-Maruyama sub-steps per pricing step (Remark rem:finecoarse). */
typedef struct {
    double horizon;
    int n_steps, substeps;
} cva_grid;

typedef struct cva_sim cva_sim;   /* opaque: tables and device buffers of one run */

/* flags of cva_sim_create */
#define CVA_KEEP_DEFAULTS  1u   /* also keep default step indices (validation)     */
#define CVA_KEEP_EXPOSURES 2u   /* also keep the MtM per counterparty and date     */
#define CVA_PROFILE        4u   /* record CUDA events around each kernel launch    */
#define CVA_GENERIC_KERNELS 8u  /* run-time-shape kernels even where a compiled
                                   instantiation exists (validation)               */

/* Prepare a simulation of M outer paths x N inner default draws for n_pf
 * portfolios sharing one model and grid. Validates every input (returns
 * CVA_EINVAL on a bad one), builds the host tables (correlation Cholesky factor,
 * Hull-White drift and bond tables, date-bucketed portfolio weights, par rates)
 * and allocates the device buffers on the current device (CVA_ENOMEM if that
 * fails). Limits: 1 <= E <= 16, 1 <= C <= 16, 1 <= n_pf <= 6, swaps of at most
 * 10 periods, n_steps <= 254, N <= 2^24, M <= 2^31, and n_pf C E (longest
 * schedule in periods) <= 5120 (the date-bucketed weights live in constant
 * memory; CVA_ENOTSUP beyond). Compiled fast paths exist for (E, C, CIR
 * counterparties first, n_pf) = (1, 2 constant, 1), (10, 8 CIR, 1) and (10, 8 CIR,
 * 6); every other shape within the limits, including constant and CIR intensities
 * in any order, runs on the run-time-shape kernels (flag CVA_GENERIC_KERNELS
 * forces them for a compiled shape; the results are the same bits). Synchronous. */
CVA_API cva_status cva_sim_create(const cva_model_desc *model, const cva_portfolio_desc *pfs,
                          int n_pf, const cva_grid *grid, uint64_t M, uint32_t N,
                          uint32_t flags, cva_sim **out);

/* Run the hierarchical simulation for global outer paths [k0, k0 + M) with the
 * Philox4x32-10 key `seed` (counters keyed by global path, step and inner
 * index, so a path range gives the same paths as a full run). Enqueues the
 * path-simulation kernel (factors, integrals, thresholds, features), the
 * pricing kernel (MtM and exposures per path and date) and the inner-default
 * kernel (default steps, averaged targets) on `stream`. */
CVA_API cva_status cva_simulate(cva_sim *sim, uint64_t seed, uint64_t k0, void *stream);

/* Twin Monte Carlo validation (Sec. ss:twin, eqs. (e:val1)-(e:val2)): run the
 * same simulation as twin copy `copy` (>= 1) branching at pricing date `date`
 * (0 <= date <= n). Outer paths follow the simulation itself up to t_date (the
 * same Philox counters, so the states up to t_date are bit-identical) and draw
 * their Euler increments after t_date, and all their inner default clocks, with
 * `copy` as the third counter word. Two copies b != b' are therefore
 * independent given the state of every path at t_date, and the targets of date
 * `date` they leave in the simulation's buffers (cva_sim_view) are the
 * conditionally independent copies xi^(1), xi^(2) of eq. (e:val1). Arguments and
 * asynchrony as cva_simulate; CVA_EINVAL for a date outside [0, n] or copy 0. */
CVA_API cva_status cva_simulate_twin(cva_sim *sim, uint64_t seed, uint64_t k0, int date, uint32_t copy,
                                     void *stream);

/* Nested Monte Carlo reference of the conditional CVA at a date (the benchmark of
 * Sec. 4.3, with copies inner paths per outer path): out_dev (device float [M])
 * receives, for every outer path, the mean over twin copies b = 1..copies
 * (cva_simulate_twin, branched at `date`) of the averaged target of portfolio pf
 * at that date, an estimate of E[xi_bar_date | state at t_date] whose error falls
 * as 1/sqrt(copies). Runs `copies` full simulations on `stream` and leaves the
 * last copy in the simulation's buffers. CVA_EINVAL for date outside [0, n),
 * copies outside [1, 2^24) or a bad portfolio index. */
CVA_API cva_status cva_nested_reference(cva_sim *sim, uint64_t seed, uint64_t k0, int pf, int date, int copies,
                                        float *out_dev, void *stream);

/* The relative error measure of the paper's nested Monte Carlo comparison:
 * sqrt(mean over paths with ref != 0 of ((phi - ref) / ref)^2). phi_dev, ref_dev:
 * device float [M]. out2 (host double [2]) receives (the relative RMSE, the number
 * of paths with ref != 0). FP64 sums in a fixed order; synchronises `stream`. */
CVA_API cva_status cva_relative_rmse(const float *phi_dev, const float *ref_dev, uint64_t M, double *out2,
                                     void *stream);

/* Sampling statistics of Prop. 1 (Sec. ss:choice1) for choosing the
 * oversimulation factor N. With the pointwise loss g = (xi_i - phi_i(Y_i))^2 of a
 * single inner draw (X) on an outer path (Y), and phi_i the regression of date i
 * (pred_dev: device float [n][M], e.g. the predictions of cva_regress_all or
 * cva_mlp_regress_all), qr_host (host double [n][2]) receives per date
 *   Q_i = E[Var(g | Y)] = E[g^2] - E[g(X^1) g(X^2)],
 *   R_i = Var(E[g | Y]) = E[g(X^1) g(X^2)] - E[g]^2,
 * estimated over the M outer paths from their first two inner draws (the same
 * default clocks as the simulation's draws 0 and 1, seed = the key of the last
 * cva_simulate; the simulation must have N >= 2). Dates 0 and n get zeros. The
 * optimal factor under the budget M (N + kappa) is N_i = sqrt(Q_i kappa / R_i)
 * (eq. (e:optom)). FP64 sums in a fixed order; synchronises `stream`. */
CVA_API cva_status cva_oversim_stats(const cva_sim *sim, int pf, const float *pred_dev, uint64_t seed,
                                     double *qr_host, void *stream);

/* Choice of the oversimulation factor from the statistics of cva_oversim_stats
 * (Prop. 1 and Heuristic 1, Sec. ss:choice1). qr_host: host double [n][2], the
 * (Q_i, R_i) of n dates. Ni_host (host double [n]) receives, per date, the N that
 * minimises the variance (R_i + Q_i / N)(N + kappa) / budget of the empirical loss at
 * a fixed budget of M (N + kappa) inner-draw units, N_i = sqrt(Q_i kappa / R_i)
 * (eq. (e:optom)), or NaN where R_i <= 0 or Q_i < 0 (no interior optimum); N_out
 * receives Heuristic 1's N, the mean of the defined N_i; M_out (nullable) receives
 * budget / (N + kappa), the outer paths the budget then pays for (NaN when budget
 * <= 0). kappa is the cost of an outer path in inner draws (cva_inner_cost_ratio).
 * CVA_ENUMERIC if no date defines N_i. Host-only, no device work. */
CVA_API cva_status cva_oversim_choice(const double *qr_host, int n, double kappa, double budget,
                                      double *Ni_host, double *N_out, double *M_out);

/* The cost kappa of one outer path in units of one inner draw, eq. (l:ratio): from
 * the times t1, t2 (any unit, > 0) of two simulations of the same M outer paths with
 * N1 != N2 inner draws, assuming time = c M (kappa + N). kappa_out (host) receives
 * (t1 N2 - t2 N1) / (t2 - t1). CVA_EINVAL for N1 == N2, equal or non-positive
 * times. Host-only, no device work. */
CVA_API cva_status cva_inner_cost_ratio(double t1, uint32_t N1, double t2, uint32_t N2, double *kappa_out);

/* The twin estimator of eq. (e:val1): the mean over M paths of
 * phi^2 - (xi1 + xi2) phi + xi1 xi2, an unbiased estimate of the L2 error
 * E[(phi - E[xi | state at the branch date])^2] of any estimate phi computed from
 * that state, with its Monte Carlo standard error. phi_dev, xi1_dev, xi2_dev:
 * device float [M]. out2 (host double [2]) receives (estimate, standard error).
 * FP64 sums in a fixed two-stage order. Synchronises `stream`. */
CVA_API cva_status cva_twin_l2(const float *phi_dev, const float *xi1_dev, const float *xi2_dev, uint64_t M,
                               double *out2, void *stream);

/* What cva_sim_view can return; shapes use n = n_steps, F factors, C
 * counterparties, P = n_pf portfolios:
 *   CVA_VIEW_FEATURES  float [n+1][F][M]   state Y_j (r^e, log chi^e, gamma^c)
 *   CVA_VIEW_TARGETS   float [P][n][M]     averaged target xi_bar_i, i = 0..n-1
 *   CVA_VIEW_DISCOUNT  float [n+1][M]      int_0^{t_j} r^0 (beta_j = exp(-value))
 *   CVA_VIEW_THRESHOLD float [n+1][C][M]   1 - exp(-Lambda_c(t_j))
 *   CVA_VIEW_EXPOSURE  float [P][n+1][C][M] (1-R_c) beta_j MtM_c(t_j)^+
 *   CVA_VIEW_MTM       float [P][n+1][C][M] MtM_c(t_j), reference ccy  (KEEP_EXPOSURES)
 *   CVA_VIEW_DEFAULTS  uint8 [M][N][C]     default step in 1..n, n+1 = none (KEEP_DEFAULTS)
 * The pointer is borrowed (owned by sim). Returns CVA_EINVAL if the view was
 * not requested at creation. */
#define CVA_VIEW_FEATURES  0
#define CVA_VIEW_TARGETS   1
#define CVA_VIEW_DISCOUNT  2
#define CVA_VIEW_THRESHOLD 3
#define CVA_VIEW_EXPOSURE  4
#define CVA_VIEW_MTM       5
#define CVA_VIEW_DEFAULTS  6
CVA_API cva_status cva_sim_view(const cva_sim *sim, int what, void **dev_ptr, size_t *bytes);

/* Device durations (milliseconds, CUDA events on the launching stream) of the
 * last cva_simulate of a sim created with CVA_PROFILE: out_ms[0] = path
 * simulation kernel, out_ms[1] = pricing kernel (MtM and exposures),
 * out_ms[2] = inner-default kernel. Waits for those events. */
CVA_API cva_status cva_sim_kernel_ms(const cva_sim *sim, float out_ms[3]);

/* Shape of a simulation: out[0..5] = M, N, n_steps, F, C, n_pf. */
CVA_API cva_status cva_sim_shape(const cva_sim *sim, int64_t out[6]);

CVA_API void cva_sim_destroy(cva_sim *sim);

/* CVA_0 of eq. (eq:CVA_portfolio) at i = 0: the mean over the M outer paths of
 * the date-0 averaged targets xi0_dev[M] (float, device), accumulated in FP64 in
 * a fixed order (bit-reproducible). Writes host out2[0] = CVA_0 and
 * out2[1] = its Monte Carlo standard error. Synchronises `stream`. */
CVA_API cva_status cva_cva0(const float *xi0_dev, uint64_t M, double *out2_host, void *stream);

/* Least-squares regression of eq. (e:forw) at one date:
 *   w = argmin_w sum_k (targets[k] - w^T phi(Y[:, k]))^2
 * features_dev: float [F][M] (state at the date, path index fastest);
 * targets_dev:  float [M];
 * basis: CVA_BASIS_LINEAR  phi = [1, Y_1, ..., Y_F]        (m = F + 1)
 *        CVA_BASIS_POLY2   phi = [1, y, y^2] of factor 0     (m = 3)
 * The normal equations are accumulated in FP64 on the centred, scaled basis and
 * solved by Cholesky in FP64. pred_dev (float [M], nullable) receives
 * phi(Y_k)^T w; coef_host (double [m], nullable) receives w in the raw basis
 * (w_0 + w_1 y + ... ). Synchronises `stream` when coef_host is not NULL.
 * CVA_ENUMERIC if the normal matrix is singular. */
#define CVA_BASIS_LINEAR 0
#define CVA_BASIS_POLY2  1
CVA_API cva_status cva_regress(const float *targets_dev, const float *features_dev, int F,
                       uint64_t M, int basis, float *pred_dev, double *coef_host,
                       void *stream);

/* Least squares of eq. (e:forw) over outer paths split into ranges, one per process
 * (and GPU), with one exchange: every range computes its part of the normal
 * equations, the parts are summed (in a fixed order, on the host or by a
 * collective), solved once, and every range predicts its own paths. Outer paths
 * are independent and the generator's counters are keyed by the global path
 * index (cva_simulate's k0), so a split run simulates exactly the paths of one
 * large run, and the summed normal matrix is the whole sample's.
 *
 * cva_regress_partial: the augmented normal matrix [phi, xi]^T [phi, xi] (host
 * double [(m+1) x (m+1)], row-major, symmetric; m = F+1 linear, 3 poly2) of the
 * basis centred on centre_dev (device float [F], poly2 [1]: a state every range
 * agrees on, e.g. path 0's), accumulated as cva_regress does (FP32 products in
 * runs, FP64 sums in a fixed order). Synchronises `stream`.
 * cva_regress_solve: host only. The summed matrix solved as cva_regress does
 * (Jacobi scaling, Cholesky in FP64, a vanishing pivot's column dropped with
 * coefficient 0): coef_centred_host (double [m], nullable) in the centred basis,
 * coef_raw_host (double [m], nullable) in the raw basis for centre_host (host
 * double copy of the centre), dropped_host (nullable) the number of dropped columns.
 * cva_regress_predict: pred_dev (device float [M]) receives phi(Y_k) . w for the
 * centred coefficients of cva_regress_solve. Synchronises `stream`. */
CVA_API cva_status cva_regress_partial(const float *targets_dev, const float *features_dev, int F, uint64_t M,
                                       int basis, const float *centre_dev, double *gram_host, void *stream);
CVA_API cva_status cva_regress_solve(const double *gram_host, int F, int basis, const double *centre_host,
                                     double *coef_centred_host, double *coef_raw_host, int *dropped_host);
CVA_API cva_status cva_regress_predict(const float *features_dev, int F, uint64_t M, int basis,
                                       const float *centre_dev, const double *coef_centred_host, float *pred_dev,
                                       void *stream);

/* CVA_0 over outer paths split into ranges (eq. (eq:CVA_portfolio) at i = 0):
 * cva_cva0_partials writes out3_host = (M, sum of xi0, sum of xi0^2) of one range,
 * FP64 in a fixed order (synchronises `stream`); cva_cva0_combine (host only) adds
 * n_parts such triples (host double [n_parts][3]) in their order and writes
 * out2_host = (CVA_0, its Monte Carlo standard error), by the formula of cva_cva0. */
CVA_API cva_status cva_cva0_partials(const float *xi0_dev, uint64_t M, double *out3_host, void *stream);
CVA_API cva_status cva_cva0_combine(const double *parts_host, int n_parts, double *out2_host);

/* The same regression for every date i = 1..n-1 of a simulation and portfolio
 * pf, all dates in one grouped launch: features of date i, targets of date i.
 * pred_dev: float [n][M] (row 0 left untouched), nullable; coef_host: double
 * [n][m] (row 0 left untouched), nullable. Synchronises when coef_host != NULL. */
CVA_API cva_status cva_regress_all(const cva_sim *sim, int pf, int basis, float *pred_dev,
                           double *coef_host, void *stream);

/* Least squares of eq. (e:forw) for every date 1..n-1 and every portfolio of a
 * simulation in one grouped launch: the portfolios share each date's features,
 * so every date's normal matrix is accumulated once (FP64) with one target column
 * per portfolio and solved once (Cholesky, FP64) for all of them. pred_dev: float
 * [n_pf][n][M] (date 0 untouched), nullable; coef_host: double [n_pf][n][m]
 * (date 0 untouched), nullable. The scratch belongs to the simulation: the first
 * call allocates it, so make one call before capturing this one in a CUDA graph.
 * Without coef_host the call does not synchronise and can be captured together
 * with cva_simulate. */
CVA_API cva_status cva_regress_portfolios(cva_sim *sim, int basis, float *pred_dev, double *coef_host,
                                          void *stream);

/* Least squares on the hierarchically simulated sample (Sec. "Learning on
 * Hierarchically Simulated Paths"), portfolio pf, every date i = 1..n-1: one row
 * per (outer path k, inner draw l), the features (X_i^{k,l}, Y_i^k) with X_i the
 * default indicators 1{tau_c <= t_i} of the C counterparties and Y_i the state
 * (Sec. 4.1), the per-draw target of eq. (eq:CVA_portfolio)
 *   xi_i^{k,l} = beta_i^{-1} sum_c (1-R_c) beta_j MtM_c(t_j)^+ 1{i < j <= n}, j = default step of c in draw l,
 * and the basis [1, Y_i - Y_i^0, X_i] (Y_i^0: path 0's state):
 *   w_i = argmin_w sum_{k,l} (xi_i^{k,l} - w^T [1, Y_i^k - Y_i^0, X_i^{k,l}])^2.
 * The M N rows are not formed: per path, exact integer counts over the N draws
 * (defaults of c, joint defaults of c and d) and the sums of the target over the
 * draws where c has defaulted give the normal equations (FP64 accumulation), solved
 * by a Jacobi-scaled Cholesky factorisation in FP64; a column whose pivot vanishes
 * (no default of c by t_i in the whole sample) is dropped, with coefficient 0.
 * Needs a simulation created with CVA_KEEP_DEFAULTS after cva_simulate; C <= 8 (one
 * warp lane per counterparty pair), 1 + F + C <= 40 and N (5C + 6) bytes of draw tables must fit 160 KB of shared
 * memory (N <= 3400 at C = 8; else CVA_ENOTSUP).
 * pred_dev: float [n][M] (nullable; date 0 untouched) receives the fit at X_i = 0
 * (every counterparty alive). coef_host: double [n][1+F+C] (nullable; date 0
 * untouched) receives w_i in the raw basis [1, Y_i, X_i]. dropped_host: int [n]
 * (nullable) receives the number of dropped columns per date (0 at date 0). The
 * scratch (n C M floats of per-path default counts, the pair and loss sums of each
 * block of 8 paths, and the Gram partials) belongs to the simulation: the first call allocates it, so make one call before capturing this
 * one in a CUDA graph. Synchronises `stream` only when coef_host or dropped_host is
 * given. */
CVA_API cva_status cva_regress_alive(cva_sim *sim, int pf, float *pred_dev, double *coef_host, int *dropped_host,
                                     void *stream);

/* Tile shapes of a simulation chosen by measurement: threads per block of the
 * path-simulation and pricing kernels, outer paths per block of the
 * inner-default kernel, and the number of blocks of the grouped regression
 * (basis `basis`). Each candidate runs on the simulation's own shapes (CUDA-event
 * timings, best of two after a warm-up); the choice is kept in the simulation and
 * cached per (device, shape) for the life of the process. report (nullable)
 * receives the choice as JSON. Runs the kernels; synchronises `stream`. */
CVA_API cva_status cva_autotune(cva_sim *sim, uint64_t seed, int basis, char *report, size_t report_len,
                                void *stream);

/* Sets the tile shapes of a simulation directly (e.g. a choice cva_autotune made
 * in an earlier process): sim_block in {64, 128}, price_block in {128, 256},
 * inner_paths_per_block in {0 (automatic), 2, 4, 8}, lsq_chunk_target in
 * [152, 2^20], and the pricing form portfolios_per_price_block: 1, 2 or 3 dividing
 * the simulation's number of portfolios (a block prices that many portfolios,
 * weights in constant memory; price_block threads), 0 (every thread prices every
 * portfolio for 2 paths with price_block = 128 or 1 path with 256, weights staged in
 * shared memory) or 4 (every portfolio of 128-path tiles on the tensor cores: the
 * MtM as a TF32 product with each operand split into head and tail, FP32
 * accumulation). None of the shapes and forms 0-3 changes any result bit; form 4
 * rounds the MtM differently (within the oracle tolerances). Returns CVA_EINVAL
 * (nothing changed) on a value outside these sets. No GPU work. */
CVA_API cva_status cva_set_tiles(cva_sim *sim, int sim_block, int price_block, int inner_paths_per_block,
                                 int lsq_chunk_target, int portfolios_per_price_block);

/* Sensitivities of CVA_0 by a hand-written adjoint (reverse-mode) sweep. The
 * sampled default indicators have zero pathwise derivative, so the function
 * differentiated is the smooth CVA_0 that the oversimulated average estimates,
 * the exact discrete form of the intensity formula eq. (eq:CVAint) at i = 0:
 *   CVA_0 = (1/M) sum_k sum_c sum_{j=1..n} (1-R_c) beta_j MtM_c(t_j)^+ (e^{-Lambda_c(t_{j-1})} - e^{-Lambda_c(t_j)})
 * over global outer paths [k0, k0 + M) of the model, one portfolio and grid of
 * cva_sim_create (same Philox counters). grad_host (host double, cva_grad_num_params
 * entries) receives dCVA_0/d theta in this order: curve levels f_e (E), rate
 * volatilities sigma^r_e (E), FX volatilities sigma^chi_e for e = 1..E-1, CIR
 * kappa_c (C), theta_c (C), nu_c (C) (gamma_0 and the swaps' fixed rates held
 * fixed); cva0_host receives the smooth CVA_0. The forward sweep keeps the
 * state every ckpt_every pricing dates (<= 16; sub-steps <= 4); the reverse sweep
 * recomputes each segment from its checkpoint. forward_only = 1 computes only
 * the smooth CVA_0 (grad_host may be NULL). Per-path adjoints are reduced in
 * FP64. The fast-path shapes of cva_sim_create with one portfolio, (E, C) = (1, 2
 * constant) and (10, 8 CIR), have compiled adjoint kernels; every other shape within
 * the limits of cva_sim_create runs the run-time-shape adjoint (same arithmetic,
 * slower: its per-path arrays live in local memory). A constant intensity's kappa_c,
 * theta_c and nu_c receive 0. Allocates and frees its buffers; synchronises `stream`. */
CVA_API cva_status cva_grad_cva0(const cva_model_desc *model, const cva_portfolio_desc *pf,
                                 const cva_grid *grid, uint64_t M, uint64_t seed, uint64_t k0,
                                 int ckpt_every, int forward_only, double *grad_host,
                                 double *cva0_host, void *stream);

/* Par fixed rate of every swap of `pf` at t = 0 under `model` (App. B third
 * case, P^sw_0 = 0): the rates the library uses when fixed_rate is NULL. Host
 * output rates_host [pf->n_swaps]. Host-only, no device work. */
CVA_API cva_status cva_par_rates(const cva_model_desc *model, const cva_portfolio_desc *pf,
                                 double *rates_host);

/* Number of parameters of cva_grad_cva0: 3E - 1 + 3C (53 for 10 economies, 8 counterparties). */
CVA_API int cva_grad_num_params(int E, int C);

/* Neural regression of Sec. 2 (eq. (e:regrkappo)) at one date: the NN+ network of
 * eq. (e:nnp) with two hidden ReLU layers of width `hidden` (64 or 128) on
 * the F <= 32 standardised factors, trained by Algorithm 1 (BaseAlg): mini-batch
 * Adam (beta = 0.9, 0.999, eps = 1e-8, step size lr) over n_batches contiguous
 * path ranges for `epochs` epochs, no output ReLU for the first floor(epochs/2)
 * epochs, then a closed-form least-squares refit of the output layer (FP64
 * normal equations) and the output ReLU; after every epoch the full-sample loss
 * decides whether the parameters are the best so far. GEMMs run on tcgen05 tensor
 * cores (BF16 operands, FP32 accumulation); the rest in FP32.
 * params_dev (device float, cva_mlp_num_params(hidden) entries) holds the
 * initial parameters and receives the best ones; layout: W1 [hidden][32]
 * (columns >= F zero), b1 [hidden], W2 [hidden][hidden], b2 [hidden],
 * w3 [hidden], b3, mu. pred_dev (float [M], nullable) receives the best
 * network's predictions, loss_dev (float [epochs], nullable) the loss after each
 * epoch. M must be a multiple of 128 * n_batches; features_dev and targets_dev
 * must be 16-byte aligned (tiles arrive by TMA and bulk copies). Width 64 trains
 * on one thread-block cluster, width 128 on a cooperative grid of one CTA per SM.
 * Synchronises `stream`. CVA_ETIMEOUT if a bounded device-side wait gave up. */
CVA_API cva_status cva_mlp_fit(const float *targets_dev, const float *features_dev, int F, uint64_t M,
                               int hidden, int n_batches, int epochs, float lr, float *params_dev,
                               float *pred_dev, float *loss_dev, void *stream);

/* Number of parameters of the network of cva_mlp_fit. */
CVA_API int cva_mlp_num_params(int hidden);

/* Launch shape cva_mlp_fit uses for M paths in n_batches batches at width hidden
 * (Algorithm 1's batch of M / n_batches paths = tiles of 128 paths): out4_host
 * (host int32 [4]) receives the number of CTAs of the trainer, its thread-block
 * cluster size (0: a cooperative grid, width 128), the tiles per batch and the
 * rounds of tiles a CTA runs per Adam step. Width 64 trains on one cluster of
 * 4, 8 or 16 CTAs with two tile slots each; width 128 on a cooperative grid with
 * one CTA per SM at most. Queries the current device; no GPU work. CVA_EINVAL
 * (CVA_ENOTSUP for another width) on the arguments cva_mlp_fit would reject. */
CVA_API cva_status cva_mlp_plan(uint64_t M, int hidden, int n_batches, int32_t *out4_host);

/* Failure-detection hook of the width-128 trainer: a CTA waiting at one of the
 * trainer's two grid barriers of an Adam step (gradient partials written; parameter
 * slices updated) gives up after grid_polls polls of the barrier's arrival counter
 * (about 32 ns apart; the default is 2^22, over 0.1 s), sets the device status word
 * and leaves its remaining waits at once, so that every CTA ends its launch and the
 * call returns CVA_ETIMEOUT (no CTA outlives its tensor-core or copy operations:
 * their own bounded waits are not shortened). 0 makes every wait give up unless
 * the barrier is already complete; UINT32_MAX restores the default. Applies to the
 * launches enqueued after it, on every device; host-only, no device work. */
CVA_API cva_status cva_mlp_set_wait_limit(uint32_t grid_polls);

/* Kernel timing of the trainers (Algorithm 1's training epochs): while on, every
 * launch of the training kernel by cva_mlp_fit, cva_mlp_first_gradient and
 * cva_mlp_regress_all (one launch per epoch and date) is bracketed by a pair of
 * CUDA events on the stream it runs on, and the call adds the launch's duration to
 * a process-wide total once it has synchronised. This call stores the totals
 * accumulated since its previous call (milliseconds, launches) in ms_host and
 * launches_host (each nullable), clears them and switches timing on (on != 0) or
 * off. The events break nothing but the overlap of one launch's start with the
 * previous launch's end. Host-only, no device work. */
CVA_API cva_status cva_mlp_kernel_timing(int on, double *ms_host, uint64_t *launches_host);

/* Validation hook of cva_mlp_fit: one Adam step on the first batch; grad_dev
 * (float [cva_mlp_num_params]) receives that batch's gradient, params_dev the
 * updated parameters. */
CVA_API cva_status cva_mlp_first_gradient(const float *targets_dev, const float *features_dev, int F,
                                          uint64_t M, int hidden, int n_batches, float lr,
                                          float *params_dev, float *grad_dev, void *stream);

/* Algorithm 2 (backward learning) over a simulation: dates n-1 down to 1, each
 * fitted by cva_mlp_fit on the state and targets of portfolio pf at that date,
 * starting from the previous date's best parameters (params_dev holds the
 * initial parameters and receives date 1's). pred_dev: float [n][M] (row 0 and
 * row n untouched). Synchronises `stream`. */
CVA_API cva_status cva_mlp_regress_all(const cva_sim *sim, int pf, int hidden, int n_batches, int epochs,
                                       float lr, float *params_dev, float *pred_dev, void *stream);

/* The paper has no counterpart for this entry point; it serves callers that
 * cannot allocate device memory when they need a fit: a framework that owns the
 * whole device through its own pool, a process held to a fixed memory budget
 * checked at start-up, or a latency-critical loop that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * It fits `groups` independent least-squares problems exactly like cva_regress
 * (same bases, same FP64 normal equations and Cholesky solve), group g reading
 * targets_dev + g*M (float [M]) and features_dev + g*F*M (float [F][M]) and
 * writing pred_dev + g*M (float [M], nullable) and coef_host + g*m (double,
 * nullable; m = F+1 linear, 3 poly2).
 *
 * It allocates nothing: its scratch (Gram partials, coefficients, status) is a
 * static 1 MiB device array inside the library, present on every device that
 * loads the library until the process exits. That array bounds the batch: a
 * call with more groups than fit (207 for the linear basis with F = 27; 1024
 * at most, e.g. for F <= 10 or the poly2 basis) returns CVA_EINVAL with the
 * limit in cva_last_error().
 *
 * Set-up: the first call on a device (and again after the device's context was
 * destroyed and re-created, e.g. by cudaDeviceReset) looks up the array's device
 * address with cudaGetSymbolAddress and sets the shared-memory limit of the
 * kernels it launches; later calls reuse both. Make that first call before any
 * stream capture. coef_host needs a synchronisation of `stream`: while `stream`
 * is being captured the call returns CVA_EINVAL unless coef_host is NULL.
 *
 * Every call shares the array and leaves its contents behind; each call writes
 * what it reads, so nothing needs clearing, but calls whose kernels overlap on
 * the GPU (e.g. on two streams) race on the array and must be ordered by the
 * caller. Synchronises `stream` when coef_host is not NULL. Singular normal
 * equations are reported (CVA_ENUMERIC) only when coef_host is given; without
 * it the predictions of such a group are not checked. */
CVA_API cva_status cva_regress_batched_static(const float *targets_dev, const float *features_dev,
                                              int groups, int F, uint64_t M, int basis,
                                              float *pred_dev, double *coef_host, void *stream);

/* The counter-based generator the kernels draw from: Philox4x32-10 (Salmon,
 * Moraes, Dror, Shaw, SC'11) with key (seed low 32 bits, seed high 32 bits).
 * For i < n: out_dev[4i..4i+3] = Philox4x32-10(ctr_dev[4i..4i+3], key). Both
 * arrays are device memory (uint32). The simulation uses the counters
 * (path k, fine step q, 0, 1 << 24 | block) for its normals and
 * (path k, inner draw l, 0, 2 << 24 | block) for its default clocks. */
CVA_API cva_status cva_philox4x32_10(const uint32_t *ctr_dev, uint32_t *out_dev, uint64_t n,
                                     uint64_t seed, void *stream);

/* Measured throughput of the SMs' plain arithmetic pipes on the current device,
 * the ceilings of the kernels that neither HBM nor the tensor cores bound (the
 * path simulation and the pricing; the paper gives no such figure). Each probe
 * runs eight independent chains of one instruction per thread on 64 warps per SM
 * and is timed with CUDA events after a warm-up launch. out5_host (host double
 * [5]) receives lane-operations per second of: fma.rn.f32, lop3.b32,
 * mul.hi.u32, ex2.approx.f32, lg2.approx.f32. Allocates a 4 KB sink; synchronises
 * `stream`; about 10 ms of GPU time. */
CVA_API cva_status cva_pipe_peaks(double *out5_host, void *stream);

/* Thread-local message describing the last error of this thread. */
CVA_API const char *cva_last_error(void);

/* Library build information: "sm_103a <version>". */
CVA_API const char *cva_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CVA_H */
