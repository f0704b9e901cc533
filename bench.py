#!/usr/bin/env python
"""Benchmark of the hierarchical pathwise-CVA hot path on one GB300 (or N, one
process per GPU under torchrun, each rank simulating its own range of outer paths).

A step is one pass of the whole path over one batch: the outer-path kernel
(factors, MtM, exposures), the inner-default kernel (N default draws per path,
averaged targets), CVA_0, and the per-date regression of the targets on the state
at every date 1..n-1. `value` is outer-path x inner-default x steps per second of
whole steps (inputs resident on the device); `e2e` is the same metric through the
public API with the model and portfolio handed over from host memory each step
and the regression output copied back to host memory.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the reference arm; there is no reference GPU code).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "outer-path·inner-default·steps/s and regression samples/s; adjoint/forward ratio"
UNIT = "outer-path*inner-default*steps/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="paper")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--lsq", action="store_true", help="least-squares regression instead of the workload's MLP")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward measurement")
    p.add_argument("--no-batched", action="store_true", help="skip the 6-portfolio CUDA-graph measurement")
    p.add_argument("--no-alive", action="store_true",
                   help="skip the least squares on (default indicators, state) over the M N sample")
    p.add_argument("--no-precision", action="store_true",
                   help="skip the 2^20-path width-128 network measurement")
    p.add_argument("--no-validation", action="store_true",
                   help="skip the twin, oversimulation and nested Monte Carlo measurements (profiling runs)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the simulation's cost against N and the S = 25 sub-step shape")
    p.add_argument("--tiles", default=None,
                   help="sim_block,price_block,inner_paths,lsq_chunks,portfolios_per_price_block for the timed "
                        "simulation (profiling runs; default: the library's defaults)")
    p.add_argument("--paths", type=int, default=None,
                   help="override the number of outer paths (small cases for profiling captures)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def alu_peak_lane_instr_per_s(sm_mhz, sms):
    """Issue peak of the SM sub-partitions: SMs x 4 schedulers x 32 lanes per clock."""
    return sms * 4 * 32 * sm_mhz * 1e6


def _shape(wl):
    m = wl.model
    CS = int(np.count_nonzero(m.cir_nu > 0))
    F = 2 * m.E - 1 + CS
    G = 10 if wl.name != "small" else 5
    return m.E, m.C, CS, F, G, len(wl.portfolios), wl.grid.substeps


def sim_instr_per_path_step(wl):
    """Algorithmic lane-instructions of the path-simulation kernel per (path, pricing
    step), counted from the method (not from the compiled code): per Euler sub-step,
    Philox4x32-10 = 10 rounds x 8 integer ops + 4 counter ops per block of four draws,
    4 ops per uniform, 20 per Box-Muller pair, F(F+1)/2 FMA for the correlation, 4 per
    rate and FX factor, 8 per CIR intensity, 5 per integrated intensity (compensated,
    non-decreasing sum), 1 for the FP64 discount integral; per pricing date 12 per
    counterparty for the threshold 1 - exp(-Lambda)."""
    E, C, CS, F, G, NPF, S = _shape(wl)
    blocks = (F + 3) // 4
    sub = blocks * (84 + 16 + 40) + F * (F + 1) // 2 + 4 * E + 4 * (E - 1) + 8 * CS + 5 * C + 1
    return S * sub + 12 * C


def price_instr_per_path_date(wl):
    """Algorithmic lane-instructions of the pricing kernel per (path, pricing date):
    20 per economy for the first live bond and the running fixing, 12 per (economy,
    reset date) for the chained bond prices and their differences (degree-8 series),
    (2G+1) per (portfolio, counterparty, economy) for the date-bucketed MtM, 3 per
    (portfolio, counterparty) for the exposure and 6 for the discount factor."""
    E, C, CS, F, G, NPF, S = _shape(wl)
    return 20 * E + 12 * E * G + NPF * C * E * (2 * G + 1) + 3 * NPF * C + 6


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work from one
# ncu capture of each kernel in its current form (profiles/), scaled to a launch by
# the units it processes. The simulation kernels were captured at 32768 paths of the
# paper workload (part of their writes still sat in the 129 MB L2 when they ended,
# so the scaled figures are lower bounds); the trainer at the benchmark's 2^17 paths.
NCU_TRAFFIC = {
    "sim_kernel": {"bytes_per_unit": (0.12e6 + 415.28e6) / (32768 * 100), "unit": "path-step",
                   "profile": "profiles/sim_price_inner_kernels_paper_32k.md"},
    "price_kernel": {"bytes_per_unit": (263.78e6 + 81.86e6) / (32768 * 100), "unit": "path-date",
                     "profile": "profiles/sim_price_inner_kernels_paper_32k.md"},
    # one launch = one epoch at one date; captured at 65536 paths, scaled by the paths
    "mlp_train_kernel": {"bytes_per_unit": (7.506432e6 + 0.0) / 65536, "unit": "path",
                         "profile": "profiles/mlp_train_kernel_paper_64k.md"},
    # width 128: one launch = one epoch at one date; captured at 131072 paths (second
    # launch of the capture), scaled by the paths
    "wide_train_kernel": {"bytes_per_unit": (15.038720e6 + 0.005120e6) / 131072, "unit": "path",
                          "profile": "profiles/wide_train_kernel_precision_128k.md"},
}


def mlp_flops_per_date(M, d, u, epochs):
    """Algorithmic FLOPs of Algorithm 1 at one date for the NN+ network d -> u -> u -> 1:
    per sample and epoch a forward pass 2(d u + u^2) and a backward pass 2(u^2 + u^2 + d u)
    (dH1, dW2, dW1), plus full-sample forward passes for the epoch losses, the refit's
    Gram matrix and the predictions (epochs + 2)."""
    fwd = 2 * (d * u + u * u)
    bwd = 2 * (u * u + u * u + d * u)
    return M * (epochs * (fwd + bwd) + (epochs + 2) * fwd)


def mlp_train_flops_per_launch(M, d, u):
    """Algorithmic FLOPs of one launch of the training kernel, one epoch of Algorithm 1
    (every sample once): forward 2(d u + u^2) and backward 2(u^2 + u^2 + d u) per sample."""
    return M * (2 * (d * u + u * u) + 2 * (u * u + u * u + d * u))


def inner_bytes_per_path(wl):
    """HBM bytes the inner-default kernel must move per outer path: thresholds and
    exposures of dates 1..n (read), the discount integrals of dates 0..n-1 (read) and
    the targets of dates 0..n-1 (written)."""
    n, C, P = wl.grid.n_steps, wl.model.C, len(wl.portfolios)
    return 4 * (n * C + P * n * C + n + P * n)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        import torch
        self.index = str(device_index)
        try:   # address the GPU by UUID: CUDA_VISIBLE_DEVICES may renumber devices
            u = str(torch.cuda.get_device_properties(device_index).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(wl, M_sample, use_mlp=None, n_threads=0):
    """Time the FP64 oracle on the first M_sample outer paths of the workload: simulation,
    targets and the per-date regression (Algorithm 2 with the NN+ network for the MLP
    workloads, least squares otherwise). Returns (seconds, threads, oracle outputs,
    per-date regression results)."""
    import oracle
    from oracle import mlp as omlp
    from paper_2211_17005_gb300 import workload
    oracle.build()
    if use_mlp is None:
        use_mlp = wl.regression == "mlp"
    t0 = time.perf_counter()
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, M_sample, wl.N, wl.seed,
                        want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"), n_threads=n_threads)
    dates = range(1, wl.grid.n_steps)
    if use_mlp:
        p0 = workload.mlp_init(wl.model.F, wl.hidden or 64)
        reg = omlp.backward_alg(p0, o["features"], o["xi_bar"], dates, n_batches=32, epochs=8, lr=1e-3)
    else:
        reg = {}
        for i in dates:
            phi = oracle.linear_features(o["features"][i]) if wl.name != "small" else \
                oracle.poly2_features(o["features"][i, 0])
            reg[i] = oracle.lsq(phi, o["xi_bar"][i])
    dt = time.perf_counter() - t0
    return dt, (n_threads or os.cpu_count()), o, reg


def sim_errors(api, o, wl, M, pf=0, keep_sim=False, tiles=None):
    """Errors of the GPU simulation (first M paths, the workload's seed, portfolio pf)
    against the oracle's outputs o on the same paths: CVA_0, every per-path target
    (against the oracle's targets rebuilt at the GPU's default step on tie-moved draws)
    and the default steps."""
    import oracle
    import torch
    from oracle import compare
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, M, wl.N, keep_defaults=True)
    if tiles:   # the tile shapes (and pricing form) of the measured run
        sim.set_tiles(tiles["sim_block"], tiles["price_block"], tiles["inner_paths_per_block"],
                      tiles["lsq_chunk_target"], tiles["portfolios_per_price_block"])
    sim.run(wl.seed)
    torch.cuda.synchronize()
    idx = sim.defaults().cpu().numpy()
    xi = sim.targets()[pf].cpu().numpy()
    c0 = sim.cva0(pf)[0]
    eps = oracle.exp_clocks(wl.seed, 0, M, wl.N, wl.model.C)
    d = compare.default_mismatches(idx, o["idx"], o["Lambda"], eps, wl.grid.n_steps)
    ref = compare.tie_corrected_targets(o, wl.model.recovery, idx, d["mism"])
    c_or, c_corr = float(o["xi_bar"][0].mean()), float(ref[0].mean())
    out = {"paths": M, "draws": d["draws"], "default_step_mismatches": d["n_mism"], "ties": d["n_tie"],
           "tie_share": d["n_tie"] / d["draws"], "mismatches_outside_tie_band": len(d["outside"]),
           "cva0_gpu": c0, "cva0_oracle": c_or, "cva0_rel_err": abs(c0 - c_or) / c_or,
           "cva0_rel_err_tie_corrected": abs(c0 - c_corr) / c_corr,
           "targets": compare.target_errors(xi, ref, c_corr),
           "tolerances": {"cva0_rel": compare.CVA0_RTOL, "target_rel": compare.XI_RTOL,
                          "target_floor_cva0": compare.XI_FLOOR_CVA0, "tie_share_max": compare.TIE_MAX_SHARE}}
    if keep_sim:
        return out, sim, c_corr
    sim.close()
    return out


def lsq_gap(pred_gpu, feats_or, xi_or, dates, cva0, poly2=False):
    """Largest and median RMS gap, in units of CVA_0, between the GPU's per-date least
    squares predictions and the oracle's QR fit on its own data."""
    import oracle
    gaps = []
    for i in dates:
        phi = oracle.poly2_features(feats_or[i, 0]) if poly2 else oracle.linear_features(feats_or[i])
        _, po = oracle.lsq(phi, xi_or[i])
        gaps.append(float(np.sqrt(np.mean((pred_gpu[i].astype(np.float64) - po) ** 2))) / cva0)
    return {"l2_gap_over_cva0_max": max(gaps), "l2_gap_over_cva0_median": float(np.median(gaps)),
            "dates": len(gaps), "bound": 1e-3}


def mlp_gaps(pred_gpu, xi_gpu, res, xi_or, dates):
    """Per-date gaps of the GPU's NN+ regression against the FP64 oracle's Algorithm 1/2:
    the relative excess of the GPU's training loss over the oracle's, and the RMS gap of
    the predictions in units of the targets' RMS."""
    lg, pg = [], []
    for i in dates:
        p_or = res[i][2]
        l_gpu = float(np.mean((pred_gpu[i].astype(np.float64) - xi_gpu[i]) ** 2))
        l_or = float(np.mean((p_or - xi_or[i]) ** 2))
        lg.append((l_gpu - l_or) / l_or)
        pg.append(float(np.sqrt(np.mean((pred_gpu[i] - p_or) ** 2)) / np.sqrt(np.mean(xi_or[i] ** 2))))
    return {"loss_excess_max": max(lg), "loss_excess_median": float(np.median(lg)),
            "pred_gap_over_target_rms_max": max(pg), "pred_gap_over_target_rms_median": float(np.median(pg)),
            "dates": len(lg)}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2211_17005_gb300 import workload
    wl = workload.make(args.workload)
    M_sample = 1024 if wl.name != "small" else 4096
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, M_sample)
    times = []
    for _ in range(args.steps):
        dt, cores, _, _ = cpu_oracle_sample(wl, M_sample)
        times.append(dt)
    t = float(np.sum(times))
    value = args.steps * M_sample * wl.N * wl.grid.n_steps / t
    cb = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"first {M_sample} of {wl.M} outer paths per step, all {wl.N} inner draws, "
                    f"{wl.grid.n_steps} dates, per-date "
                    + ("NN+ Algorithm 2" if wl.regression == "mlp" else "least squares")}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": describe(wl), "M_sample": M_sample},
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


def describe(wl):
    m = wl.model
    return (f"{wl.name}: E={m.E} economies, C={m.C} counterparties, F={m.F} factors, "
            f"{sum(p.n_swaps for p in wl.portfolios)} swaps in {len(wl.portfolios)} portfolio(s), "
            f"n={wl.grid.n_steps} steps over {wl.grid.horizon:g}y, S={wl.grid.substeps}, "
            f"M={wl.M}, N={wl.N}")


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2211_17005_gb300 import api, build, workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    build.build()
    wl = workload.make(args.workload, M=args.paths)
    basis = "poly2" if wl.name == "small" else "linear"
    use_mlp = wl.regression == "mlp" and not args.lsq
    hidden, n_batches, epochs, lr = (wl.hidden or 64), 32, 8, 1e-3
    if use_mlp:
        p_init = api.mlp_pack(workload.mlp_init(wl.model.F, hidden), hidden)
        p_work = p_init.clone()

    def regress(s):
        """Regression at every date 1..n-1: Algorithm 2 with the NN+ network for the
        MLP workloads, one grouped least-squares launch otherwise."""
        if use_mlp:
            p_work.copy_(p_init)      # every step starts Algorithm 2 from the same initial network
            return api.mlp_regress_all(s, p_work, hidden=hidden, n_batches=n_batches, epochs=epochs, lr=lr)
        return s.regress_all(0, basis=basis, want_coef=False)[0]
    k0 = rank * wl.M          # weak scaling: each rank owns its own outer paths
    sim = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N, profile=True)
    if args.tiles:
        sim.set_tiles(*(int(v) for v in args.tiles.split(",")))
    stream = torch.cuda.current_stream()
    n = wl.grid.n_steps

    def step(seed):
        sim.run(seed, k0=k0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pred = regress(sim)
        ev1.record(stream)
        c0 = sim.cva0(0)
        return c0, (ev0, ev1), pred

    if use_mlp:
        api.mlp_kernel_timing(True)      # event pairs around each train launch (created in the warm-up)
    for w in range(args.warmup):
        step(1000 + w)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if use_mlp:
        api.mlp_kernel_timing(False)     # clears the warm-up's totals; on again for the last timed step
    sim_ms, price_ms, inner_ms, reg_ev = [], [], [], []
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        start.record(stream)
        for s in range(args.steps):
            if use_mlp and s == args.steps - 1:
                api.mlp_kernel_timing(True)   # event pairs around the last step's train launches
            c0, evs, last_pred = step(s + 1)
            a_ms, p_ms, i_ms = sim.kernel_ms()
            sim_ms.append(a_ms)
            price_ms.append(p_ms)
            inner_ms.append(i_ms)
            reg_ev.append(evs)
        end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    train_t = api.mlp_kernel_timing(False) if use_mlp else None
    total_ms = start.elapsed_time(end)
    reg_ms = [a.elapsed_time(b) for a, b in reg_ev]
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    units_per_step = wl.M * wl.N * n * world
    value = units_per_step * args.steps / (t_max / 1e3)

    # ---- twin Monte Carlo validation of the last step's regression at the middle date ----
    twin = None
    if rank == 0 and not args.no_validation:
        i_tw = n // 2
        phi = last_pred[i_tw].clone()
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        xs = []
        for cpy in (1, 2):
            sim.run_twin(args.steps, i_tw, cpy, k0=k0)
            xs.append(sim.targets()[0, i_tw].clone())
        est, se = api.twin_l2(phi, xs[0], xs[1])
        t1e.record(stream)
        torch.cuda.synchronize()
        scale = float(torch.mean(xs[0].double() * xs[1].double()))   # estimates E[(E[xi | state])^2]
        twin = {"date": i_tw, "regression": "the step's" + (" NN+ network" if use_mlp else " least squares"),
                "l2_error": est, "l2_se": se,
                "relative_rmse": (max(est, 0.0) ** 0.5) / (scale ** 0.5) if scale > 0 else None,
                "ms": t0e.elapsed_time(t1e),
                "estimator": "mean of phi^2 - (xi1 + xi2) phi + xi1 xi2 over two copies branched at the date"}

    # ---- oversimulation factor (Prop. 1, Heuristic 1) for the step's regression ----
    oversim = None
    if rank == 0 and not args.no_validation:
        sim.run(args.steps, k0=k0)   # the buffers hold twin copy 2: the step's own paths again
        torch.cuda.synchronize()
        Qs, Rs = sim.oversim_stats(last_pred, args.steps)
        N_small, N_big = 8, 512   # a wide spread of N: the time difference is the measured quantity
        sim_small = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, N_small)
        sim_big = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, N_big)
        def sim_time(sx, reps=10):
            sx.run(1, k0=k0)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                sx.run(1, k0=k0)
            a1.record(stream)
            torch.cuda.synchronize()
            return a0.elapsed_time(a1) / reps
        t_small, t_big = sim_time(sim_small), sim_time(sim_big)
        sim_small.close()
        sim_big.close()
        kappa = api.inner_cost_ratio(t_small, N_small, t_big, N_big)
        Ni, N_star, M_star = api.oversimulation_choice(Qs[1:n], Rs[1:n], kappa, budget=wl.M * (wl.N + kappa))
        oversim = {"kappa": kappa, "timings_ms": {f"N={N_small}": t_small, f"N={N_big}": t_big},
                   "N_heuristic1": N_star, "M_for_the_same_budget": M_star,
                   "N_i_median": float(np.nanmedian(Ni)), "Q_over_R_median": float(np.nanmedian(Qs[1:n] / Rs[1:n])),
                   "regression": "the step's" + (" NN+ network" if use_mlp else " least squares"),
                   "note": "kappa: cost of an outer path in inner draws from two simulations of the same M (eq. (l:ratio))"}

    # ---- the simulation's cost against N at fixed M, and at the paper's S = 25 sub-steps ----
    extras = None
    if rank == 0 and not args.no_extras and wl.name == "paper":
        def time_sim(grid, Nx, reps=5):
            xs = api.Simulation(wl.model, wl.portfolios, grid, wl.M, Nx, profile=True)
            xs.run(1, k0=k0)
            torch.cuda.synchronize()
            parts = []
            for r in range(reps):
                xs.run(2 + r, k0=k0)
                torch.cuda.synchronize()
                parts.append(xs.kernel_ms())
            xs.close()
            med = np.median(np.array(parts), axis=0)
            return {"ms": float(med.sum()), "path_simulation_ms": float(med[0]), "pricing_ms": float(med[1]),
                    "inner_defaults_ms": float(med[2])}
        by_N = {f"N={Nx}": time_sim(wl.grid, Nx) for Nx in (1, 8, 64, 256, 1024)}
        g25 = workload.Grid(wl.grid.horizon, wl.grid.n_steps, 25)
        s25 = time_sim(g25, wl.N)
        s25["value"] = wl.M * wl.N * n / (s25["ms"] / 1e3)
        s25["unit"] = UNIT
        extras = {"simulation_vs_N": by_N,
                  "note_N": f"M = {wl.M}, n = {n}: the inner draws are the only part that grows with N",
                  "substeps_25": s25,
                  "note_S": "the paper's Euler grid (25 sub-steps per pricing step), N as configured",
                  "timing": "median of 5 simulations after one warm-up, CUDA events of the library (profiling flag)"}

    # ---- nested Monte Carlo reference at the middle date (first 16384 paths, 1024 copies) ----
    nested = None
    if rank == 0 and not args.no_validation:
        Mv, K = min(16384, wl.M), 1024
        i_n = n // 2
        sim_v = api.Simulation(wl.model, wl.portfolios, wl.grid, Mv, wl.N)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        ref_n = sim_v.nested_reference(args.steps, i_n, K, k0=k0)
        q1.record(stream)
        torch.cuda.synchronize()
        rr, cnt = api.relative_rmse(last_pred[i_n, :Mv].contiguous(), ref_n)
        sim_v.close()
        nested = {"date": i_n, "paths": Mv, "copies": K, "relative_rmse": rr, "paths_with_nonzero_reference": cnt,
                  "ms": q0.elapsed_time(q1),
                  "regression": "the step's" + (" NN+ network" if use_mlp else " least squares"),
                  "measure": "sqrt(mean(((pred - nested) / nested)^2)) over paths with a nonzero nested value"}

    # ---- end to end through the public API: host inputs in, host results out ----
    pinned = torch.empty((n, wl.M), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 5))
    h2d = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        sim2 = api.Simulation(wl.model, wl.portfolios, wl.grid, wl.M, wl.N)
        sim2.run(s + 1, k0=k0)
        pred = regress(sim2)
        c0e = sim2.cva0(0)
        pinned.copy_(pred, non_blocking=True)
        torch.cuda.synchronize()
        sim2.close()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    E, C, G = wl.model.E, wl.model.C, (10 if wl.name != "small" else 5)
    h2d = 8 * (n + 1) * E * G + 8 * (n // 1 + 2) * E + 4 * (n + 1) + 4 * n * wl.grid.substeps * E
    d2h = 4 * n * wl.M + 16
    e2e_value = units_per_step / e2e_s

    # kernels of this library launched per step: path simulation, pricing, inner defaults,
    # the two CVA_0 reduction stages, then the regression: for Algorithm 2 one
    # standardisation launch and per date E train launches, E loss passes, the refit's
    # Gram pass and the prediction pass, and the refit; for least squares the grouped
    # Gram, solve and prediction launches
    launches_per_step = 3 + 2 + ((1 + (n - 1) * (2 * epochs + 3)) if use_mlp else 3)

    # ---- roofline of the dominant kernel ----
    pk, src = peaks()
    s_avg, p_avg, i_avg = float(np.mean(sim_ms)), float(np.mean(price_ms)), float(np.mean(inner_ms))
    clk = clocks.summary()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak_alu = alu_peak_lane_instr_per_s(sm_mhz, n_sms)
    pipes = api.pipe_peaks() if rank == 0 else None
    kern = {"sim_kernel": (sim_instr_per_path_step(wl), s_avg, "path-step"),
            "price_kernel": (price_instr_per_path_date(wl), p_avg, "path-date")}
    alu = {}
    for name, (per_unit, ms, unit) in kern.items():
        ach = per_unit * wl.M * n / (ms / 1e3)
        tr = NCU_TRAFFIC.get(name) if wl.name == "paper" else None
        alu[name] = {"bound": "alu", "kernel": name, "achieved": ach / 1e12, "peak": peak_alu / 1e12,
                     "unit": "T lane-instr/s", "frac": ach / peak_alu,
                     "traffic": tr["bytes_per_unit"] * wl.M * n if tr else None,
                     "traffic_source": tr["profile"] if tr else None,
                     "algorithmic_instr_per_unit": per_unit, "unit_of_work": unit, "ms": ms}
    dom = max(alu, key=lambda k: alu[k]["ms"])
    roof = dict(alu[dom])
    roof["peak_source"] = f"{n_sms} SMs x 128 lanes x {sm_mhz:g} MHz ({src} max SM clock)"
    hbm = pk.get("hbm_gbs", 6800.0)
    inner_gbs = inner_bytes_per_path(wl) * wl.M / (i_avg / 1e3) / 1e9
    reg_bytes = 4 * (n - 1) * wl.M * (wl.model.F + 1 + 1)
    reg_gbs = reg_bytes / (np.mean(reg_ms) / 1e3) / 1e9
    mlp_roof = None
    if use_mlp:
        per_date = mlp_flops_per_date(wl.M, wl.model.F, hidden, epochs)
        flops = per_date * (n - 1)
        tf_alg2 = flops / (np.mean(reg_ms) / 1e3) / 1e12
        peak_tf = pk.get("bf16_tflops_sustained", 1720.9)
        per_launch = mlp_train_flops_per_launch(wl.M, wl.model.F, hidden)
        launch_ms = train_t["ms"] / max(train_t["launches"], 1)
        tf = per_launch / (launch_ms / 1e3) / 1e12
        tr = (NCU_TRAFFIC.get("mlp_train_kernel") if (wl.name == "paper" and hidden == 64) else
              NCU_TRAFFIC.get("wide_train_kernel") if (wl.name == "precision" and hidden == 128) else None)
        mlp_roof = {"bound": "tensor", "kernel": "mlp_train_kernel" if hidden == 64 else "wide_train_kernel",
                    "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                    "traffic": tr["bytes_per_unit"] * wl.M if tr else None,
                    "traffic_source": tr["profile"] if tr else None,
                    "algorithmic_flops_per_launch": per_launch, "launch_ms": launch_ms,
                    "launches": train_t["launches"], "ms": train_t["ms"],
                    "timing": "CUDA events around every train launch of the last timed step, on its stream",
                    "peak_source": "measured bf16 cuBLAS, sustained",
                    "algorithm2": {"achieved": tf_alg2, "frac": tf_alg2 / peak_tf, "ms": float(np.mean(reg_ms)),
                                   "algorithmic_flops_per_date": per_date, "dates": n - 1,
                                   "note": "every pass of Algorithm 2 (training, loss sweeps, refit, predictions) "
                                           "over the whole regression time"}}

    # ---- adjoint / forward cost of CVA_0 sensitivities (adjoint workload, rank 0) ----
    adj = None
    if rank == 0 and not args.no_adjoint:
        awl = workload.make("adjoint", M=args.paths)
        apf = api.frozen(awl.model, awl.portfolios[0])

        def timed(fwd_only):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c, g = api.grad_cva0(awl.model, apf, awl.grid, awl.M, awl.seed, ckpt_every=10, forward_only=fwd_only)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), c

        timed(True)
        timed(False)
        t_f = [timed(True)[0] for _ in range(3)]
        t_a = [timed(False)[0] for _ in range(3)]
        adj = {"workload": describe(awl) + ", 53 parameters, checkpoint every 10 dates",
               "adjoint_ms": float(np.median(t_a)), "smooth_forward_ms": float(np.median(t_f)),
               "ratio": float(np.median(t_a) / np.median(t_f))}

    # ---- batched workload: 6 portfolios, all simulations and 120 x 6 regressions replayed as one CUDA graph ----
    batched = None
    if rank == 0 and not args.no_batched:
        bwl = workload.make("batched", M=args.paths)
        bsim = api.Simulation(bwl.model, bwl.portfolios, bwl.grid, bwl.M, bwl.N)
        tiles = bsim.autotune(bwl.seed, "linear")
        bpred = torch.zeros((bsim.n_pf, bsim.n, bsim.M), dtype=torch.float32, device="cuda")
        bsim.run(bwl.seed)
        bsim.regress_portfolios("linear", pred=bpred)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            with torch.cuda.graph(graph, stream=gs):
                bsim.run(bwl.seed, stream=gs)
                bsim.regress_portfolios("linear", pred=bpred, stream=gs)
        graph.replay()
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        g0.record(stream)
        for _ in range(reps):
            graph.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / reps
        bn = bwl.grid.n_steps
        batched = {"workload": describe(bwl), "regression": "least squares [1, Y] for 6 x 119 (portfolio, date) pairs, "
                   "one grouped launch, shared normal matrices", "graph_ms": gms,
                   "value": bwl.M * bwl.N * bn / (gms / 1e3), "unit": UNIT,
                   "regression_samples_per_s": bwl.M * (bn - 1) * len(bwl.portfolios) / (gms / 1e3),
                   "tiles": tiles, "replays": reps, "l2": "working set 48 GB > L2"}
        bsim.close()
        del bpred, graph
        # where a replay's time goes: the same launches run eagerly with per-kernel events
        # (the tile choice is the cached one)
        psim = api.Simulation(bwl.model, bwl.portfolios, bwl.grid, bwl.M, bwl.N, profile=True)
        psim.autotune(bwl.seed, "linear")
        ppred = torch.zeros((psim.n_pf, psim.n, psim.M), dtype=torch.float32, device="cuda")
        parts = []
        for _ in range(2):
            psim.run(bwl.seed)
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            psim.regress_portfolios("linear", pred=ppred)
            r1.record(stream)
            torch.cuda.synchronize()
            parts.append(list(psim.kernel_ms()) + [r0.elapsed_time(r1)])
        k = np.min(np.array(parts), axis=0)
        batched["eager_breakdown_ms"] = {"path_simulation": float(k[0]), "pricing": float(k[1]),
                                         "inner_defaults": float(k[2]), "grouped_least_squares": float(k[3])}
        psim.close()
        del ppred

    # ---- least squares on (default indicators X, state Y) over the M N hierarchical sample (rank 0) ----
    alive = None
    if rank == 0 and not args.no_alive and args.workload in ("paper", "small"):
        xwl = workload.make(args.workload, M=args.paths)
        xsim = api.Simulation(xwl.model, xwl.portfolios, xwl.grid, xwl.M, xwl.N, keep_defaults=True)
        xsim.run(xwl.seed)
        xpred = torch.zeros((xsim.n, xsim.M), dtype=torch.float32, device="cuda")
        _, xcoef, xdrop = xsim.regress_alive(0, pred=xpred)          # allocates the scratch
        torch.cuda.synchronize()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        x0.record(stream)
        for _ in range(reps):
            xsim.regress_alive(0, pred=xpred, want_coef=False)
        x1.record(stream)
        torch.cuda.synchronize()
        xms = x0.elapsed_time(x1) / reps
        xn, xM, xN, xC, xF = xwl.grid.n_steps, xwl.M, xwl.N, xwl.model.C, xwl.model.F
        # bytes a single pass must move: default steps, exposures, discount integrals,
        # features and targets of the regressed dates, predictions written
        xbytes = xM * xN * xC + 4 * xM * ((xn + 1) * (xC + 1) + (xn - 1) * (xF + 2))
        xgbs = xbytes / (xms / 1e3) / 1e9
        alive = {"workload": describe(xwl),
                 "regression": f"least squares on [1, Y ({xF}), X ({xC})] over M N = {xM * xN} rows per date, "
                               f"{xn - 1} dates, per-path exact draw statistics (no M N design)",
                 "ms": xms, "rows_per_s": xM * xN * (xn - 1) / (xms / 1e3),
                 "dropped_columns": int(np.sum(xdrop)),
                 "roofline": {"bound": "hbm", "kernel": "cva_regress_alive (4 kernels)", "achieved": xgbs,
                              "peak": hbm, "unit": "GB/s", "frac": xgbs / hbm, "traffic": None,
                              "algorithmic_bytes": int(xbytes),
                              "note": "latency-bound per-path event walk, not HBM-bound"}}
        xsim.close()
        del xpred

    # ---- the 2^20-path workload with the width-128 network (rank 0) ----
    precision = None
    if rank == 0 and not args.no_precision and args.workload != "precision":
        pwl = workload.make("precision", M=args.paths)
        psim = api.Simulation(pwl.model, pwl.portfolios, pwl.grid, pwl.M, pwl.N)
        pinit = api.mlp_pack(workload.mlp_init(pwl.model.F, pwl.hidden), pwl.hidden)
        pn = pwl.grid.n_steps
        psim.run(pwl.seed)
        api.mlp_kernel_timing(True)
        api.mlp_regress_all(psim, pinit.clone(), hidden=pwl.hidden)   # warm-up, creates the timing events
        torch.cuda.synchronize()
        api.mlp_kernel_timing(False)
        sims, regs = [], []
        for _ in range(3):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            psim.run(pwl.seed)
            e1.record(stream)
            api.mlp_regress_all(psim, pinit.clone(), hidden=pwl.hidden)
            e2.record(stream)
            torch.cuda.synchronize()
            sims.append(e0.elapsed_time(e1))
            regs.append(e1.elapsed_time(e2))
        api.mlp_kernel_timing(True)      # one more repetition, outside the median, times each train launch
        api.mlp_regress_all(psim, pinit.clone(), hidden=pwl.hidden)
        p_train = api.mlp_kernel_timing(False)
        p_sim, p_reg = float(np.median(sims)), float(np.median(regs))
        pflops = mlp_flops_per_date(pwl.M, pwl.model.F, pwl.hidden, epochs) * (pn - 1)
        ptf = pflops / (p_reg / 1e3) / 1e12
        peak_tf = pk.get("bf16_tflops_sustained", 1720.9)
        p_launch = mlp_train_flops_per_launch(pwl.M, pwl.model.F, pwl.hidden)
        p_launch_ms = p_train["ms"] / max(p_train["launches"], 1)
        p_tf = p_launch / (p_launch_ms / 1e3) / 1e12
        precision = {"workload": describe(pwl) + f", NN+ {pwl.model.F}->{pwl.hidden}->{pwl.hidden}->1, Algorithm 2 "
                                                 f"over {pn - 1} dates (E={epochs}, |B|={n_batches})",
                     "sim_ms": p_sim, "regression_ms": p_reg, "step_ms": p_sim + p_reg, "repetitions": 3,
                     "timing": "median of 3 (simulation, Algorithm 2) pairs after a warm-up, CUDA events",
                     "trainer": api.mlp_plan(pwl.M, pwl.hidden, n_batches),
                     "value": pwl.M * pwl.N * pn / ((p_sim + p_reg) / 1e3), "unit": UNIT,
                     "regression_samples_per_s": pwl.M * (pn - 1) / (p_reg / 1e3),
                     "roofline": {"bound": "tensor", "kernel": "wide_train_kernel",
                                  "achieved": p_tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": p_tf / peak_tf,
                                  "traffic": NCU_TRAFFIC["wide_train_kernel"]["bytes_per_unit"] * pwl.M,
                                  "traffic_source": NCU_TRAFFIC["wide_train_kernel"]["profile"],
                                  "algorithmic_flops_per_launch": p_launch,
                                  "launch_ms": p_launch_ms, "launches": p_train["launches"],
                                  "timing": "CUDA events around every train launch of a 4th repetition",
                                  "peak_source": "measured bf16 cuBLAS, sustained",
                                  "algorithm2": {"achieved": ptf, "frac": ptf / peak_tf, "algorithmic_flops": pflops,
                                                 "note": "every pass of Algorithm 2 over the whole regression "
                                                         "time"}}}
        psim.close()

    # ---- the FP64 oracle: CPU baseline on a path prefix, and the error of every
    # benchmarked result against it (rank 0; after every timed region) ----
    cpu, errors = None, None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import compare as ocmp
        from oracle import mlp as omlp
        import oracle
        M_s = 4096 if wl.name != "small" else wl.M
        dt, cores, o, reg_or = cpu_oracle_sample(wl, M_s, use_mlp)
        cpu = {"value": M_s * wl.N * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {M_s} of {wl.M} outer paths, all {wl.N} inner draws, {n} dates, "
                         f"per-date {'NN+ Algorithm 2' if use_mlp else 'least squares'} ({dt:.1f} s)"}
        # one host core: the oracle's simulation and regression of the first 512 paths
        M_1 = 512 if wl.name != "small" else 2048
        dt1, _, _, _ = cpu_oracle_sample(wl, M_1, use_mlp and M_1 % 32 == 0, n_threads=1)
        cpu["one_core"] = {"value": M_1 * wl.N * n / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"first {M_1} paths, simulation on 1 thread, numpy regression ({dt1:.1f} s)"}
        errors = {"note": "GPU result on the first paths of the workload (its seed) against the FP64 oracle on "
                          "the same paths; targets and CVA_0 also against the oracle rebuilt at the GPU's default "
                          "step on tie-moved draws"}
        e_sim, gsim, c_corr = sim_errors(api, o, wl, M_s, keep_sim=True)
        errors["timed_workload"] = e_sim
        g_lsq, _ = gsim.regress_all(0, basis=basis, want_coef=False)
        errors["timed_workload"]["least_squares"] = lsq_gap(g_lsq.cpu().numpy(), o["features"], o["xi_bar"],
                                                            range(1, n), c_corr, poly2=(basis == "poly2"))
        if use_mlp:
            g_pred = api.mlp_regress_all(gsim, p_init.clone(), hidden=hidden, n_batches=n_batches,
                                         epochs=epochs, lr=lr).cpu().numpy()
            errors["timed_workload"]["nn_algorithm2"] = mlp_gaps(g_pred, gsim.targets()[0].cpu().numpy()
                                                                 .astype(np.float64), reg_or, o["xi_bar"],
                                                                 range(1, n))
        gsim.close()
        del o, reg_or

        if not args.no_precision and args.workload != "precision":
            pwl = workload.make("precision", M=args.paths)
            Mp = 4096
            po = oracle.simulate(pwl.model, pwl.portfolios[0], pwl.grid, 0, Mp, pwl.N, pwl.seed,
                                 want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
            e_p, psim2, pc = sim_errors(api, po, pwl, Mp, keep_sim=True)
            i_m = pwl.grid.n_steps // 2
            feats_t = psim2.features()[i_m].contiguous()
            targ_t = psim2.targets()[0, i_m].contiguous()
            pp = api.mlp_pack(workload.mlp_init(pwl.model.F, pwl.hidden), pwl.hidden)
            pred_g, _ = api.mlp_fit(targ_t, feats_t, pp, hidden=pwl.hidden, n_batches=n_batches, epochs=epochs, lr=lr)
            Zo, _, _ = omlp.standardize(po["features"][i_m].T)
            bp, _ = omlp.base_alg(workload.mlp_init(pwl.model.F, pwl.hidden), Zo, po["xi_bar"][i_m],
                                  n_batches=n_batches, epochs=epochs, lr=lr)
            e_p["nn_algorithm1_middle_date"] = mlp_gaps({i_m: pred_g.cpu().numpy()},
                                                        {i_m: targ_t.cpu().numpy().astype(np.float64)},
                                                        {i_m: (bp, None, omlp.forward(bp, Zo, 1)[0])},
                                                        po["xi_bar"], [i_m])
            psim2.close()
            errors["precision"] = e_p
            del po

        if not args.no_batched:
            bwl = workload.make("batched", M=args.paths)
            Mb, pb = 1024, len(bwl.portfolios) - 1      # the 2000-swap portfolio
            bo = oracle.simulate(bwl.model, bwl.portfolios[pb], bwl.grid, 0, Mb, bwl.N, bwl.seed,
                                 want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"))
            e_b, bsim2, bc = sim_errors(api, bo, bwl, Mb, pf=pb, keep_sim=True,
                                        tiles=batched["tiles"] if batched else None)
            bpred2, _ = bsim2.regress_portfolios("linear")
            e_b["least_squares"] = lsq_gap(bpred2[pb].cpu().numpy(), bo["features"], bo["xi_bar"],
                                           range(1, bwl.grid.n_steps), bc)
            e_b["portfolio"] = f"{pb} ({bwl.portfolios[pb].n_swaps} swaps) of the six, simulated together"
            e_b["tiles"] = batched["tiles"] if batched else None
            bsim2.close()
            errors["batched"] = e_b
            del bo

        if not args.no_adjoint:
            awl = workload.make("adjoint", M=args.paths)
            apf = api.frozen(awl.model, awl.portfolios[0])
            Ma = 128
            c_g, g_g = api.grad_cva0(awl.model, apf, awl.grid, Ma, awl.seed, ckpt_every=10)
            from oracle import dual as odual
            ref = odual.smooth_cva0_grad(awl.model, apf, awl.grid, Ma, awl.seed)
            c_o, fd = ref["cva0"], ref["grad"]
            sc = float(np.max(np.abs(fd)))
            big = np.abs(fd) > 1e-3 * sc
            errors["adjoint"] = {"paths": Ma, "parameters": int(fd.size),
                                 "smooth_cva0_rel_err": abs(c_g - c_o) / c_o,
                                 "grad_max_abs_err_over_max_grad": float(np.max(np.abs(g_g - fd))) / sc,
                                 "grad_max_rel_err_components_above_1e-3_max": float(np.max(np.abs(g_g - fd)[big]
                                                                                         / np.abs(fd[big]))),
                                 "reference": "the oracle's FP64 forward-mode (dual-number) gradient of its smooth "
                                              "CVA_0 on the same paths (common random numbers)"}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": describe(wl),
                          "regression": (f"NN+ {wl.model.F}->{hidden}->{hidden}->1, Algorithm 2 over {n - 1} dates, "
                                         f"E={epochs}, |B|={n_batches}, Adam lr={lr}, tcgen05 BF16 GEMMs")
                          if use_mlp else f"least squares, basis {basis}",
                          "seed_per_step": "1..K", "l2": "working set > L2: 2.3 GB written per step",
                          "parallelism": f"{world} rank(s), disjoint outer-path ranges"},
               "sim_ms": s_avg + p_avg + i_avg, "sim_kernel_ms": s_avg, "price_kernel_ms": p_avg,
               "inner_kernel_ms": i_avg, "regression_ms": float(np.mean(reg_ms)),
               "sim_throughput": wl.M * wl.N * n / ((s_avg + p_avg + i_avg) / 1e3),
               "alu_kernels": alu,
               "pipe_peaks_measured": ({k: v / 1e12 for k, v in pipes.items()} | {
                   "unit": "T lane-op/s", "issue_peak": peak_alu / 1e12,
                   "note": "cva_pipe_peaks: 8 independent chains per thread, 64 warps per SM"}) if pipes else None,
               "regression_samples_per_s": wl.M * (n - 1) / (np.mean(reg_ms) / 1e3),
               "inner_kernel_gbs": inner_gbs, "regression_gbs": reg_gbs, "hbm_peak_gbs": hbm,
               "cva0": c0[0], "cva0_se": c0[1],
               "roofline": (mlp_roof if (mlp_roof and mlp_roof["ms"] > roof["ms"]) else roof),
               "mlp_roofline": mlp_roof, "twin_validation": twin, "oversimulation": oversim,
               "nested_validation": nested, "paper_shape_extras": extras,
               "adjoint_forward": adj, "batched": batched, "alive_regression": alive,
               "precision": precision,
               "cpu_baseline": cpu, "errors_vs_oracle": errors,
               "clocks": clk,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h)},
               "gpu_launches": launches_per_step * args.steps}
        print(json.dumps(out))
    sim.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
