"""The algorithmic work counts behind the benchmark's roofline fractions (CPU).

`achieved` in every roofline entry is an algorithmic count per unit of work times
the units a launch processes, divided by the launch's measured time. These tests
recount the units from the shapes of the operations (GEMM by GEMM, array by
array) instead of from the closed forms in bench.py, and hold the per-unit figures
that the documentation quotes for the timed workloads.
"""
import numpy as np
import pytest

import bench
from paper_2211_17005_gb300 import workload


def _gemm_flops(rows, k, n):
    return 2 * rows * k * n


@pytest.mark.parametrize("M,d,u", [(1 << 17, 27, 64), (1 << 20, 27, 128), (4096, 5, 64)])
def test_train_flops_per_launch_counts_every_gemm_of_an_epoch(M, d, u):
    """One epoch of Algorithm 1 sees every sample once: forward X W1^T and H1 W2^T,
    backward dH1 = dH2 W2 and the weight gradients dW2 = dH2^T H1, dW1 = dH1^T X (the
    output layer's d -> 1 products are vector work, not counted)."""
    fwd = _gemm_flops(M, d, u) + _gemm_flops(M, u, u)
    bwd = _gemm_flops(M, u, u) + _gemm_flops(u, M, u) + _gemm_flops(u, M, d)
    assert bench.mlp_train_flops_per_launch(M, d, u) == fwd + bwd


def test_train_flops_of_the_timed_launches():
    # the figures stated beside the measured launch times
    assert bench.mlp_train_flops_per_launch(1 << 17, 27, 64) == 4127195136
    assert bench.mlp_train_flops_per_launch(1 << 20, 27, 128) == 117574729728


def test_flops_per_date_adds_the_full_sample_passes():
    """Algorithm 1 at one date: E training epochs plus E loss passes, the refit's Gram
    pass and the prediction pass, each a full-sample forward pass."""
    M, d, u, E = 1 << 17, 27, 64, 8
    fwd = _gemm_flops(M, d, u) + _gemm_flops(M, u, u)
    assert bench.mlp_flops_per_date(M, d, u, E) == E * bench.mlp_train_flops_per_launch(M, d, u) + (E + 2) * fwd


def test_inner_bytes_per_path_counts_the_arrays_read_and_written():
    """Per outer path: thresholds [n][C] and exposures [P][n][C] of dates 1..n and the
    discount integrals [n] read, targets [P][n] written, 4 bytes each."""
    for name in ("paper", "batched"):
        wl = workload.make(name, M=256)
        n, C, P = wl.grid.n_steps, wl.model.C, len(wl.portfolios)
        arrays = {"thresholds": (n, C), "exposures": (P, n, C), "discount": (n,), "targets": (P, n)}
        assert bench.inner_bytes_per_path(wl) == 4 * sum(int(np.prod(s)) for s in arrays.values())
    # 7.2 KB per path at the timed workload, 30.2 KB with six portfolios and 120 dates
    assert bench.inner_bytes_per_path(workload.make("paper", M=256)) == 7200
    assert bench.inner_bytes_per_path(workload.make("batched", M=256)) == 30240


def test_instruction_counts_of_the_timed_workload():
    """The per-unit lane-instruction counts quoted for the path simulation and the
    pricing at the timed workload (27 factors, 10 economies, 8 CIR counterparties,
    one portfolio, one Euler sub-step)."""
    wl = workload.make("paper", M=256)
    E, C, CS, F, G, P, S = bench._shape(wl)
    assert (E, C, CS, F, G, P, S) == (10, 8, 8, 27, 10, 1, 1)
    assert bench.sim_instr_per_path_step(wl) == 1635
    assert bench.price_instr_per_path_date(wl) == 3110


def test_alu_issue_peak():
    # 152 SMs x 4 schedulers x 32 lanes at 2070 MHz
    assert bench.alu_peak_lane_instr_per_s(2070.0, 152) == pytest.approx(40.27392e12)
