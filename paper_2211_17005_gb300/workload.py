"""Seeded synthetic inputs for the hierarchical CVA workloads.

This module only draws random model parameters and random swap terms. It holds
none of the method's arithmetic: no pricing, no par rates, no simulation and no
Cholesky factorisation. Both the CUDA path and the FP64 oracle take what it
returns as their common input, and each side derives everything else itself.

Workload recipes (Sec. 4.3 of the paper describes the case study: 10 economies,
8 clients, 27 diffusive factors, 500 random swaps at par, n = 100 pricing steps):

* ``small``     1 Hull-White economy (a=0.1, sigma=0.01, flat 2%), 2 counterparties
                with constant hazards 0.02/0.05 and R=0.4, 10 swaps, 50 steps over 5y,
                M=16384 outer paths, N=8 inner defaults, least squares on [1, r, r^2].
* ``paper``     10 economies (a~U[0.05,0.2], sigma~U[0.005,0.015], flat curves
                f~U[0.01,0.03]), 9 lognormal FX (vol~U[0.05,0.15], chi_0=1), 8 CIR
                counterparties (kappa=0.5, theta~U[0.01,0.05], nu=0.05, gamma_0=theta,
                R=0.4), 27 correlated factors, 500 swaps, 100 steps over 10y,
                M=2^17, N=64, MLP 27->64->64->1.
* ``adjoint``   the ``paper`` model at M=2^17 (sensitivities of CVA_0).
* ``precision`` the ``paper`` model at M=2^20, N=128, MLP 27->128->128->1.
* ``batched``   the ``paper`` model with 6 portfolios (50..2000 swaps), 120 steps over
                10y, M=2^20, N=256, linear least squares on [1, Y_t].
* ``mixed``     a shape with no compiled instantiation: 3 economies (paper ranges), 5
                counterparties with constant and CIR intensities interleaved (nu = 0,
                0.05, 0, 0.05, 0.05; the constant ones gamma = 0.02, 0.04), 4
                portfolios of 20, 60, 150, 300 swaps, 40 steps over 10y (quarterly
                pricing, annual resets), M=4096, N=16, linear least squares.

Swap terms: notional ~ LogNormal(0, 0.5); payer (omega=+1) or receiver (-1) with
probability 1/2; currency and counterparty uniform; maturity U[lo, hi] years rounded
to the nearest integer >= 1, annual resets (delta = 1), spot start, fixed rate at par
(each side computes the par rate from the model's curve).

Correlation matrix: off-diagonal entries i.i.d. U[-0.3, 0.3], shrunk towards the
identity, C(lam) = I + lam (R - I), with the largest lam in {1, 0.95, ..., 0.05}
whose smallest eigenvalue is >= 0.05 (an i.i.d. draw at F=27 is not positive
definite). Factor order: r^0..r^{E-1}, log chi^1..log chi^{E-1}, then the
intensities of the counterparties with nu > 0.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

GENERATOR_SEED = 20221130


@dataclasses.dataclass
class Model:
    E: int
    C: int
    hw_a: np.ndarray          # [E]
    hw_sigma: np.ndarray      # [E]
    curve: np.ndarray         # [E] flat initial curve level per economy
    fx_vol: np.ndarray        # [E] entry 0 unused (reference currency)
    fx0: np.ndarray           # [E] entry 0 is 1
    cir_kappa: np.ndarray     # [C]
    cir_theta: np.ndarray     # [C]
    cir_nu: np.ndarray        # [C] 0 => constant intensity gamma0
    gamma0: np.ndarray        # [C]
    recovery: np.ndarray      # [C]
    corr: np.ndarray          # [F, F] correlation of the stochastic factors
    corr_shrink: float = 1.0

    @property
    def n_stoch_cpty(self) -> int:
        return int(np.count_nonzero(self.cir_nu > 0))

    @property
    def F(self) -> int:
        return self.E + (self.E - 1) + self.n_stoch_cpty


@dataclasses.dataclass
class Portfolio:
    ccy: np.ndarray        # [S] int32
    cpty: np.ndarray       # [S] int32
    notional: np.ndarray   # [S] float64
    omega: np.ndarray      # [S] int32, +1 payer, -1 receiver
    n_periods: np.ndarray  # [S] int32, maturity in periods of length delta
    delta: float = 1.0
    fixed_rate: Optional[np.ndarray] = None   # [S]; None: par at t = 0

    @property
    def n_swaps(self) -> int:
        return int(self.ccy.shape[0])


@dataclasses.dataclass
class Grid:
    horizon: float
    n_steps: int
    substeps: int = 1


@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    portfolios: List[Portfolio]
    grid: Grid
    M: int
    N: int
    regression: str            # "lsq-poly2", "lsq-linear", "mlp"
    hidden: Optional[int] = None
    seed: int = 1              # simulation seed (Philox key)


def _shrunk_correlation(rng: np.random.Generator, F: int, rho_max: float = 0.3,
                        min_eig: float = 0.05):
    R = np.eye(F)
    iu = np.triu_indices(F, 1)
    R[iu] = rng.uniform(-rho_max, rho_max, size=len(iu[0]))
    R = R + np.triu(R, 1).T
    for lam in np.arange(1.0, 0.0, -0.05):
        Cm = np.eye(F) + lam * (R - np.eye(F))
        if np.linalg.eigvalsh(Cm).min() >= min_eig:
            return Cm, float(lam)
    return np.eye(F), 0.0


def _swaps(rng: np.random.Generator, n: int, E: int, C: int, mat_lo: float,
           mat_hi: float) -> Portfolio:
    ccy = rng.integers(0, E, size=n).astype(np.int32)
    cpty = rng.integers(0, C, size=n).astype(np.int32)
    notional = rng.lognormal(0.0, 0.5, size=n)
    omega = np.where(rng.uniform(size=n) < 0.5, 1, -1).astype(np.int32)
    mat = rng.uniform(mat_lo, mat_hi, size=n)
    n_periods = np.maximum(1, np.rint(mat)).astype(np.int32)
    return Portfolio(ccy=ccy, cpty=cpty, notional=notional, omega=omega,
                     n_periods=n_periods, delta=1.0)


def small_model() -> Model:
    return Model(
        E=1, C=2,
        hw_a=np.array([0.1]), hw_sigma=np.array([0.01]), curve=np.array([0.02]),
        fx_vol=np.zeros(1), fx0=np.ones(1),
        cir_kappa=np.zeros(2), cir_theta=np.array([0.02, 0.05]), cir_nu=np.zeros(2),
        gamma0=np.array([0.02, 0.05]), recovery=np.array([0.4, 0.4]),
        corr=np.eye(1))


def paper_model(rng: np.random.Generator, E: int = 10, C: int = 8) -> Model:
    hw_a = rng.uniform(0.05, 0.2, size=E)
    hw_sigma = rng.uniform(0.005, 0.015, size=E)
    curve = rng.uniform(0.01, 0.03, size=E)
    fx_vol = np.concatenate([[0.0], rng.uniform(0.05, 0.15, size=E - 1)])
    fx0 = np.ones(E)
    theta = rng.uniform(0.01, 0.05, size=C)
    F = E + (E - 1) + C
    corr, lam = _shrunk_correlation(rng, F)
    return Model(E=E, C=C, hw_a=hw_a, hw_sigma=hw_sigma, curve=curve, fx_vol=fx_vol,
                 fx0=fx0, cir_kappa=np.full(C, 0.5), cir_theta=theta,
                 cir_nu=np.full(C, 0.05), gamma0=theta.copy(),
                 recovery=np.full(C, 0.4), corr=corr, corr_shrink=lam)


def mixed_model(rng: np.random.Generator) -> Model:
    """3 economies, 5 counterparties: constant intensities at 0 and 2, CIR at 1, 3, 4."""
    E, C = 3, 5
    hw_a = rng.uniform(0.05, 0.2, size=E)
    hw_sigma = rng.uniform(0.005, 0.015, size=E)
    curve = rng.uniform(0.01, 0.03, size=E)
    fx_vol = np.concatenate([[0.0], rng.uniform(0.05, 0.15, size=E - 1)])
    theta = rng.uniform(0.01, 0.05, size=C)
    stoch = np.array([False, True, False, True, True])
    const = np.array([0.02, 0.0, 0.04, 0.0, 0.0])
    F = E + (E - 1) + int(stoch.sum())
    corr, lam = _shrunk_correlation(rng, F)
    return Model(E=E, C=C, hw_a=hw_a, hw_sigma=hw_sigma, curve=curve, fx_vol=fx_vol, fx0=np.ones(E),
                 cir_kappa=np.where(stoch, 0.5, 0.0), cir_theta=np.where(stoch, theta, const),
                 cir_nu=np.where(stoch, 0.05, 0.0), gamma0=np.where(stoch, theta, const),
                 recovery=np.full(C, 0.4), corr=corr, corr_shrink=lam)


def make(name: str, M: Optional[int] = None, N: Optional[int] = None,
         n_steps: Optional[int] = None, substeps: int = 1, seed: int = 1,
         n_swaps: Optional[int] = None) -> Workload:
    """Build one of the named workloads; keyword overrides shrink it for tests."""
    if name == "small":
        rng = np.random.default_rng(GENERATOR_SEED + 1)
        model = small_model()
        pf = _swaps(rng, n_swaps or 10, 1, 2, 1.0, 5.0)
        grid = Grid(5.0, n_steps or 50, substeps)
        return Workload(name, model, [pf], grid, M or 16384, N or 8, "lsq-poly2", seed=seed)
    if name in ("paper", "adjoint", "precision"):
        rng = np.random.default_rng(GENERATOR_SEED + 2)
        model = paper_model(rng)
        pf = _swaps(rng, n_swaps or 500, model.E, model.C, 1.0, 10.0)
        grid = Grid(10.0, n_steps or 100, substeps)
        if name == "paper":
            return Workload(name, model, [pf], grid, M or (1 << 17), N or 64, "mlp",
                            hidden=64, seed=seed)
        if name == "adjoint":
            return Workload(name, model, [pf], grid, M or (1 << 17), N or 64, "none",
                            seed=seed)
        return Workload(name, model, [pf], grid, M or (1 << 20), N or 128, "mlp",
                        hidden=128, seed=seed)
    if name == "batched":
        rng = np.random.default_rng(GENERATOR_SEED + 2)
        model = paper_model(rng)
        sizes = [50, 120, 300, 500, 1000, 2000]
        pfs = [_swaps(rng, s, model.E, model.C, 1.0, 10.0) for s in sizes]
        grid = Grid(10.0, n_steps or 120, substeps)
        return Workload(name, model, pfs, grid, M or (1 << 20), N or 256, "lsq-linear",
                        seed=seed)
    if name == "mixed":
        rng = np.random.default_rng(GENERATOR_SEED + 3)
        model = mixed_model(rng)
        pfs = [_swaps(rng, n_swaps or s, model.E, model.C, 1.0, 10.0) for s in (20, 60, 150, 300)]
        grid = Grid(10.0, n_steps or 40, substeps)
        return Workload(name, model, pfs, grid, M or 4096, N or 16, "lsq-linear", seed=seed)
    raise ValueError(f"unknown workload {name!r}")


def single_swap_model(gammas=(0.02, 0.05), recovery=0.4) -> Model:
    """One Hull-White economy with constant-hazard counterparties (used by pins)."""
    m = small_model()
    m.C = len(gammas)
    m.cir_theta = np.array(gammas, dtype=float)
    m.gamma0 = np.array(gammas, dtype=float)
    m.cir_kappa = np.zeros(m.C)
    m.cir_nu = np.zeros(m.C)
    m.recovery = np.full(m.C, recovery)
    return m


def mlp_init(d: int, u: int, seed: int = GENERATOR_SEED + 7):
    """Initial parameters of the NN+ regressor (two hidden layers of width u on d
    inputs): weights and biases U(-1/sqrt(fan_in), 1/sqrt(fan_in)), mu = 0. They are
    an input of the training, shared by the CUDA path and the oracle."""
    rng = np.random.default_rng(seed)

    def unif(fan_in, *shape):
        b = 1.0 / np.sqrt(fan_in)
        return rng.uniform(-b, b, size=shape)

    return {"W1": unif(d, u, d), "b1": unif(d, u), "W2": unif(u, u, u), "b2": unif(u, u),
            "w3": unif(u, u), "b3": np.array(unif(u, 1)[0]), "mu": np.array(0.0)}
