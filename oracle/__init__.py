"""FP64 CPU oracle for the hierarchical pathwise CVA scheme (arXiv 2211.17005).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it; the product
path never imports it. It shares no code with the CUDA library.

* ``cva_oracle.c`` (built into ``_build/liboracle.so``) simulates the outer paths,
  prices every swap with the three-case formula of App. B, draws the inner default
  clocks of eq. (e:tau) and assembles the averaged target of eq. (eq:CVA_portfolio).
* ``lsq`` solves the per-date least-squares problem of eq. (e:forw) by Householder
  QR (numpy), on the standardised feature map.
* ``twin_l2`` is the twin Monte Carlo estimator of eq. (e:val1) (Sec. ss:twin), and
  ``simulate(..., copy=(date, b))`` runs twin copy b branching at a pricing date.
* ``alive_lsq`` is the least-squares learner on the hierarchically simulated sample
  (X_i^{k,l}, Y_i^k, xi_i^{k,l}) of size M N (Sec. "Learning on Hierarchically
  Simulated Paths"; X the default indicators, Y the market state, Sec. 4.1), with
  the M N design matrix written out row by row.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (binary64, no fast-math, OpenMP)."""
    src = os.path.join(_HERE, "cva_oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Model(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int), ("C", ctypes.c_int)] + [
        (n, ctypes.POINTER(ctypes.c_double)) for n in
        ("a", "sigma_r", "f", "sigma_chi", "chi0", "kappa", "theta", "nu", "gamma0",
         "recovery", "corr")]


class _Portfolio(ctypes.Structure):
    _fields_ = [("n_swaps", ctypes.c_int),
                ("ccy", ctypes.POINTER(ctypes.c_int)), ("cpty", ctypes.POINTER(ctypes.c_int)),
                ("omega", ctypes.POINTER(ctypes.c_int)),
                ("n_periods", ctypes.POINTER(ctypes.c_int)),
                ("notional", ctypes.POINTER(ctypes.c_double)), ("delta", ctypes.c_double),
                ("fixed_rate", ctypes.POINTER(ctypes.c_double))]


class _Grid(ctypes.Structure):
    _fields_ = [("horizon", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("substeps", ctypes.c_int)]


class _Out(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in
                ("features", "I0", "Lambda", "mtm", "swap_pv")] + [
        ("idx", ctypes.POINTER(ctypes.c_uint16)),
        ("xi_bar", ctypes.POINTER(ctypes.c_double)),
        ("smooth", ctypes.POINTER(ctypes.c_double))]


def _load(path: str):
    L = ctypes.CDLL(path)
    L.oracle_simulate.restype = ctypes.c_int
    L.oracle_simulate.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Portfolio),
                                  ctypes.POINTER(_Grid), ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.POINTER(_Out)]
    L.oracle_simulate_copy.restype = ctypes.c_int
    L.oracle_simulate_copy.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Portfolio),
                                       ctypes.POINTER(_Grid), ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.POINTER(_Out)]
    L.oracle_exp_clocks_copy.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]
    L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
    L.oracle_uniform.restype = ctypes.c_double
    L.oracle_uniform.argtypes = [ctypes.c_uint32]
    L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.oracle_exp_clock.restype = ctypes.c_double
    L.oracle_exp_clock.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_int]
    L.oracle_exp_clocks.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.oracle_zc.restype = ctypes.c_double
    L.oracle_zc.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double]
    L.oracle_par_rate.restype = ctypes.c_double
    L.oracle_par_rate.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double]
    L.oracle_n_factors.restype = ctypes.c_int
    L.oracle_n_factors.argtypes = [ctypes.POINTER(_Model)]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


class use_library:
    """Context manager that points this module at another build of the oracle source
    (used by the tests that plant a mistake in a copy of the source)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def d(self, x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        self.refs.append(a)
        return _dp(a)

    def i(self, x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
        self.refs.append(a)
        return _ip(a)


def _model_struct(model, keep: _Keep) -> _Model:
    return _Model(model.E, model.C, keep.d(model.hw_a), keep.d(model.hw_sigma),
                  keep.d(model.curve), keep.d(model.fx_vol), keep.d(model.fx0),
                  keep.d(model.cir_kappa), keep.d(model.cir_theta), keep.d(model.cir_nu),
                  keep.d(model.gamma0), keep.d(model.recovery), keep.d(model.corr))


def _pf_struct(pf, keep: _Keep) -> _Portfolio:
    fr = getattr(pf, "fixed_rate", None)
    return _Portfolio(pf.n_swaps, keep.i(pf.ccy), keep.i(pf.cpty), keep.i(pf.omega),
                      keep.i(pf.n_periods), keep.d(pf.notional), float(pf.delta),
                      keep.d(fr) if fr is not None else ctypes.POINTER(ctypes.c_double)())


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 x uint32, key = 2 x uint32 -> 4 x uint32."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(o[i]) for i in range(4)]


def uniform(x: int) -> float:
    return float(lib().oracle_uniform(int(x) & 0xFFFFFFFF))


def normals(seed: int, k: int, q: int, F: int) -> np.ndarray:
    z = np.zeros(F)
    lib().oracle_normals(seed, k, q, F, _dp(z))
    return z


def exp_clock(seed: int, k: int, l: int, c: int) -> float:
    return float(lib().oracle_exp_clock(seed, k, l, c))


def exp_clocks(seed: int, k0: int, k1: int, N: int, C: int, copy: int = 0) -> np.ndarray:
    """Standard exponential clocks epsilon of every inner draw: [k1-k0, N, C] (of twin
    copy `copy` when >= 1)."""
    out = np.zeros((k1 - k0, N, C))
    lib().oracle_exp_clocks_copy(seed, k0, k1, N, C, copy, _dp(out))
    return out


def zc(model, e: int, t: float, T: float, r: float) -> float:
    keep = _Keep()
    m = _model_struct(model, keep)
    return float(lib().oracle_zc(ctypes.byref(m), e, t, T, r))


def par_rates(model, pf) -> np.ndarray:
    """Par fixed rate of every swap of a portfolio at t = 0 (App. B, P^sw_0 = 0)."""
    return np.array([par_rate(model, int(e), int(m), float(pf.delta)) for e, m in zip(pf.ccy, pf.n_periods)])


def par_rate(model, e: int, n_periods: int, delta: float) -> float:
    keep = _Keep()
    m = _model_struct(model, keep)
    return float(lib().oracle_par_rate(ctypes.byref(m), e, n_periods, delta))


def n_factors(model) -> int:
    keep = _Keep()
    m = _model_struct(model, keep)
    return int(lib().oracle_n_factors(ctypes.byref(m)))


def simulate(model, pf, grid, k0: int, k1: int, N: int, seed: int,
             want=("features", "I0", "Lambda", "mtm", "idx", "xi_bar"),
             n_threads: int = 0, copy=None) -> Dict[str, np.ndarray]:
    """Run the oracle on outer paths [k0, k1); return the requested arrays. With
    copy = (date, b) the run is twin copy b >= 1 branching at that pricing date.

    Shapes: features [n+1, F, M], I0 [n+1, M], Lambda [n+1, C, M], mtm [n+1, C, M],
    swap_pv [n+1, S, M], idx [M, N, C] (uint16; n+1 = no default), xi_bar [n, M],
    smooth [n, M].
    """
    n, C, M = grid.n_steps, model.C, k1 - k0
    F = n_factors(model)
    shapes = {"features": (n + 1, F, M), "I0": (n + 1, M), "Lambda": (n + 1, C, M),
              "mtm": (n + 1, C, M), "swap_pv": (n + 1, pf.n_swaps, M),
              "idx": (M, N, C), "xi_bar": (n, M), "smooth": (n, M)}
    res: Dict[str, np.ndarray] = {}
    ptrs = {}
    for key in ("features", "I0", "Lambda", "mtm", "swap_pv", "xi_bar", "smooth"):
        if key in want:
            res[key] = np.zeros(shapes[key])
            ptrs[key] = _dp(res[key])
        else:
            ptrs[key] = ctypes.POINTER(ctypes.c_double)()
    if "idx" in want:
        res["idx"] = np.zeros(shapes["idx"], dtype=np.uint16)
        idx_p = res["idx"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))
    else:
        idx_p = ctypes.POINTER(ctypes.c_uint16)()
    out = _Out(ptrs["features"], ptrs["I0"], ptrs["Lambda"], ptrs["mtm"], ptrs["swap_pv"],
               idx_p, ptrs["xi_bar"], ptrs["smooth"])
    keep = _Keep()
    m = _model_struct(model, keep)
    p = _pf_struct(pf, keep)
    g = _Grid(float(grid.horizon), int(grid.n_steps), int(grid.substeps))
    branch_date, b = (1 << 30, 0) if copy is None else (int(copy[0]), int(copy[1]))
    rc = lib().oracle_simulate_copy(ctypes.byref(m), ctypes.byref(p), ctypes.byref(g),
                                    k0, k1, N, seed, branch_date, b, n_threads, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"oracle_simulate failed with code {rc}")
    return res


def oversim_stats(o: Dict[str, np.ndarray], recovery: np.ndarray, pred: np.ndarray):
    """Q_i and R_i of Prop. 1 from the first two inner draws of every path (oracle
    outputs `idx`, `mtm`, `I0`; pred [n, M]): with the single-draw target
    xi^l_i = e^{I0_i} sum_c (1 - R_c) e^{-I0_j} MtM_c(j)^+ at j = idx_c^l if i < j <= n,
    and g_l = (xi^l_i - pred_i)^2, Q_i = mean(g^2) - mean(g_0 g_1) and
    R_i = mean(g_0 g_1) - mean(g)^2 (mean(g), mean(g^2) over both draws); dates 0
    and n are zero."""
    idx, mtm, I0 = o["idx"].astype(np.int64), o["mtm"], o["I0"]
    n1, C, M = mtm.shape
    n = n1 - 1
    V = (1.0 - np.asarray(recovery))[None, :, None] * np.exp(-I0)[:, None, :] * np.maximum(mtm, 0.0)  # [n+1, C, M]
    Q, R = np.zeros(n), np.zeros(n)
    kk = np.arange(M)
    for i in range(1, n):
        g = []
        for l in range(2):
            j = idx[:, l, :].T                                              # [C, M]
            v = np.where(j <= n, V[np.minimum(j, n), np.arange(C)[:, None], kk[None, :]], 0.0)
            xi = np.exp(I0[i]) * np.sum(np.where(j > i, v, 0.0), axis=0)
            g.append((xi - pred[i]) ** 2)
        m1 = 0.5 * (g[0].mean() + g[1].mean())
        m2 = 0.5 * ((g[0] ** 2).mean() + (g[1] ** 2).mean())
        m12 = (g[0] * g[1]).mean()
        Q[i], R[i] = m2 - m12, m12 - m1 * m1
    return Q, R


def draw_targets(o: Dict[str, np.ndarray], recovery: np.ndarray, date: int) -> np.ndarray:
    """The per-draw target xi_i^{k,l} at pricing date i (eq. (eq:CVA_portfolio) on one
    inner draw): e^{I0_i} sum_c (1 - R_c) e^{-I0_j} MtM_c(j)^+ with j = idx_c^{k,l},
    for the counterparties whose default step j satisfies i < j <= n. Oracle
    outputs `idx` [M, N, C], `mtm`, `I0`; returns [M, N]."""
    idx, mtm, I0 = o["idx"].astype(np.int64), o["mtm"], o["I0"]
    n1, C, M = mtm.shape
    n = n1 - 1
    V = (1.0 - np.asarray(recovery))[None, :, None] * np.exp(-I0)[:, None, :] * np.maximum(mtm, 0.0)
    kk = np.arange(M)[:, None, None]
    cc = np.arange(C)[None, None, :]
    v = V[np.minimum(idx, n), cc, kk]                          # [M, N, C]
    live = (idx > date) & (idx <= n)
    return np.exp(I0[date])[:, None] * np.sum(np.where(live, v, 0.0), axis=2)


def default_indicators(o: Dict[str, np.ndarray], date: int) -> np.ndarray:
    """X_i^{k,l}: 1 where counterparty c has defaulted by t_i (its default step is
    at most i), else 0; returns [M, N, C]."""
    return (o["idx"].astype(np.int64) <= date).astype(np.float64)


def alive_lsq(o: Dict[str, np.ndarray], recovery: np.ndarray, date: int, with_defaults: bool = True):
    """Least squares of the per-draw target on (X_i, Y_i) over the hierarchically
    simulated sample of size M N: one row per (outer path k, inner draw l) with
    Y^{k,l} = Y^k, the basis [1, z_1..z_F, X_1..X_C] (z the standardised state of
    `linear_features`), solved by Householder QR. Columns other than the intercept
    that are constant over the M N rows (a counterparty with no default by t_i, or
    a state component with no spread) are left out and get coefficient 0.
    with_defaults=False leaves out every X column (the Y-only learner).

    Returns a dict: w [1 + F + C] (the basis above), alive [M] = the fitted value
    at X = 0 (every counterparty alive), fitted [M, N], dropped (list of column
    indices left out)."""
    Y = o["features"][date]                                   # [F, M]
    F, M = Y.shape
    xi = draw_targets(o, recovery, date)                      # [M, N]
    N = xi.shape[1]
    X = default_indicators(o, date)                           # [M, N, C]
    C = X.shape[2]
    phiY = linear_features(Y)                                 # [M, 1 + F]
    rows = np.concatenate([np.repeat(phiY[:, None, :], N, axis=1), X], axis=2).reshape(M * N, 1 + F + C)
    if not with_defaults:
        rows[:, 1 + F:] = 0.0
    keep = [0] + [j for j in range(1, 1 + F + C) if np.ptp(rows[:, j]) > 0.0]
    w_keep, _ = lsq(rows[:, keep], xi.reshape(M * N))
    w = np.zeros(1 + F + C)
    w[keep] = w_keep
    fitted = (rows @ w).reshape(M, N)
    return {"w": w, "alive": phiY @ w[:1 + F], "fitted": fitted,
            "dropped": [j for j in range(1, 1 + F + C) if j not in keep]}


def twin_l2(phi: np.ndarray, xi1: np.ndarray, xi2: np.ndarray):
    """Twin Monte Carlo estimate of the L2 error E[(phi - E[xi | state])^2] (eq.
    (e:val1)): the mean over paths of phi^2 - (xi1 + xi2) phi + xi1 xi2, where xi1
    and xi2 are two copies of the target that are independent given the state phi
    is computed from; returns (estimate, standard error)."""
    f, a, b = (np.asarray(v, dtype=np.float64) for v in (phi, xi1, xi2))
    t = f * f - (a + b) * f + a * b
    se = float(t.std(ddof=1) / np.sqrt(t.size)) if t.size > 1 else 0.0
    return float(t.mean()), se


def cva0(xi_bar: np.ndarray):
    """CVA_0 = mean over outer paths of the averaged target at t_0, and its standard error."""
    x0 = np.asarray(xi_bar[0], dtype=np.float64)
    return float(x0.mean()), float(x0.std(ddof=1) / np.sqrt(x0.size)) if x0.size > 1 else 0.0


def poly2_features(y: np.ndarray) -> np.ndarray:
    """[1, z, z^2] with z the standardised short rate (mean 0, variance 1 over paths)."""
    sd = y.std()
    z = (y - y.mean()) / (sd if sd > 0 else 1.0)
    return np.stack([np.ones_like(z), z, z * z], axis=1)


def linear_features(Y: np.ndarray) -> np.ndarray:
    """[1, z_1, ..., z_F] with each factor standardised over paths. Y is [F, M]."""
    mu = Y.mean(axis=1, keepdims=True)
    sd = Y.std(axis=1, keepdims=True)
    sd[sd == 0] = 1.0
    Z = (Y - mu) / sd
    return np.concatenate([np.ones((1, Y.shape[1])), Z], axis=0).T


def lsq(phi: np.ndarray, xi: np.ndarray):
    """Least squares of eq. (e:forw) by Householder QR: w = argmin ||xi - phi w||.

    Returns (w, predictions phi w). phi is [M, m], xi is [M].
    """
    Q, R = np.linalg.qr(np.asarray(phi, dtype=np.float64), mode="reduced")
    w = np.linalg.solve(R, Q.T @ np.asarray(xi, dtype=np.float64))
    return w, phi @ w
