"""Python face of the C ABI: torch tensors in, torch tensors out.

Only argument marshalling lives here; every step of the method runs in the CUDA
library. Device memory of a simulation is owned by the library and exposed as
borrowed torch tensors (``__cuda_array_interface__``), valid while the
``Simulation`` object is alive.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _native as nat

_F32, _U8 = "<f4", "|u1"


class _Keep:
    def __init__(self):
        self.refs = []

    def d(self, x) -> ctypes.POINTER(ctypes.c_double):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        self.refs.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def i(self, x) -> ctypes.POINTER(ctypes.c_int32):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
        self.refs.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def model_desc(model, keep: _Keep) -> nat.ModelDesc:
    return nat.ModelDesc(model.E, model.C, keep.d(model.hw_a), keep.d(model.hw_sigma), keep.d(model.curve),
                       keep.d(model.fx_vol), keep.d(model.fx0), keep.d(model.cir_kappa),
                       keep.d(model.cir_theta), keep.d(model.cir_nu), keep.d(model.gamma0),
                       keep.d(model.recovery), keep.d(model.corr))


def portfolio_desc(pf, keep: _Keep) -> nat.PortfolioDesc:
    fr = getattr(pf, "fixed_rate", None)
    return nat.PortfolioDesc(pf.n_swaps, keep.i(pf.ccy), keep.i(pf.cpty), keep.i(pf.omega),
                             keep.i(pf.n_periods), keep.d(pf.notional), float(pf.delta),
                             keep.d(fr) if fr is not None else ctypes.POINTER(ctypes.c_double)())


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _DevArray:
    """Minimal __cuda_array_interface__ carrier for a borrowed device buffer."""

    def __init__(self, ptr: int, shape: Tuple[int, ...], typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2, "strides": None,
                                         "stream": None}


class Simulation:
    """M outer paths x N inner defaults of the hierarchical scheme (Sec. 3.2) for one
    model, grid and up to 6 portfolios; device buffers are allocated once."""

    def __init__(self, model, portfolios: Sequence, grid, M: int, N: int,
                 keep_defaults: bool = False, keep_exposures: bool = False, profile: bool = False,
                 generic: bool = False):
        L = N_lib()
        keep = _Keep()
        md = model_desc(model, keep)
        pds = (nat.PortfolioDesc * len(portfolios))(*[portfolio_desc(p, keep) for p in portfolios])
        gd = nat.GridDesc(float(grid.horizon), int(grid.n_steps), int(grid.substeps))
        flags = ((nat.KEEP_DEFAULTS if keep_defaults else 0) | (nat.KEEP_EXPOSURES if keep_exposures else 0)
                 | (nat.PROFILE if profile else 0) | (nat.GENERIC_KERNELS if generic else 0))
        h = ctypes.c_void_p()
        nat.check(L.cva_sim_create(ctypes.byref(md), pds, len(portfolios), ctypes.byref(gd), int(M), int(N),
                                 flags, ctypes.byref(h)), "cva_sim_create")
        self._h = h
        shp = (ctypes.c_int64 * 6)()
        nat.check(L.cva_sim_shape(h, shp), "cva_sim_shape")
        self.M, self.N, self.n, self.F, self.C, self.n_pf = (int(x) for x in shp)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            N_lib().cva_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seed: int, k0: int = 0, stream: Optional[torch.cuda.Stream] = None):
        """Enqueue the outer-path and inner-default kernels for paths [k0, k0+M)."""
        nat.check(N_lib().cva_simulate(self._h, int(seed), int(k0), _stream_handle(stream)), "cva_simulate")
        return self

    def run_twin(self, seed: int, date: int, copy: int, k0: int = 0, stream: Optional[torch.cuda.Stream] = None):
        """Run the simulation as twin copy `copy` (>= 1) branching at pricing date `date`
        (twin Monte Carlo validation); its targets of that date are one conditionally
        independent copy of the target given the state at t_date."""
        nat.check(N_lib().cva_simulate_twin(self._h, int(seed), int(k0), int(date), int(copy),
                                            _stream_handle(stream)), "cva_simulate_twin")
        return self

    def nested_reference(self, seed: int, date: int, copies: int, pf: int = 0, k0: int = 0,
                         stream=None) -> torch.Tensor:
        """Nested Monte Carlo reference of the conditional CVA at `date` for every path:
        the mean of `copies` twin copies' targets (device float [M]). Overwrites the
        simulation's buffers (the last copy stays)."""
        out = torch.empty(self.M, dtype=torch.float32, device=self.device)
        nat.check(N_lib().cva_nested_reference(self._h, int(seed), int(k0), pf, int(date), int(copies),
                                               ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
                  "cva_nested_reference")
        return out

    def oversim_stats(self, pred: torch.Tensor, seed: int, pf: int = 0, stream=None):
        """Q_i and R_i of Prop. 1 per date (numpy [n] each) for the regression `pred`
        ([n, M] device float) of the simulation run with key `seed`."""
        assert pred.is_cuda and pred.dtype == torch.float32 and pred.is_contiguous()
        assert pred.shape == (self.n, self.M) and self.N >= 2
        out = np.zeros((self.n, 2))
        nat.check(N_lib().cva_oversim_stats(self._h, pf, ctypes.c_void_p(pred.data_ptr()), int(seed),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            _stream_handle(stream)), "cva_oversim_stats")
        return out[:, 0], out[:, 1]

    def kernel_ms(self) -> Tuple[float, float, float]:
        """(path simulation, pricing, inner defaults) device milliseconds of the last run."""
        out = (ctypes.c_float * 3)()
        nat.check(N_lib().cva_sim_kernel_ms(self._h, out), "cva_sim_kernel_ms")
        return float(out[0]), float(out[1]), float(out[2])

    def _view(self, what: int, shape, typestr=_F32) -> torch.Tensor:
        p = ctypes.c_void_p()
        b = ctypes.c_size_t()
        nat.check(N_lib().cva_sim_view(self._h, what, ctypes.byref(p), ctypes.byref(b)), "cva_sim_view")
        t = torch.as_tensor(_DevArray(p.value, shape, typestr), device=self.device)
        t._cva_owner = self          # keep the simulation alive while the view is
        return t

    def features(self):
        return self._view(nat.VIEW_FEATURES, (self.n + 1, self.F, self.M))

    def targets(self):
        return self._view(nat.VIEW_TARGETS, (self.n_pf, self.n, self.M))

    def discount_integral(self):
        return self._view(nat.VIEW_DISCOUNT, (self.n + 1, self.M))

    def thresholds(self):
        return self._view(nat.VIEW_THRESHOLD, (self.n + 1, self.C, self.M))

    def exposures(self):
        return self._view(nat.VIEW_EXPOSURE, (self.n_pf, self.n + 1, self.C, self.M))

    def mtm(self):
        return self._view(nat.VIEW_MTM, (self.n_pf, self.n + 1, self.C, self.M))

    def defaults(self):
        return self._view(nat.VIEW_DEFAULTS, (self.M, self.N, self.C), _U8)

    def cva0(self, pf: int = 0, stream=None) -> Tuple[float, float]:
        return cva0(self.targets()[pf, 0], stream=stream)

    def regress_portfolios(self, basis: str = "linear", pred: Optional[torch.Tensor] = None, stream=None,
                           want_coef: bool = False):
        """Least squares at every date 1..n-1 for every portfolio in one grouped launch;
        returns (predictions [n_pf, n, M] on the device, coefficients [n_pf, n, m] or None)."""
        b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
        m = 3 if b == nat.BASIS_POLY2 else self.F + 1
        if pred is None:
            pred = torch.zeros((self.n_pf, self.n, self.M), dtype=torch.float32, device=self.device)
        coef = np.zeros((self.n_pf, self.n, m)) if want_coef else None
        cp = coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_coef else None
        nat.check(N_lib().cva_regress_portfolios(self._h, b, ctypes.c_void_p(pred.data_ptr()), cp,
                                                 _stream_handle(stream)), "cva_regress_portfolios")
        return pred, coef

    def regress_alive(self, pf: int = 0, pred: Optional[torch.Tensor] = None, stream=None,
                      want_coef: bool = True):
        """Least squares on (default indicators X_i, state Y_i) over the M N
        hierarchical sample at every date 1..n-1 (see cva_regress_alive); the
        simulation must keep its default steps (keep_defaults=True). Returns
        (the fit at X = 0 [n, M] on the device, coefficients [n, 1+F+C] in the raw
        basis [1, Y, X] or None, dropped columns per date [n] or None)."""
        if pred is None:
            pred = torch.zeros((self.n, self.M), dtype=torch.float32, device=self.device)
        m = self.F + 1 + self.C
        coef = np.zeros((self.n, m)) if want_coef else None
        dropped = np.zeros(self.n, dtype=np.int32) if want_coef else None
        cp = coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_coef else None
        dp = dropped.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if want_coef else None
        nat.check(N_lib().cva_regress_alive(self._h, int(pf), ctypes.c_void_p(pred.data_ptr()), cp, dp,
                                            _stream_handle(stream)), "cva_regress_alive")
        return pred, coef, dropped

    def autotune(self, seed: int = 1, basis: str = "linear", stream=None) -> dict:
        """Pick the tile shapes by measurement (see cva_autotune); returns the choice."""
        import json
        buf = ctypes.create_string_buffer(512)
        b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
        nat.check(N_lib().cva_autotune(self._h, int(seed), b, buf, 512, _stream_handle(stream)), "cva_autotune")
        return json.loads(buf.value.decode())

    def set_tiles(self, sim_block: int, price_block: int, inner_paths_per_block: int, lsq_chunk_target: int,
                  portfolios_per_price_block: int = 1) -> None:
        """Set the tile shapes directly (see cva_set_tiles), e.g. a saved autotune choice."""
        nat.check(N_lib().cva_set_tiles(self._h, int(sim_block), int(price_block), int(inner_paths_per_block),
                                        int(lsq_chunk_target), int(portfolios_per_price_block)), "cva_set_tiles")

    def regress_all(self, pf: int = 0, basis: str = "poly2", stream=None, want_coef: bool = True):
        """Least squares at every date 1..n-1 in one grouped launch; returns
        (predictions [n, M] on the device, coefficients [n, m] numpy or None)."""
        b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
        m = 3 if b == nat.BASIS_POLY2 else self.F + 1
        pred = torch.zeros((self.n, self.M), dtype=torch.float32, device=self.device)
        coef = np.zeros((self.n, m)) if want_coef else None
        cp = coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_coef else None
        nat.check(N_lib().cva_regress_all(self._h, pf, b, ctypes.c_void_p(pred.data_ptr()), cp,
                                        _stream_handle(stream)), "cva_regress_all")
        return pred, coef


def N_lib():
    return nat.lib()


def cva0(xi0: torch.Tensor, stream=None) -> Tuple[float, float]:
    """CVA_0 and its standard error from the date-0 targets (device float tensor [M])."""
    assert xi0.is_cuda and xi0.dtype == torch.float32 and xi0.is_contiguous()
    out = np.zeros(2)
    nat.check(N_lib().cva_cva0(ctypes.c_void_p(xi0.data_ptr()), xi0.numel(),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_handle(stream)),
            "cva_cva0")
    return float(out[0]), float(out[1])


def relative_rmse(phi: torch.Tensor, ref: torch.Tensor, stream=None) -> Tuple[float, int]:
    """sqrt(mean((phi - ref)^2 / ref^2)) over the paths where ref != 0, and their number."""
    for t in (phi, ref):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == phi.numel()
    out = np.zeros(2)
    nat.check(N_lib().cva_relative_rmse(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(ref.data_ptr()),
                                        phi.numel(), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        _stream_handle(stream)), "cva_relative_rmse")
    return float(out[0]), int(out[1])


def inner_cost_ratio(t1: float, N1: int, t2: float, N2: int) -> float:
    """The cost kappa of an outer path in units of inner draws from two timings at the
    same M (see cva_inner_cost_ratio)."""
    k = ctypes.c_double()
    nat.check(N_lib().cva_inner_cost_ratio(float(t1), int(N1), float(t2), int(N2), ctypes.byref(k)),
              "cva_inner_cost_ratio")
    return float(k.value)


def oversimulation_choice(Q, R, kappa: float, budget: Optional[float] = None):
    """Prop. 1 and Heuristic 1 (see cva_oversim_choice): (N_i per date, N, M or None)."""
    qr = np.ascontiguousarray(np.stack([np.asarray(Q, dtype=np.float64), np.asarray(R, dtype=np.float64)], axis=1))
    n = qr.shape[0]
    Ni = np.zeros(n)
    N, M = ctypes.c_double(), ctypes.c_double()
    _dp = ctypes.POINTER(ctypes.c_double)
    nat.check(N_lib().cva_oversim_choice(qr.ctypes.data_as(_dp), n, float(kappa),
                                         float(budget) if budget is not None else 0.0, Ni.ctypes.data_as(_dp),
                                         ctypes.byref(N), ctypes.byref(M)), "cva_oversim_choice")
    return Ni, float(N.value), (float(M.value) if budget is not None else None)


def twin_l2(phi: torch.Tensor, xi1: torch.Tensor, xi2: torch.Tensor, stream=None) -> Tuple[float, float]:
    """Twin estimate of the L2 error of phi (eq. (e:val1)) from two conditionally
    independent copies of the target, with its standard error (device float [M] each)."""
    for t in (phi, xi1, xi2):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == phi.numel()
    out = np.zeros(2)
    nat.check(N_lib().cva_twin_l2(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(xi1.data_ptr()),
                                  ctypes.c_void_p(xi2.data_ptr()), phi.numel(),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_handle(stream)),
              "cva_twin_l2")
    return float(out[0]), float(out[1])


def regress(targets: torch.Tensor, features: torch.Tensor, basis: str = "linear",
            want_pred: bool = True, want_coef: bool = True, stream=None):
    """Least squares of eq. (e:forw) at one date: targets [M], features [F, M] (device
    float tensors). Returns (predictions [M] or None, raw-basis coefficients or None)."""
    assert targets.is_cuda and features.is_cuda
    assert targets.dtype == torch.float32 and features.dtype == torch.float32
    targets = targets.contiguous()
    features = features.contiguous()
    F, M = features.shape
    b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
    m = 3 if b == nat.BASIS_POLY2 else F + 1
    pred = torch.empty(M, dtype=torch.float32, device=targets.device) if want_pred else None
    coef = np.zeros(m) if want_coef else None
    nat.check(N_lib().cva_regress(ctypes.c_void_p(targets.data_ptr()), ctypes.c_void_p(features.data_ptr()), F, M,
                                b, ctypes.c_void_p(pred.data_ptr()) if want_pred else None,
                                coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_coef else None,
                                _stream_handle(stream)), "cva_regress")
    return pred, coef


def pipe_peaks(stream=None) -> dict:
    """Measured lane-operations per second of the SMs' FMA, ALU, integer multiply-high
    and MUFU pipes (see cva_pipe_peaks)."""
    out = np.zeros(5)
    nat.check(N_lib().cva_pipe_peaks(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_handle(stream)),
              "cva_pipe_peaks")
    return dict(zip(("fma_f32", "lop3_b32", "mul_hi_u32", "ex2_f32", "lg2_f32"), (float(x) for x in out)))


def philox4x32_10(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Philox4x32-10 blocks of the counters ctr (device int32/uint32 tensor [n, 4])."""
    assert ctr.is_cuda and ctr.shape[-1] == 4 and ctr.element_size() == 4
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    nat.check(N_lib().cva_philox4x32_10(ctypes.c_void_p(ctr.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctr.numel() // 4, int(seed), _stream_handle(stream)), "cva_philox4x32_10")
    return out


# ---------------------------------------------------------------- MLP ------

MLP_IN = 32


def mlp_num_params(hidden: int) -> int:
    return int(N_lib().cva_mlp_num_params(hidden))


def mlp_plan(M: int, hidden: int = 64, n_batches: int = 32) -> dict:
    """Launch shape of the trainer for M paths in n_batches batches (see cva_mlp_plan)."""
    out = (ctypes.c_int32 * 4)()
    nat.check(N_lib().cva_mlp_plan(int(M), int(hidden), int(n_batches), out), "cva_mlp_plan")
    return {"ctas": int(out[0]), "cluster": int(out[1]), "tiles_per_batch": int(out[2]), "rounds": int(out[3])}


def mlp_kernel_timing(on: bool) -> dict:
    """Switch the trainers' per-launch event timing on or off; returns the totals
    accumulated since the previous call (see cva_mlp_kernel_timing)."""
    ms, n = ctypes.c_double(0.0), ctypes.c_uint64(0)
    nat.check(N_lib().cva_mlp_kernel_timing(1 if on else 0, ctypes.byref(ms), ctypes.byref(n)),
              "cva_mlp_kernel_timing")
    return {"ms": float(ms.value), "launches": int(n.value)}


def mlp_pack(p, hidden: int) -> torch.Tensor:
    """Flat device parameter vector from a dict (W1 [u, d<=32], b1, W2, b2, w3, b3, mu)."""
    W1 = np.zeros((hidden, MLP_IN))
    W1[:, :p["W1"].shape[1]] = p["W1"]
    flat = np.concatenate([W1.ravel(), np.ravel(p["b1"]), np.ravel(p["W2"]), np.ravel(p["b2"]),
                           np.ravel(p["w3"]), [float(p["b3"])], [float(p["mu"])]]).astype(np.float32)
    assert flat.size == mlp_num_params(hidden)
    return torch.from_numpy(flat).cuda()


def mlp_unpack(flat: torch.Tensor, hidden: int, d: int):
    v = flat.detach().cpu().numpy().astype(np.float64)
    u = hidden
    o = 0
    W1 = v[o:o + u * MLP_IN].reshape(u, MLP_IN)[:, :d]; o += u * MLP_IN
    b1 = v[o:o + u]; o += u
    W2 = v[o:o + u * u].reshape(u, u); o += u * u
    b2 = v[o:o + u]; o += u
    w3 = v[o:o + u]; o += u
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "w3": w3, "b3": np.array(v[o]), "mu": np.array(v[o + 1])}


def mlp_fit(targets: torch.Tensor, features: torch.Tensor, params: torch.Tensor, hidden: int = 64,
            n_batches: int = 32, epochs: int = 8, lr: float = 1e-3, want_pred: bool = True, stream=None):
    """Algorithm 1 at one date on device tensors (targets [M], features [F, M]); params is
    updated in place to the best parameters. Returns (predictions [M] or None, losses [epochs])."""
    F, M = features.shape
    pred = torch.empty(M, dtype=torch.float32, device=targets.device) if want_pred else None
    losses = torch.empty(epochs, dtype=torch.float32, device=targets.device)
    nat.check(N_lib().cva_mlp_fit(ctypes.c_void_p(targets.data_ptr()), ctypes.c_void_p(features.data_ptr()), F, M,
                                  hidden, n_batches, epochs, float(lr), ctypes.c_void_p(params.data_ptr()),
                                  ctypes.c_void_p(pred.data_ptr()) if want_pred else None,
                                  ctypes.c_void_p(losses.data_ptr()), _stream_handle(stream)), "cva_mlp_fit")
    return pred, losses.cpu().numpy()


def mlp_first_gradient(targets, features, params, hidden=64, n_batches=32, lr=1e-3, stream=None):
    F, M = features.shape
    grad = torch.empty_like(params)
    nat.check(N_lib().cva_mlp_first_gradient(ctypes.c_void_p(targets.data_ptr()),
                                             ctypes.c_void_p(features.data_ptr()), F, M, hidden, n_batches,
                                             float(lr), ctypes.c_void_p(params.data_ptr()),
                                             ctypes.c_void_p(grad.data_ptr()), _stream_handle(stream)),
              "cva_mlp_first_gradient")
    return grad


def mlp_regress_all(sim: "Simulation", params: torch.Tensor, pf: int = 0, hidden: int = 64, n_batches: int = 32,
                    epochs: int = 8, lr: float = 1e-3, stream=None) -> torch.Tensor:
    """Algorithm 2 over every date n-1..1 of a simulation; returns predictions [n, M]."""
    pred = torch.zeros((sim.n, sim.M), dtype=torch.float32, device=sim.device)
    nat.check(N_lib().cva_mlp_regress_all(sim._h, pf, hidden, n_batches, epochs, float(lr),
                                          ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(pred.data_ptr()),
                                          _stream_handle(stream)), "cva_mlp_regress_all")
    return pred


# ------------------------------------------------------------ adjoint ------

def par_rates(model, pf) -> np.ndarray:
    """The par fixed rates at t = 0 the library uses for `pf` under `model`."""
    keep = _Keep()
    out = np.zeros(pf.n_swaps)
    nat.check(N_lib().cva_par_rates(ctypes.byref(model_desc(model, keep)), ctypes.byref(portfolio_desc(pf, keep)),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "cva_par_rates")
    return out


def frozen(model, pf):
    """A copy of `pf` whose fixed rates are the par rates under `model` (trade terms that
    do not move when the model's parameters are bumped)."""
    import dataclasses
    return dataclasses.replace(pf, fixed_rate=par_rates(model, pf))


def grad_params(model) -> np.ndarray:
    """theta in the order of cva_grad_cva0: f (E), sigma^r (E), sigma^chi_1..E-1, kappa, theta, nu (C each)."""
    return np.concatenate([model.curve, model.hw_sigma, model.fx_vol[1:], model.cir_kappa, model.cir_theta,
                           model.cir_nu]).astype(np.float64)


def with_params(model, theta) -> "object":
    """A copy of `model` with the parameters of grad_params replaced by theta."""
    import dataclasses
    E, C = model.E, model.C
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    curve = t[o:o + E].copy(); o += E
    hw_sigma = t[o:o + E].copy(); o += E
    fx_vol = np.concatenate([[model.fx_vol[0]], t[o:o + E - 1]]); o += E - 1
    kappa = t[o:o + C].copy(); o += C
    theta_c = t[o:o + C].copy(); o += C
    nu = t[o:o + C].copy()
    return dataclasses.replace(model, curve=curve, hw_sigma=hw_sigma, fx_vol=fx_vol, cir_kappa=kappa,
                               cir_theta=theta_c, cir_nu=nu)


def grad_cva0(model, pf, grid, M: int, seed: int = 1, k0: int = 0, ckpt_every: int = 10,
              forward_only: bool = False, stream=None):
    """(smooth CVA_0, dCVA_0/dtheta or None) by the adjoint kernel; see cva_grad_cva0."""
    keep = _Keep()
    md = model_desc(model, keep)
    pd = portfolio_desc(pf, keep)
    gd = nat.GridDesc(float(grid.horizon), int(grid.n_steps), int(grid.substeps))
    npar = int(N_lib().cva_grad_num_params(model.E, model.C))
    g = np.zeros(npar)
    c0 = ctypes.c_double()
    nat.check(N_lib().cva_grad_cva0(ctypes.byref(md), ctypes.byref(pd), ctypes.byref(gd), int(M), int(seed), int(k0),
                                    int(ckpt_every), 1 if forward_only else 0,
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(c0),
                                    _stream_handle(stream)), "cva_grad_cva0")
    return float(c0.value), (None if forward_only else g)


class SmoothCVA0(torch.autograd.Function):
    """CVA_0 (smooth form) as a function of theta = grad_params(model); backward returns
    the adjoint sensitivities. Usage: SmoothCVA0.apply(theta, model, portfolio, grid, M, seed)."""

    @staticmethod
    def forward(ctx, theta, model, pf, grid, M, seed):
        m = with_params(model, theta.detach().cpu().numpy())
        c0, g = grad_cva0(m, pf, grid, M, seed)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(c0, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None
