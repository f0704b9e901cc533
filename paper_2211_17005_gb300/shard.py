"""Outer paths split over processes, one per GPU (torch.distributed).

Every rank simulates its own range of global outer paths (cva_simulate's k0: the
generator's counters are keyed by the global path index, so the ranges together
are exactly the paths of one large run). The data path needs no exchange; the
estimators that pool all paths combine FP64 partial sums once:

* CVA_0 and its standard error from every rank's (M, sum xi0, sum xi0^2);
* each least-squares fit of eq. (e:forw) from every rank's augmented normal matrix,
  accumulated with a centring state all ranks share, solved once and applied by
  every rank to its own paths.

The sum over ranks is taken in rank order on every rank (all_gather, then a
fixed-order sum on the host), so all ranks hold the same bits whatever reduction
tree the backend would use. Only marshalling and the exchange live here; the
partial sums, the combination and the solve run in the C library.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np
import torch
import torch.distributed as dist

from . import _native as nat

_dp = ctypes.POINTER(ctypes.c_double)


def path_range(M_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(k0, M) of rank's contiguous share of M_total global outer paths."""
    lo = (M_total * rank) // world
    hi = (M_total * (rank + 1)) // world
    return lo, hi - lo


def gather_rank_order(x: np.ndarray, group=None) -> np.ndarray:
    """Every rank's FP64 array, stacked in rank order ([world, ...]) on every rank."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return np.stack([o.cpu().numpy() for o in out])


def sum_rank_order(x: np.ndarray, group=None) -> np.ndarray:
    """The sum over ranks of an FP64 array, added in rank order (same bits on every rank)."""
    parts = gather_rank_order(x, group)
    s = parts[0].copy()
    for p in parts[1:]:
        s = s + p
    return s


def combine_cva0(parts: np.ndarray) -> Tuple[float, float]:
    """CVA_0 and its standard error from (M, sum, sum of squares) triples [n, 3]."""
    p = np.ascontiguousarray(parts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(2)
    nat.check(nat.lib().cva_cva0_combine(p.ctypes.data_as(_dp), p.shape[0], out.ctypes.data_as(_dp)),
              "cva_cva0_combine")
    return float(out[0]), float(out[1])


def solve(gram: np.ndarray, F: int, basis: int, centre: np.ndarray):
    """The fit of a summed augmented normal matrix (host only): (coefficients in the
    centred basis, in the raw basis, number of dropped columns)."""
    m = 3 if basis == nat.BASIS_POLY2 else F + 1
    g = np.ascontiguousarray(gram, dtype=np.float64)
    assert g.shape == (m + 1, m + 1)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    wc, wr, nd = np.zeros(m), np.zeros(m), ctypes.c_int()
    nat.check(nat.lib().cva_regress_solve(g.ctypes.data_as(_dp), F, basis, c.ctypes.data_as(_dp),
                                          wc.ctypes.data_as(_dp), wr.ctypes.data_as(_dp), ctypes.byref(nd)),
              "cva_regress_solve")
    return wc, wr, int(nd.value)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _distributed() -> bool:
    return dist.is_available() and dist.is_initialized()


def cva0_partial(xi0: torch.Tensor, stream=None) -> np.ndarray:
    """(M, sum, sum of squares) of this rank's date-0 targets (device float [M])."""
    assert xi0.is_cuda and xi0.dtype == torch.float32 and xi0.is_contiguous()
    part = np.zeros(3)
    nat.check(nat.lib().cva_cva0_partials(ctypes.c_void_p(xi0.data_ptr()), xi0.numel(), part.ctypes.data_as(_dp),
                                          _stream(stream)), "cva_cva0_partials")
    return part


def cva0(xi0: torch.Tensor, group=None, stream=None) -> Tuple[float, float]:
    """CVA_0 and its standard error over the paths of every rank (xi0: this rank's
    date-0 targets); without a process group, over this process's paths."""
    part = cva0_partial(xi0, stream)
    return combine_cva0(gather_rank_order(part, group) if _distributed() else part[None])


def regress_partial(targets: torch.Tensor, features: torch.Tensor, centre: torch.Tensor, basis: str = "linear",
                    stream=None) -> np.ndarray:
    """This rank's augmented normal matrix ((m+1) x (m+1), FP64) of the basis centred on
    `centre` (device float [F]; [1] for poly2)."""
    b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
    F, M = features.shape
    m = 3 if b == nat.BASIS_POLY2 else F + 1
    for t in (targets, features, centre):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    gram = np.zeros((m + 1, m + 1))
    nat.check(nat.lib().cva_regress_partial(ctypes.c_void_p(targets.data_ptr()), ctypes.c_void_p(features.data_ptr()),
                                            F, M, b, ctypes.c_void_p(centre.data_ptr()), gram.ctypes.data_as(_dp),
                                            _stream(stream)), "cva_regress_partial")
    return gram


def regress_predict(features: torch.Tensor, centre: torch.Tensor, coef_centred: np.ndarray, basis: str = "linear",
                    pred: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """phi(Y_k) . w on this rank's paths for centred coefficients w (device float [M])."""
    b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
    F, M = features.shape
    w = np.ascontiguousarray(coef_centred, dtype=np.float64)
    if pred is None:
        pred = torch.empty(M, dtype=torch.float32, device=features.device)
    nat.check(nat.lib().cva_regress_predict(ctypes.c_void_p(features.data_ptr()), F, M, b,
                                            ctypes.c_void_p(centre.data_ptr()), w.ctypes.data_as(_dp),
                                            ctypes.c_void_p(pred.data_ptr()), _stream(stream)), "cva_regress_predict")
    return pred


def regress(targets: torch.Tensor, features: torch.Tensor, centre: torch.Tensor, basis: str = "linear",
            group=None, stream=None, pred: Optional[torch.Tensor] = None):
    """Least squares of eq. (e:forw) over the paths of every rank (targets [M], features
    [F, M]: this rank's paths; centre: the same state on every rank). Returns (this
    rank's predictions [M], raw-basis coefficients, number of dropped columns)."""
    b = nat.BASIS_POLY2 if basis == "poly2" else nat.BASIS_LINEAR
    gram = regress_partial(targets, features, centre, basis, stream)
    gsum = sum_rank_order(gram, group) if _distributed() else gram
    wc, wr, nd = solve(gsum, features.shape[0], b, centre.detach().cpu().numpy().astype(np.float64))
    return regress_predict(features, centre, wc, basis, pred, stream), wr, nd
