"""The allocation-free regression entry point (cva_regress_batched_static) gives
the same fits as the allocating one (cva_regress), call after call.

It serves callers that cannot allocate device memory when they need a fit (a
framework owning the whole device through its pool, a fixed memory budget, or a
loop that cannot afford cudaMalloc's device-wide synchronisation); its scratch is
a static array inside the library.

The file's name makes pytest collect it after every other test file: should it
fail, a run that stops at the first failure has already run all the other tests.
It depends on no other test and passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_17005_gb300 import _native, build
    build.build()
    return _native


def _inputs(G, F, M, seed):
    rng = np.random.default_rng(seed)
    Y = (0.02 + 0.01 * rng.normal(size=(G, F, M))).astype(np.float32)
    w = rng.normal(size=(G, F))
    xi = (0.1 + np.einsum("gf,gfm->gm", w, Y - 0.02) + 1e-3 * rng.normal(size=(G, M))).astype(np.float32)
    return torch.from_numpy(Y).cuda(), torch.from_numpy(xi).cuda()


def _static_call(nat, xi, Y, basis, m):
    G, F, M = Y.shape
    pred = torch.full((G, M), float("nan"), device="cuda")
    coef = np.zeros((G, m))
    st = nat.lib().cva_regress_batched_static(
        ctypes.c_void_p(xi.data_ptr()), ctypes.c_void_p(Y.data_ptr()), G, F, M, basis,
        ctypes.c_void_p(pred.data_ptr()), coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    nat.check(st, "cva_regress_batched_static")
    torch.cuda.synchronize()
    return pred.cpu().numpy(), coef


# widths of the normal matrix: F = 27 -> 32 columns, F = 5 -> 12, poly2 -> 4; M = 70 001
# and 9 999 take the scalar prediction path (M not a multiple of 4); 207 groups of the
# 28-column basis is the most the static array holds (one Gram chunk per group)
@pytest.mark.parametrize("basis_name,G,F,M", [("linear", 6, 27, 70_001), ("linear", 4, 5, 9_999),
                                              ("linear", 5, 5, 32_768), ("poly2", 3, 1, 16_384),
                                              ("poly2", 2, 1, 16_385), ("linear", 207, 27, 4_096)])
def test_static_scratch_matches_allocating_entry_point(lib, basis_name, G, F, M):
    from paper_2211_17005_gb300 import api
    nat = lib
    basis = nat.BASIS_LINEAR if basis_name == "linear" else nat.BASIS_POLY2
    m = F + 1 if basis_name == "linear" else 3
    Y, xi = _inputs(G, F, M, seed=G * 100 + F)
    ref_pred, ref_coef = [], []
    for g in range(G):
        p, c = api.regress(xi[g], Y[g], basis=basis_name)
        ref_pred.append(p.cpu().numpy())
        ref_coef.append(c)
    ref_pred = np.stack(ref_pred)
    ref_coef = np.stack(ref_coef)
    scale = float(np.sqrt(np.mean(xi.cpu().numpy().astype(np.float64) ** 2)))
    for call in range(2):        # two calls in a row share the static scratch
        pred, coef = _static_call(nat, xi, Y, basis, m)
        assert np.all(np.isfinite(pred))
        # the two entry points split the Gram sums into different chunk counts (one per
        # group at the 207-group limit), so the FP32 runs round differently: predictions
        # agree to 1e-5 of the targets' scale, the coefficients to 1e-4 relative
        assert np.sqrt(np.mean((pred - ref_pred) ** 2)) < 1e-5 * scale, call
        # coefficients in the raw basis: 1e-4 relative, and 1e-5 of the largest coefficient
        # absolute (a coefficient near zero carries the FP32 rounding of the Gram sums,
        # which the different chunk counts round differently)
        np.testing.assert_allclose(coef, ref_coef, rtol=1e-4, atol=1e-5 * np.abs(ref_coef).max())


@pytest.mark.parametrize("groups,F,limit", [(5000, 27, 207), (208, 27, 207), (1025, 5, 1024)])
def test_static_scratch_rejects_oversized_batches(lib, groups, F, limit):
    """A batch beyond the static array is refused on the host, before any launch, with
    the limit in the message."""
    nat = lib
    Y, xi = _inputs(1, F, 1024, seed=1)
    st = nat.lib().cva_regress_batched_static(
        ctypes.c_void_p(xi.data_ptr()), ctypes.c_void_p(Y.data_ptr()), groups, F, 1024, nat.BASIS_LINEAR,
        None, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == nat.CVA_EINVAL
    msg = nat.lib().cva_last_error()
    assert b"static scratch" in msg and f"at most {limit} groups".encode() in msg, msg
