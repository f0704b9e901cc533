"""The C-ABI library loads and exports every entry point include/cva.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cva.h")).read()
    return sorted(set(re.findall(r"CVA_API\s+[\w\s\*]+?\b(cva_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libcva():
    from paper_2211_17005_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("cva_sim_create", "cva_simulate", "cva_cva0", "cva_regress", "cva_regress_all",
                 "cva_sim_view", "cva_sim_destroy", "cva_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(libcva):
    for name in declared_symbols():
        assert hasattr(libcva, name), name


def test_binding_signatures_cover_the_header():
    from paper_2211_17005_gb300 import _native
    assert sorted(_native.SIGNATURES) == declared_symbols()


def test_version_string(libcva):
    libcva.cva_version.restype = ctypes.c_char_p
    assert libcva.cva_version().startswith(b"sm_103a")


def test_invalid_inputs_are_rejected_on_the_host(libcva):
    """Validation happens before any device call: bad shapes return CVA_EINVAL."""
    import numpy as np
    from paper_2211_17005_gb300 import _native as N, api, workload as W
    L = N.lib()
    wl = W.make("small", M=64)
    keep = api._Keep()
    md = api.model_desc(wl.model, keep)
    pd = (N.PortfolioDesc * 1)(api.portfolio_desc(wl.portfolios[0], keep))
    h = ctypes.c_void_p()
    bad_grid = N.GridDesc(5.0, 0, 1)
    assert L.cva_sim_create(ctypes.byref(md), pd, 1, ctypes.byref(bad_grid), 64, 8, 0, ctypes.byref(h)) == N.CVA_EINVAL
    assert b"grid" in L.cva_last_error()
    g = N.GridDesc(5.0, 50, 1)
    assert L.cva_sim_create(ctypes.byref(md), pd, 1, ctypes.byref(g), 0, 8, 0, ctypes.byref(h)) == N.CVA_EINVAL
    assert L.cva_sim_create(ctypes.byref(md), pd, 1, ctypes.byref(g), 64, 0, 0, ctypes.byref(h)) == N.CVA_EINVAL
    # non-SPD correlation
    m2 = W.paper_model(np.random.default_rng(0))
    m2.corr = m2.corr.copy()
    m2.corr[0, 1] = m2.corr[1, 0] = 1.0
    m2.corr[0, 2] = m2.corr[2, 0] = -1.0
    md2 = api.model_desc(m2, keep)
    assert L.cva_sim_create(ctypes.byref(md2), pd, 1, ctypes.byref(g), 64, 8, 0, ctypes.byref(h)) == N.CVA_EINVAL
    # reset period not on the pricing grid
    g3 = N.GridDesc(5.0, 7, 1)
    assert L.cva_sim_create(ctypes.byref(md), pd, 1, ctypes.byref(g3), 64, 8, 0, ctypes.byref(h)) == N.CVA_EINVAL
    # regress / cva0 argument checks
    assert L.cva_cva0(None, 0, None, None) == N.CVA_EINVAL
    assert L.cva_regress(None, None, 1, 0, 0, None, None, None) == N.CVA_EINVAL


def test_python_binding_marshals_and_reports_errors(libcva):
    """The torch-facing binding builds the C structs and surfaces a host-side
    validation error as CvaError (no device call is reached)."""
    from paper_2211_17005_gb300 import api, workload as W
    from paper_2211_17005_gb300._native import CvaError, CVA_EINVAL
    wl = W.make("paper", M=64)
    with pytest.raises(CvaError) as ei:
        api.Simulation(wl.model, wl.portfolios, W.Grid(10.0, 300, 1), 64, 8)
    assert ei.value.status == CVA_EINVAL
    with pytest.raises(CvaError):
        api.Simulation(wl.model, wl.portfolios, wl.grid, 64, 0)


def test_oversimulation_choice_edges(libcva):
    """Prop. 1 / Heuristic 1 in the library (host only): dates without an interior
    optimum get NaN and are left out of the mean; no usable date is an error; the
    cost ratio needs two different draw counts."""
    import numpy as np
    from paper_2211_17005_gb300 import api
    from paper_2211_17005_gb300._native import CvaError, CVA_EINVAL, CVA_ENUMERIC
    Ni, N, M = api.oversimulation_choice([4.0, 1.0, -1.0], [1.0, 0.0, 1.0], 100.0, budget=1e6)
    assert Ni[0] == np.sqrt(4.0 * 100.0 / 1.0) and np.isnan(Ni[1]) and np.isnan(Ni[2])
    assert N == Ni[0] and M == 1e6 / (N + 100.0)
    with pytest.raises(CvaError) as ei:
        api.oversimulation_choice([1.0], [0.0], 10.0)
    assert ei.value.status == CVA_ENUMERIC
    with pytest.raises(CvaError) as ei:
        api.inner_cost_ratio(1.0, 8, 2.0, 8)
    assert ei.value.status == CVA_EINVAL
