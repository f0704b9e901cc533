"""Outer paths split over two processes (torch.distributed, gloo, on the CPU): the
exchange that pools the ranks' estimates. Each rank takes its own range of global
paths; its partial sums (computed here from the FP64 oracle's run of that range, in
place of the GPU's cva_cva0_partials / cva_regress_partial) go through the rank-order
exchange of paper_2211_17005_gb300.shard and the library's host combination and
solve. Two ranks must give the one-rank results: CVA_0, its standard error and the
least-squares fits of every date. The same calls on a GPU are checked in
tests/test_gpu_shard.py; a multi-GPU run is not measured on hardware."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _estimates(name, k0, k1, combine_cva0, sum_parts, solve):
    """CVA_0 and the fits of dates 1..n-1 from the oracle's run of paths [k0, k1), with
    the partial sums pooled by sum_parts (an exchange, or nothing for one rank)."""
    import oracle
    from paper_2211_17005_gb300 import _native as nat, workload as W
    wl = W.make(name, M=2048, N=8, n_steps=10)
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, k0, k1, wl.N, wl.seed, want=("features", "xi_bar"))
    first = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, 1, wl.N, wl.seed, want=("features",))
    xi0 = o["xi_bar"][0]
    c0 = combine_cva0(sum_parts(np.array([[k1 - k0, xi0.sum(), (xi0 * xi0).sum()]]), stack=True))
    poly2 = name == "small"
    basis = nat.BASIS_POLY2 if poly2 else nat.BASIS_LINEAR
    fits = []
    for i in range(1, wl.grid.n_steps):
        Y = o["features"][i]                                   # [F, M]
        centre = first["features"][i, :1, 0] if poly2 else first["features"][i, :, 0]
        if poly2:
            d = Y[0] - centre[0]
            A = np.stack([np.ones_like(d), d, d * d, o["xi_bar"][i]], axis=1)
        else:
            A = np.concatenate([np.ones((1, Y.shape[1])), Y - centre[:, None], o["xi_bar"][i][None]]).T
        gram = sum_parts(A.T @ A, stack=False)
        _, w_raw, _ = solve(gram, Y.shape[0], basis, centre)
        fits.append(w_raw)
    return c0, np.array(fits)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        from paper_2211_17005_gb300 import shard

        def pooled(x, stack):
            return shard.gather_rank_order(x)[:, 0] if stack else shard.sum_rank_order(x)
        res = {}
        for name in ("small", "paper"):
            k0, M = shard.path_range(2048, rank, world)
            res[name] = _estimates(name, k0, k0 + M, shard.combine_cva0, pooled, shard.solve)
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_pool_to_the_one_rank_estimates(oracle_lib):
    from paper_2211_17005_gb300 import build, shard
    build.build()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0, p.exitcode
        res = dict(out)
    for name in ("small", "paper"):
        one = _estimates(name, 0, 2048, shard.combine_cva0, lambda x, stack: x, shard.solve)
        (c_a, f_a), (c_b, f_b) = res[0][name], res[1][name]
        # both ranks hold the same bits
        assert c_a == c_b and np.array_equal(f_a, f_b)
        # and the one-rank estimates, up to the order of the FP64 sums
        assert c_a[0] == pytest.approx(one[0][0], rel=1e-13) and c_a[1] == pytest.approx(one[0][1], rel=1e-9)
        np.testing.assert_allclose(f_a, one[1], rtol=1e-8, atol=1e-12 * np.abs(one[1]).max())


def test_host_solve_of_a_normal_matrix_equals_qr(oracle_lib):
    """cva_regress_solve on a summed normal matrix gives the least-squares fit of the
    oracle's Householder QR (same predictions), and drops a column with no spread."""
    import oracle
    from paper_2211_17005_gb300 import _native as nat, build, shard, workload as W
    build.build()
    wl = W.make("paper", M=1500, N=8, n_steps=10)
    o = oracle.simulate(wl.model, wl.portfolios[0], wl.grid, 0, wl.M, wl.N, wl.seed, want=("features", "xi_bar"))
    Y, xi = o["features"][5], o["xi_bar"][5]
    c = Y[:, 0]
    A = np.concatenate([np.ones((1, Y.shape[1])), Y - c[:, None], xi[None]]).T
    _, w_raw, nd = shard.solve(A.T @ A, Y.shape[0], nat.BASIS_LINEAR, c)
    _, p_qr = oracle.lsq(oracle.linear_features(Y), xi)
    p = np.concatenate([np.ones((1, Y.shape[1])), Y]).T @ w_raw
    assert nd == 0
    assert np.max(np.abs(p - p_qr)) < 1e-9 * np.sqrt(np.mean(xi ** 2))
    Y2 = Y.copy()
    Y2[3] = Y2[3, 0]                                    # a factor without spread
    A2 = np.concatenate([np.ones((1, Y.shape[1])), Y2 - Y2[:, :1], xi[None]]).T
    _, w2, nd2 = shard.solve(A2.T @ A2, Y.shape[0], nat.BASIS_LINEAR, Y2[:, 0])
    assert nd2 == 1 and w2[4] == 0.0
