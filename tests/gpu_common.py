"""Shared helpers of the GPU tests: library handle and oracle comparisons."""
import numpy as np
import pytest


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def lib():
    from paper_0801_1222_gb300 import build, hfqmc
    build.build()
    require_cuda()
    return hfqmc


def make_pair(orc, beta, grids, chains, seed=1, n_wrap=64, accept_rule="metropolis",
              precision="f64_rank1", **kw):
    """A GPU context and an oracle with identical grids, chains, seed, G0."""
    from paper_0801_1222_gb300 import inputs
    h = lib()
    U = [g[0] for g in grids]
    dtau = [g[1] for g in grids]
    ctx = h.HFQMC(beta, U, dtau, chains, seed=seed, precision=precision, n_wrap=n_wrap,
                  accept_rule=accept_rule, **kw)
    q = orc.OracleHFQMC(beta, grids, chains, seed=seed, n_wrap=n_wrap,
                        accept_rule={"metropolis": 0, "heat_bath": 1}[accept_rule])
    for i, (Ug, dt) in enumerate(grids):
        L = int(round(beta / dt))
        g0 = inputs.bethe_G0_tau(beta, L)
        ctx.set_G0(i, g0)
        q.set_G0(i, g0)
    return ctx, q


def compare_chains(ctx, q, rel_tol=1e-10):
    """Decision parity (hash, counts, field) and G agreement, every chain."""
    worst = 0.0
    for g, chains in enumerate(q.chains):
        for c, och in enumerate(chains):
            gc = ctx.get_chain(g, c)
            assert gc["t"] == och.t
            assert gc["hash"] == och.decision_hash, (g, c)
            assert gc["accepted"] == och.stats[1], (g, c)
            assert gc["proposals"] == och.stats[0]
            assert gc["recomputes"] == och.stats[2]
            assert np.array_equal(gc["s"], och.s)
            scale = max(np.abs(och.Gup).max(), np.abs(och.Gdn).max())
            err = max(np.abs(gc["Gup"] - och.Gup).max(), np.abs(gc["Gdn"] - och.Gdn).max())
            assert err <= rel_tol * scale, (g, c, err)
            if och.n_meas:
                assert np.max(np.abs(gc["acc"] - och.acc)) <= rel_tol * och.n_meas
                # double occupancy summed over the measured sweeps ("Benchmark
                # results": D at fixed dtau), each sweep's D <= 1/4
                D_sum, _ = ctx.get_chain_D(g, c)
                assert abs(D_sum - och.accD[0]) <= rel_tol * och.n_meas, (g, c, D_sum, och.accD[0])
            worst = max(worst, err / scale)
    return worst
