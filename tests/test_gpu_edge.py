"""Edge cases of the sweep through the C ABI: the smallest grids (Lambda = 1,
2, 3), the largest the delayed path takes (Lambda = 512, more rows than
threads), the large-Lambda workload shape (Lambda = 500, where k is lowered
to fit the panels on chip: to 8 with both spins' panels, to 24 when the
sweep keeps G_up only), and the size limits."""
import numpy as np
import pytest

from gpu_common import compare_chains, lib, make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 2, 3])
def test_tiny_grids_fp64_decisions(orc, L):
    beta = 2.0
    ctx, q = make_pair(orc, beta, [(4.0, beta / L)], [3], n_wrap=4)
    ctx.sweep(5, 50)
    q.sweep(5, 50)
    compare_chains(ctx, q)
    assert np.max(np.abs(ctx.get_G(0)[0] - q.get_G(0)[0])) < 1e-10


@pytest.mark.parametrize("L", [1, 2, 3])
def test_tiny_grids_fp32_delayed(orc, L):
    beta = 2.0
    ctx, q = make_pair(orc, beta, [(4.0, beta / L)], [3], precision="f32_delayed", n_wrap=4,
                       drift_fail=1.0)
    ctx.sweep(5, 50)
    q.sweep(5, 50)
    G, E = ctx.get_G(0)
    Go, Eo = q.get_G(0)
    assert np.all(np.isfinite(G))
    assert np.max(np.abs(G - Go)) <= 1e-5 + 3 * np.max(np.sqrt(E ** 2 + Eo ** 2))


def test_lambda_512_delayed_follows_oracle(orc):
    """Lambda = 512 (two rows per thread): over a short run most chains
    follow the oracle's decisions, and those that do hold G within the FP32
    drift (at least two must, so the comparison cannot pass empty)."""
    beta = 51.2
    ctx, q = make_pair(orc, beta, [(4.8, 0.1)], [4], precision="f32_delayed", n_wrap=-1,
                       drift_fail=1.0)
    ctx.sweep(0, 1)
    q.sweep(0, 1)
    same = 0
    for c, och in enumerate(q.chains[0]):
        gc = ctx.get_chain(0, c)
        assert gc["accepted"] > 100
        if gc["hash"] == och.decision_hash:
            same += 1
            err = max(np.abs(gc["Gup"] - och.Gup).max(), np.abs(gc["Gdn"] - och.Gdn).max())
            assert err < 1e-3
    assert same >= 2


@pytest.mark.parametrize("beta,U,dtau,k,k_fit", [(50.0, 4.8, 0.1, 64, 24), (40.0, 5.0, 0.125, 40, 40)])
def test_one_spin_layout_deeper_delay_follows_oracle(orc, beta, U, dtau, k, k_fit):
    """The particle-hole symmetric bath runs the G_up-only sweep, whose panels
    hold one spin: at Lambda = 500 the requested k = 64 is lowered to 24
    (8 with both spins' panels), at Lambda = 320 k = 40 fits (16 with both).
    With the recompute every 64 accepted flips, most chains follow the
    oracle's decisions over a sweep, and those that do hold both spins' G
    within the FP32 drift (at least two must)."""
    ctx, q = make_pair(orc, beta, [(U, dtau)], [4], precision="f32_delayed", k=k, n_wrap=64,
                       drift_fail=1.0)
    ctx.sweep(0, 1)
    q.sweep(0, 1)
    st = ctx.get_stats(0)
    assert st["ph_symmetric"] == 1 and st["k"] == k_fit, st
    assert st["recomputes"] >= 4 and st["recompute_fallbacks"] == 0
    same = 0
    for c, och in enumerate(q.chains[0]):
        gc = ctx.get_chain(0, c)
        assert gc["accepted"] > 64
        if gc["hash"] == och.decision_hash:
            same += 1
            err = max(np.abs(gc["Gup"] - och.Gup).max(), np.abs(gc["Gdn"] - och.Gdn).max())
            assert err < 1e-3
    assert same >= 2


def test_large_lambda_workload_shape_runs():
    """Lambda = 500 (U = 4.8, beta = 50): the requested k = 64 does not fit the
    panels on chip, so the library lowers it (to 24 for the G_up-only sweep
    of this particle-hole symmetric bath); FP32 G(tau) follows the FP64 path
    on the same chains over a short run."""
    from paper_0801_1222_gb300 import inputs
    h = lib()
    beta, U, L = 50.0, 4.8, 500
    g0 = inputs.bethe_G0_tau(beta, L)
    res = {}
    for prec in ("f64_rank1", "f32_delayed"):
        ctx = h.HFQMC(beta, U, [0.1], [4], seed=3, precision=prec, k=64, n_wrap=64 if prec == "f32_delayed" else -1,
                      drift_fail=1.0)
        ctx.set_G0(0, g0)
        ctx.sweep(0, 2)
        res[prec] = (ctx.get_G(0), ctx.get_stats(0))
        ctx.close()
    (G64, _), _ = res["f64_rank1"]
    (G32, _), st = res["f32_delayed"]
    assert st["k"] == 24 and st["recomputes"] > 0 and st["drift_max"] < 1.0
    assert np.max(np.abs(G32 - G64)) < 5e-3


def test_size_limits():
    from paper_0801_1222_gb300 import inputs
    h = lib()
    with pytest.raises(h.HFQMCError) as ei:
        h.HFQMC(60.0, 4.0, [60.0 / 600], [1], precision="f32_delayed")
    assert ei.value.name == "EINVAL"
    ctx = h.HFQMC(60.0, 4.0, [60.0 / 600], [1], precision="f64_rank1", n_wrap=-1)
    ctx.set_G0(0, inputs.bethe_G0_tau(60.0, 600))
    ctx.sweep(0, 1)
    G, _ = ctx.get_G(0)
    assert np.all(np.isfinite(G)) and abs(G[0] + 0.5) < 1e-9
