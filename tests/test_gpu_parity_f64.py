"""GPU FP64 rank-1 path against the FP64 oracle, through the C ABI.

Same Philox stream, same bath: the accept/reject sequence must be identical
(decision hash over every accepted (sweep, slice), accept count, final field)
and G must agree to 1e-10 relative; measured G(tau) likewise.  Sizes span
several warps' worth of slices with ragged tails, both shared-memory-resident
and HBM-resident G, the longest-first queue over uneven grids, recomputes,
both acceptance rules and repeated calls."""
import numpy as np
import pytest

from gpu_common import compare_chains, lib, make_pair

pytestmark = pytest.mark.gpu


def test_single_grid_L16_decisions(orc):
    ctx, q = make_pair(orc, 8.0, [(4.0, 0.5)], [1], n_wrap=64)
    ctx.sweep(100, 1000)
    q.sweep(100, 1000)
    compare_chains(ctx, q)
    G, E = ctx.get_G(0)
    Go, Eo = q.get_G(0)
    assert np.max(np.abs(G - Go)) < 1e-10
    assert np.max(np.abs(E - Eo)) < 1e-9


def test_L100_eight_chains_decisions(orc):
    ctx, q = make_pair(orc, 20.0, [(5.0, 0.2)], [8], n_wrap=64)
    ctx.sweep(5, 20)
    q.sweep(5, 20)
    compare_chains(ctx, q)
    G, E = ctx.get_G(0)
    Go, Eo = q.get_G(0)
    assert np.max(np.abs(G - Go)) < 1e-10
    assert np.max(np.abs(E - Eo)) < 1e-10


def test_uneven_grids_resident_and_hbm(orc):
    # Lambda = 37 (ragged), 100 (shared-memory G), 130 (HBM G); U differs per grid
    grids = [(4.0, 10.0 / 37), (5.0, 0.1), (5.2, 10.0 / 130)]
    ctx, q = make_pair(orc, 10.0, grids, [3, 2, 2], n_wrap=32)
    ctx.sweep(3, 6)
    q.sweep(3, 6)
    compare_chains(ctx, q)
    for g in range(3):
        assert np.max(np.abs(ctx.get_G(g)[0] - q.get_G(g)[0])) < 1e-10



def test_hbm_workspace_blocked_inversion_L200(orc):
    """Lambda = 200: the FP64 workspace does not fit in shared memory, so the
    initial G of each chain comes from the inversion by 16-column panels
    (implicit pivoting); the decisions and G follow the oracle's LU solve to
    1e-10 over several sweeps with recomputes."""
    ctx, q = make_pair(orc, 20.0, [(5.0, 0.1)], [2], n_wrap=64)
    ctx.sweep(1, 2)
    q.sweep(1, 2)
    compare_chains(ctx, q)

def test_heat_bath_decisions(orc):
    ctx, q = make_pair(orc, 8.0, [(4.0, 0.25)], [4], accept_rule="heat_bath", n_wrap=16)
    ctx.sweep(20, 100)
    q.sweep(20, 100)
    compare_chains(ctx, q)


def test_repeated_calls_and_graph_replay(orc):
    ctx, q = make_pair(orc, 8.0, [(4.0, 0.25)], [3], n_wrap=16)
    for nw, nm in [(10, 0), (0, 40), (0, 40), (5, 7)]:
        ctx.sweep(nw, nm)
        q.sweep(nw, nm)
    compare_chains(ctx, q)
    assert np.max(np.abs(ctx.get_G(0)[0] - q.get_G(0)[0])) < 1e-10
    assert np.max(np.abs(ctx.get_G(0)[1] - q.get_G(0)[1])) < 1e-10


def test_set_G0_again_keeps_field(orc):
    from paper_0801_1222_gb300 import inputs
    ctx, q = make_pair(orc, 8.0, [(4.0, 0.5)], [2])
    ctx.sweep(10, 10)
    q.sweep(10, 10)
    g0 = inputs.bethe_G0_tau(8.0, 16) * 0.9 + 0.1 * inputs.atomic_G0_tau(16)
    ctx.set_G0(0, g0)
    q.set_G0(0, g0)
    ctx.sweep(5, 30)
    q.sweep(5, 30)
    compare_chains(ctx, q)
    assert np.max(np.abs(ctx.get_G(0)[0] - q.get_G(0)[0])) < 1e-10


def test_U0_everything_accepted_G_is_G0(orc):
    from paper_0801_1222_gb300 import inputs
    ctx, q = make_pair(orc, 8.0, [(0.0, 0.5)], [2], n_wrap=8)
    ctx.sweep(2, 10)
    st = ctx.get_stats(0)
    assert st["proposals"] == st["accepted"] == 2 * 12 * 16
    G, _ = ctx.get_G(0)
    assert np.max(np.abs(G[:16] - inputs.bethe_G0_tau(8.0, 16))) < 1e-15


def test_single_grid_full_length_matches_enumeration():
    """Lambda = 16 workload, full length on the GPU, against the stored 2^16
    enumeration (tests/golden/single_L16_exact.txt)."""
    import os
    from paper_0801_1222_gb300 import inputs
    h = lib()
    exact = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "single_L16_exact.txt"))
    ctx = h.HFQMC(8.0, 4.0, [0.5], [1], seed=1, precision="f64_rank1", n_wrap=64)
    ctx.set_G0(0, inputs.bethe_G0_tau(8.0, 16))
    ctx.sweep(10_000, 100_000)
    G, E = ctx.get_G(0)
    z = (G[1:16] - exact[1:16]) / E[1:16]
    assert np.all(np.abs(z) < 4.0), z
    assert abs(G[0] + 0.5) < 1e-12 and abs(G[16] + 0.5) < 1e-12
    D, D_err = ctx.get_D(0)
    assert np.isfinite(D_err) and 0.0 < D_err < 1e-3
    assert abs(D - exact[17]) <= 4.0 * D_err, (D, exact[17], D_err)


def test_errors_surface_as_status_codes():
    from paper_0801_1222_gb300 import inputs
    h = lib()
    ctx = h.HFQMC(8.0, 4.0, [0.5, 0.25], [1, 1], precision="f64_rank1")
    ctx.set_G0(0, inputs.bethe_G0_tau(8.0, 16))
    with pytest.raises(h.HFQMCError) as ei:
        ctx.sweep(1, 1)
    assert ei.value.name == "ESTATE"
    with pytest.raises(h.HFQMCError) as ei:
        ctx.set_G0(5, inputs.bethe_G0_tau(8.0, 16))
    assert ei.value.name == "EINVAL"
    bad = inputs.bethe_G0_tau(8.0, 32)
    bad[3] = np.nan
    with pytest.raises(h.HFQMCError) as ei:
        ctx.set_G0(1, bad)
    assert ei.value.name == "EINVAL"
