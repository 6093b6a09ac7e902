"""The DMFT loops (Fig. 1 cycles) with the GPU's FP64 rank-1 path as the
impurity solver against the same loops with the oracle as the solver: same
grids, chains, seeds and recompute interval, so the two solvers take the same
accept/reject decisions and return G(tau) equal to 1e-10; the host glue is
the same, so every bath update G0(iw) must agree to 1e-9.  Covered: the
multigrid loop, the conventional fixed-dtau loop, and the batched loop over
several U values in one context (the config-5 structure), plus that config's
full shape (four U values x six grids, 1024 chains) for one short iteration
on the FP32 delayed path."""
import numpy as np
import pytest

from gpu_common import lib

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _pair(h, orc, beta, grids, chains, seed=3, n_wrap=16):
    U = [g[0] for g in grids]
    dt = [g[1] for g in grids]
    gpu = h.HFQMC(beta, U, dt, chains, seed=seed, precision="f64_rank1", n_wrap=n_wrap, drift_fail=1.0)
    ora = orc.OracleHFQMC(beta, grids, chains, seed=seed, n_wrap=n_wrap)
    return gpu, ora


def test_multigrid_dmft_updates_match_the_oracle_solver(orc):
    from paper_0801_1222_gb300 import dmft
    h = lib()
    beta, U = 4.0, 4.0
    dtaus = [0.5, 0.4, 0.25]
    gpu, ora = _pair(h, orc, beta, [(U, d) for d in dtaus], [4, 4, 4])
    la = dmft.MultigridDMFT(gpu, beta, dtaus, n_fine=401, n_iw=1024, mix=0.8)
    lb = dmft.MultigridDMFT(ora, beta, dtaus, n_fine=401, n_iw=1024, mix=0.8)
    for it, (nw, nm) in enumerate([(20, 150), (5, 150), (5, 150)]):
        ra, rb = la.iterate(nw, nm), lb.iterate(nw, nm)
        assert np.max(np.abs(la.G0_iw - lb.G0_iw)) <= TOL, it
        assert abs(ra["D"] - rb["D"]) <= TOL
        np.testing.assert_allclose(ra["G_fine"], rb["G_fine"], rtol=0, atol=TOL)
    gpu.close()


def test_fixed_dtau_dmft_updates_match_the_oracle_solver(orc):
    from paper_0801_1222_gb300 import dmft
    h = lib()
    beta, U, dt = 4.0, 4.0, 0.25
    gpu, ora = _pair(h, orc, beta, [(U, dt)], [6])
    la = dmft.FixedDtauDMFT(gpu, beta, dt, n_fine=401, n_iw=1024)
    lb = dmft.FixedDtauDMFT(ora, beta, dt, n_fine=401, n_iw=1024)
    for it in range(3):
        ra, rb = la.iterate(10 if it == 0 else 2, 200), lb.iterate(10 if it == 0 else 2, 200)
        assert np.max(np.abs(la.G0_iw - lb.G0_iw)) <= TOL, it
        assert abs(ra["D_grids"][0] - rb["D_grids"][0]) <= TOL
    gpu.close()


def test_batched_multi_U_dmft_matches_the_oracle_solver(orc):
    from paper_0801_1222_gb300 import dmft
    h = lib()
    beta = 4.0
    Us, dtaus = [4.0, 5.0], [0.5, 0.25]
    grids = [(U, d) for U in Us for d in dtaus]
    gpu, ora = _pair(h, orc, beta, grids, [3, 4, 3, 4])
    la = dmft.BatchedMultigridDMFT(gpu, beta, Us, dtaus, n_fine=401, n_iw=1024, mix=0.8)
    lb = dmft.BatchedMultigridDMFT(ora, beta, Us, dtaus, n_fine=401, n_iw=1024, mix=0.8)
    for it in range(2):
        ra, rb = la.iterate(10, 100), lb.iterate(10, 100)
        for u in range(2):
            assert np.max(np.abs(la.loops[u].G0_iw - lb.loops[u].G0_iw)) <= TOL, (it, u)
            assert abs(ra[u]["D"] - rb[u]["D"]) <= TOL
    # the two U values really run different problems
    assert np.max(np.abs(la.loops[0].G0_iw - la.loops[1].G0_iw)) > 1e-3
    gpu.close()


def test_config5_shape_one_short_iteration():
    """Four U values x six grids (Lambda 80 .. 320), 1024 chains in one FP32
    delayed context: two DMFT iterations with a few sweeps and particle-hole
    symmetric baths (so every grid keeps G_up only); every U's bath update is
    finite and D lies in (0, 1/4), decreasing with U."""
    from paper_0801_1222_gb300 import dmft, inputs
    h = lib()
    w = inputs.WORKLOADS["dmft_c5"]
    grids = inputs.workload_grids("dmft_c5")
    assert len(grids) == 24 and sum(g[3] for g in grids) == 1024
    beta = w["beta"]
    ctx = h.HFQMC(beta, [g[0] for g in grids], [g[1] for g in grids], [g[3] for g in grids], seed=1,
                  precision="f32_delayed", drift_fail=1.0)
    loop = dmft.BatchedMultigridDMFT(ctx, beta, w["U"], [beta / L for L in w["L"]], n_fine=801, n_iw=2048,
                                     ph_symmetric=True)
    loop.iterate(5, 20)
    recs = loop.iterate(5, 20)  # the updated baths, made particle-hole symmetric, keep G_up only
    Ds = [r["D"] for r in recs]
    assert all(np.all(np.isfinite(lp.G0_iw)) for lp in loop.loops)
    assert all(0.0 < d < 0.25 for d in Ds) and Ds[0] > Ds[-1]
    for g in range(24):
        st = ctx.get_stats(g)
        assert st["n_wrap"] == 64 and st["accepted"] > 0 and st["ph_symmetric"] == 1
    ctx.close()
