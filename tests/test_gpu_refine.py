"""The FP32 delayed path's recompute by Newton refinement (hfq_refine.cuh)
against the FP64 oracle, through the C ABI.

With n_wrap = 1 every accepted flip is followed by a recompute, so the FP32 G
that a run leaves behind was refined right after the last flip: it must equal
the oracle's FP64 Green matrices for the final field (fresh LU solve of the
Hirsch-Fye Dyson equation) to within a few times the FP32 rounding of those
matrices -- the accuracy a from-scratch FP64 recompute stored in FP32 has.  A
residual formed with FP32-level accuracy (an inexact tensor-core
accumulation, a wrong slice weight or level) would leave errors a hundred
times larger.  Grids: ragged Lambda = 37, G on chip (100), G in HBM with one
and two row blocks (200, 240), and Lambda = 500 (four row blocks, eight K
chunks)."""
import numpy as np
import pytest

from gpu_common import lib, make_pair

pytestmark = pytest.mark.gpu


def _fp32_rounding(G):
    return np.max(np.abs(G.astype(np.float32).astype(np.float64) - G))


@pytest.mark.parametrize("beta,U,L,chains", [
    (10.0, 4.0, 37, 3),
    (20.0, 5.0, 100, 2),
    (20.0, 5.0, 200, 2),
    (40.0, 5.0, 240, 2),
    (50.0, 4.8, 500, 1),
])
def test_refined_G_equals_fresh_fp64_inverse(orc, beta, U, L, chains):
    ctx, q = make_pair(orc, beta, [(U, beta / L)], [chains], precision="f32_delayed", n_wrap=1,
                       drift_fail=1.0, recompute="refine")
    ctx.sweep(0, 1)
    st = ctx.get_stats(0)
    assert st["accepted"] > 0 and st["recomputes"] == st["accepted"]
    assert st["recompute_fallbacks"] == 0, st
    M = q.chains[0][0].M
    lam = q.chains[0][0].lmbda
    for c in range(chains):
        ch = ctx.get_chain(0, c)
        for sig, G in ((1, ch["Gup"]), (-1, ch["Gdn"])):
            Gx, _ = orc.green(M, ch["s"], lam, sig)
            err = np.max(np.abs(G - Gx))
            assert err <= 4.0 * _fp32_rounding(Gx) + 1e-9, (L, c, sig, err, _fp32_rounding(Gx))


def test_refine_and_gauss_jordan_follow_the_oracle(orc):
    """N_wrap = 64 on Lambda = 100 and 200: over a short run most chains take
    the oracle's decisions, and their G stays within the FP32 drift of 64
    flips of it, with either recompute."""
    for rec in ("refine", "gj"):
        ctx, q = make_pair(orc, 20.0, [(5.0, 0.2), (5.0, 0.1)], [4, 2], precision="f32_delayed", n_wrap=64,
                           drift_fail=1.0, recompute=rec)
        ctx.sweep(1, 1)
        q.sweep(1, 1)
        same = 0
        for g in range(2):
            st = ctx.get_stats(g)
            assert st["recomputes"] > 0 and st["drift_max"] < 1e-3
            if rec == "refine":
                assert st["recompute_fallbacks"] == 0
            for c, och in enumerate(q.chains[g]):
                gc = ctx.get_chain(g, c)
                if gc["hash"] == och.decision_hash:
                    same += 1
                    err = max(np.abs(gc["Gup"] - och.Gup).max(), np.abs(gc["Gdn"] - och.Gdn).max())
                    assert err < 1e-3, (rec, g, c, err)
        assert same >= 3
        ctx.close()


@pytest.mark.parametrize("L,beta", [(100, 20.0), (240, 40.0)])
def test_refine_hands_large_residuals_to_gauss_jordan(orc, L, beta):
    """A residual above the step threshold sends the recompute to the FP64
    Gauss-Jordan inversion from the field.  With the threshold set to 1e-12
    every recompute falls back (G on chip at Lambda = 100, in HBM at 240):
    the fallbacks are counted and, with n_wrap = 1, the G a run leaves
    behind is the from-scratch inverse, as on the Gauss-Jordan path."""
    ctx, q = make_pair(orc, beta, [(5.0, beta / L)], [2], precision="f32_delayed", n_wrap=1,
                       drift_fail=1.0, recompute="refine", refine_max=1e-12)
    ctx.sweep(0, 1)
    st = ctx.get_stats(0)
    assert st["recomputes"] == st["accepted"] > 0
    assert st["recompute_fallbacks"] == st["recomputes"], st
    M, lam = q.chains[0][0].M, q.chains[0][0].lmbda
    for c in range(2):
        ch = ctx.get_chain(0, c)
        for sig, G in ((1, ch["Gup"]), (-1, ch["Gdn"])):
            Gx, _ = orc.green(M, ch["s"], lam, sig)
            assert np.max(np.abs(G - Gx)) <= 2.0 * _fp32_rounding(Gx) + 1e-9


def test_refine_takes_long_recompute_intervals(orc):
    """At N_wrap = 8192 (drift of a few 1e-3) the residual still allows Newton
    steps: the recomputes run without fallback and the drift stays bounded."""
    ctx, q = make_pair(orc, 40.0, [(5.0, 40.0 / 240)], [2], precision="f32_delayed", n_wrap=8192,
                       drift_fail=1.0, recompute="refine")
    ctx.sweep(0, 200)
    st = ctx.get_stats(0)
    assert st["recomputes"] >= 2 and st["drift_max"] < 0.1, st


def test_paired_G_tau_with_refine_at_nwrap_64():
    """The paired FP32-vs-FP64 criterion of tests/test_gpu_precision.py at
    the configurations' own recompute interval, N_wrap = 64, with the
    refinement: Lambda = 200 and 240, 500 sweeps (several hundred recomputes
    per chain)."""
    from test_gpu_precision import _assert_within, paired_run
    res = paired_run(40.0, [(5.0, 40.0 / 200), (5.0, 40.0 / 240)], 16, 21, 30, 470, n_wrap=64,
                     recompute="refine")
    for r in res:
        assert r["stats"]["recompute_fallbacks"] == 0
        assert np.max(np.abs(r["mean"])) < 1e-7
        _assert_within(r, 100)


def test_particle_hole_mirror_and_both_spins_refined(orc):
    """A particle-hole symmetric bath (the Bethe bath at half filling) turns
    the mirror on: with ph_symmetry = 0 the sweep keeps G_up only (G_dn =
    1 - G_up^T written when the call ends), with 1 the sweep updates both
    spins and the recompute refines G_up and sets G_dn = 1 - G_up^T.  With
    ph_symmetry = -1, or for a bath that is not symmetric, both spins are
    refined.  Every variant leaves G_up and G_dn within 4x FP32 rounding of the
    oracle's fresh FP64 inverses (n_wrap = 1)."""
    from paper_0801_1222_gb300 import inputs
    h = lib()
    beta, U, L = 20.0, 5.0, 200
    sym = inputs.bethe_G0_tau(beta, L)
    tau = np.arange(L) * beta / L
    asym = sym + 2e-3 * np.sin(2 * np.pi * tau / beta)  # G0(tau) != G0(beta - tau)
    for g0, phs, expect in ((sym, 0, 1), (sym, 1, 1), (sym, -1, 0), (asym, 0, 0)):
        ctx = h.HFQMC(beta, U, [beta / L], [2], seed=4, precision="f32_delayed", n_wrap=1,
                      drift_fail=1.0, recompute="refine", ph_symmetry=phs)
        ctx.set_G0(0, g0)
        ctx.sweep(0, 1)
        st = ctx.get_stats(0)
        assert st["ph_symmetric"] == expect and st["recompute_fallbacks"] == 0
        M = orc.bath_matrix(g0)
        lam = orc.lam(beta / L, U)
        for c in range(2):
            ch = ctx.get_chain(0, c)
            for sig, G in ((1, ch["Gup"]), (-1, ch["Gdn"])):
                Gx, _ = orc.green(M, ch["s"], lam, sig)
                assert np.max(np.abs(G - Gx)) <= 4.0 * _fp32_rounding(Gx) + 1e-9, (phs, expect, c, sig)
        ctx.close()


@pytest.mark.parametrize("L,beta,chains", [(100, 20.0, 4), (240, 40.0, 3), (37, 10.0, 4)])
def test_mirrored_sweep_follows_the_oracle(orc, L, beta, chains):
    """The sweep that keeps G_up only (every grid's bath particle-hole
    symmetric, ph_symmetry = 0) against the one that updates both spins
    (ph_symmetry = 1) and the FP64 oracle, same seeds, N_wrap 64 with the
    refinement: G on chip (Lambda = 100), in HBM (240), ragged (37).  The
    chains that took the oracle's decisions hold G_up within the FP32 drift of
    64 flips of it, G_dn = 1 - G_up^T bit for bit (written as 1 - x in FP32),
    and the measured G(tau) and D within the drift of the two-spin sweep's."""
    from paper_0801_1222_gb300 import inputs
    h = lib()
    res = {}
    for phs in (0, 1):
        ctx, qp = make_pair(orc, beta, [(5.0, beta / L)], [chains], precision="f32_delayed", n_wrap=64,
                            drift_fail=1.0, recompute="refine", ph_symmetry=phs)
        ctx.sweep(1, 2)
        if phs == 0:
            q = qp  # the oracle the mirrored sweep is compared with
            q.sweep(1, 2)
        st = ctx.get_stats(0)
        assert st["ph_symmetric"] == 1 and st["recompute_fallbacks"] == 0 and st["drift_max"] < 1e-3
        res[phs] = (ctx.get_G(0), ctx.get_D(0), [ctx.get_chain(0, c) for c in range(chains)])
        ctx.close()
    same = 0
    for c, och in enumerate(q.chains[0]):
        ch = res[0][2][c]
        np.testing.assert_array_equal(ch["Gdn"].astype(np.float32),
                                      (np.eye(L, dtype=np.float32) - ch["Gup"].astype(np.float32).T))
        if ch["hash"] == och.decision_hash:
            same += 1
            assert np.abs(ch["Gup"] - och.Gup).max() < 1e-3
            assert np.abs(ch["Gdn"] - och.Gdn).max() < 1e-3
    assert same >= 2
    # the two sweeps follow the same decisions as long as their FP32 rounding allows;
    # chains that agree give the same measured G(tau) to the drift
    agree = [c for c in range(chains) if res[0][2][c]["hash"] == res[1][2][c]["hash"]]
    assert len(agree) >= 2
    for c in agree:
        a, b = res[0][2][c], res[1][2][c]
        assert np.abs(a["acc"] - b["acc"]).max() < 1e-3


def test_mirror_turns_off_when_a_bath_loses_its_symmetry(orc):
    """set_G0 with an asymmetric bath on one grid of two switches the sweep
    back to both spins (the cached graph of the mirrored sweep is dropped):
    the decisions then follow the oracle's with that bath, and G_dn is no
    longer 1 - G_up^T."""
    from paper_0801_1222_gb300 import inputs
    h = lib()
    beta, L = 20.0, 100
    grids = [(5.0, beta / L), (5.0, beta / L)]
    ctx, q = make_pair(orc, beta, grids, [3, 3], precision="f32_delayed", n_wrap=64, drift_fail=1.0,
                       recompute="refine")
    ctx.sweep(0, 2)  # mirrored sweep, graph captured
    q.sweep(0, 2)
    tau = np.arange(L) * beta / L
    asym = inputs.bethe_G0_tau(beta, L) + 2e-3 * np.sin(2 * np.pi * tau / beta)
    ctx.set_G0(1, asym)
    q.set_G0(1, asym)
    assert ctx.get_stats(0)["ph_symmetric"] == 1 and ctx.get_stats(1)["ph_symmetric"] == 0
    ctx.sweep(0, 2)
    q.sweep(0, 2)
    same = 0
    for c, och in enumerate(q.chains[1]):
        ch = ctx.get_chain(1, c)
        if ch["hash"] == och.decision_hash:
            same += 1
            assert np.abs(ch["Gdn"] - och.Gdn).max() < 1e-3
        assert np.abs(ch["Gdn"] - (np.eye(L) - ch["Gup"].T)).max() > 1e-4
    assert same >= 1
    ctx.close()
