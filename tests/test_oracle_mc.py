"""Pins for the oracle's full Monte Carlo chain.

* Atomic limit (no hybridisation, G0(tau) = -1/2): the Trotter decoupling is
  exact at any dtau, so brute-force enumeration must give the closed forms
  g(tau) = (e^{tau U/2} + e^{(beta-tau) U/2}) / (2 (1 + e^{beta U/2})) and
  D = 1 / (2 + 2 e^{beta U/2}).
* Single-grid workload (Lambda = 16, U = 4, beta = 8, Bethe bath): Monte Carlo
  must hit the exact discrete-dtau G(tau) from enumeration of all 2^16 fields
  within its error bars.
* Detailed balance at Lambda = 4: the visited-field histogram matches w(s)/Z.
* U = 0: every proposal is accepted and G(tau) = G0(tau).
"""
import numpy as np
import pytest

from paper_0801_1222_gb300 import inputs


def _atomic_closed_form(beta, U, L):
    tau = np.arange(L) * beta / L
    g = (np.exp(tau * U / 2) + np.exp((beta - tau) * U / 2)) / (2 * (1 + np.exp(beta * U / 2)))
    D = 1.0 / (2 + 2 * np.exp(beta * U / 2))
    return g, D


@pytest.mark.parametrize("beta,U,L", [(4.0, 3.0, 8), (2.0, 5.0, 4), (6.0, 2.0, 12)])
def test_brute_force_atomic_limit_closed_form(orc, beta, U, L):
    M = orc.bath_matrix(inputs.atomic_G0_tau(L))
    g, D, Z = orc.brute_force(M, orc.lam(beta / L, U))
    gc, Dc = _atomic_closed_form(beta, U, L)
    assert np.max(np.abs(g - gc)) < 1e-13
    assert abs(D - Dc) < 1e-14


def test_mc_atomic_limit(orc):
    beta, U, L = 4.0, 3.0, 8
    q = orc.OracleHFQMC(beta, [(U, beta / L)], [8], seed=3, n_wrap=32)
    q.set_G0(0, inputs.atomic_G0_tau(L))
    q.sweep(500, 20000)
    G, err = q.get_G(0)
    gc, Dc = _atomic_closed_form(beta, U, L)
    assert np.all(np.abs(G[:L] + gc) <= 4 * err[:L] + 1e-12)
    D, Derr = q.get_D(0)
    assert abs(D - Dc) <= 4 * Derr


def test_mc_single_grid_matches_enumeration(orc):
    """Lambda = 16 single-chain workload, full length (10^4 + 10^5 sweeps)."""
    beta, U, L = 8.0, 4.0, 16
    g0 = inputs.bethe_G0_tau(beta, L)
    q = orc.OracleHFQMC(beta, [(U, beta / L)], [1], seed=1, n_wrap=64)
    q.set_G0(0, g0)
    q.sweep(10_000, 100_000)
    G, err = q.get_G(0)
    g_ex, D_ex, _ = orc.brute_force(orc.bath_matrix(g0), orc.lam(beta / L, U))
    z = (G[1:L] + g_ex[1:L]) / err[1:L]
    assert np.all(np.abs(z) < 4.0), z
    # chi-square over tau (particle-hole symmetry makes k and L-k identical)
    half = z[: L // 2]
    assert (half ** 2).sum() < len(half) + 5 * np.sqrt(2 * len(half))
    # half filling: G_up_ll + G_dn_ll = 1 for every field, so G(0+) = G(beta-) = -1/2
    assert abs(G[0] + 0.5) < 1e-12 and abs(G[L] + 0.5) < 1e-12
    D, _ = q.get_D(0)
    assert abs(D - D_ex) < 2e-3


def test_heat_bath_rule_matches_enumeration(orc):
    beta, U, L = 4.0, 4.0, 8
    g0 = inputs.bethe_G0_tau(beta, L)
    q = orc.OracleHFQMC(beta, [(U, beta / L)], [16], seed=9, accept_rule=1)
    q.set_G0(0, g0)
    q.sweep(200, 5000)
    G, err = q.get_G(0)
    g_ex, _, _ = orc.brute_force(orc.bath_matrix(g0), orc.lam(beta / L, U))
    assert np.all(np.abs(G[1:L] + g_ex[1:L]) <= 4 * err[1:L])


def test_detailed_balance_lambda4(orc):
    beta, U, L = 2.0, 4.0, 4
    g0 = inputs.bethe_G0_tau(beta, L)
    M = orc.bath_matrix(g0)
    lm = orc.lam(beta / L, U)
    _, _, Z, w = orc.brute_force(M, lm, return_weights=True)
    p = w / Z
    freqs = []
    for c in range(48):
        ch = orc.Chain.new(M, lm, 17, c, 0)
        hist = np.zeros(1 << L, dtype=np.int64)
        orc.run_chain(ch, 100, 20000, n_wrap=64, hist=hist)
        freqs.append(hist / hist.sum())
    freqs = np.array(freqs)
    mean = freqs.mean(axis=0)
    se = freqs.std(axis=0, ddof=1) / np.sqrt(len(freqs))
    assert np.all(np.abs(mean - p) < 5 * se + 1e-12), (mean, p)


def test_U0_all_accepted_and_G_is_G0(orc):
    beta, L = 8.0, 16
    g0 = inputs.bethe_G0_tau(beta, L)
    q = orc.OracleHFQMC(beta, [(0.0, beta / L)], [2], seed=1, n_wrap=16)
    q.set_G0(0, g0)
    q.sweep(2, 10)
    for ch in q.chains[0]:
        assert ch.stats[0] == ch.stats[1] == 12 * L
        assert np.array_equal(ch.Gup, orc.bath_matrix(g0))
    G, err = q.get_G(0)
    assert np.max(np.abs(G[:L] - g0)) < 1e-15


def test_multigrid_api_and_seed_independence(orc):
    beta = 4.0
    grids = [(4.0, 0.5), (4.0, 0.25)]
    q1 = orc.OracleHFQMC(beta, grids, [3, 2], seed=5)
    q2 = orc.OracleHFQMC(beta, grids, [3, 2], seed=5, threads=1)
    for q in (q1, q2):
        for i, (U, dt) in enumerate(grids):
            q.set_G0(i, inputs.bethe_G0_tau(beta, int(round(beta / dt))))
        q.sweep(10, 50)
    for i in range(2):
        a, ea = q1.get_G(i)
        b, eb = q2.get_G(i)
        assert np.array_equal(a, b) and np.array_equal(ea, eb)
    # chains are distinct streams
    h = {c.decision_hash for cs in q1.chains for c in cs}
    assert len(h) == 5


def test_golden_file_is_current(orc):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "single_L16_exact.txt")
    vals = np.loadtxt(path)
    g0 = inputs.bethe_G0_tau(8.0, 16)
    g, D, _ = orc.brute_force(orc.bath_matrix(g0), orc.lam(0.5, 4.0))
    assert np.max(np.abs(vals[:16] + g)) < 1e-14 and abs(vals[17] - D) < 1e-14
