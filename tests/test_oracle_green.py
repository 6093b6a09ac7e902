"""Pins for the oracle's Green-function algebra (initial G, ratio, update).

Each check is fixed by mathematics, not by re-running the oracle's formula:
U = 0 leaves G = G0; the flip ratio equals the ratio of determinants of
A = 1 + (1 - G0)(e^V - 1); a rank-1 updated G equals a fresh inversion for the
new field; at half filling G_dn(s) = 1 - G_up(s)^T; the measurement of the bath
matrix returns -G0(tau)."""
import numpy as np
import pytest

from paper_0801_1222_gb300 import inputs


def _setup(beta=8.0, L=16, U=4.0):
    g0 = inputs.bethe_G0_tau(beta, L)
    return g0, beta / L


def test_U0_gives_G0_exactly(orc):
    g0, dtau = _setup()
    M = orc.bath_matrix(g0)
    lm = orc.lam(dtau, 0.0)
    assert lm == 0.0
    s = orc.init_field(16, 3, 0, 0)
    for sigma in (1, -1):
        G, det = orc.green(M, s, lm, sigma)
        assert np.array_equal(G, M)
        assert det == 1.0


def test_measure_of_bath_is_minus_G0(orc):
    g0 = inputs.bethe_G0_tau(20.0, 100)
    g = orc.measure_g(orc.bath_matrix(g0))
    assert np.max(np.abs(g + g0)) < 1e-15


def test_lambda_definition(orc):
    for dtau, U in [(0.5, 4.0), (0.2, 5.0), (0.1, 4.8)]:
        lm = orc.lam(dtau, U)
        assert abs(np.cosh(lm) - np.exp(dtau * U / 2)) < 1e-14


def test_green_dyson_relation_between_fields(orc):
    """Hirsch-Fye's Dyson relation ties the Green matrices of two fields s,
    s' together: G' = G + (G - 1)(e^{V' - V} - 1) G' with V = sigma lambda s.
    It follows from G^{-1} = (M^{-1} - 1) e^V + 1 and holds for any pair of
    fields, so the oracle's G for one field is checked against its G for
    others (a flipped sign of V, or the factors (1 - M) and (e^V - 1) in the
    other order, break it).  Fields differing in one, a few and half of the
    slices, both spins, at Lambda = 16 and 100."""
    rng = np.random.default_rng(5)
    for beta, L, U in ((8.0, 16, 4.0), (20.0, 100, 5.0)):
        g0, dtau = _setup(beta, L, U)
        M = orc.bath_matrix(g0)
        lm = orc.lam(dtau, U)
        s = orc.init_field(L, 7, 1, 0)
        for nflip in (1, 3, L // 2):
            s2 = s.copy()
            s2[rng.choice(L, nflip, replace=False)] *= -1
            for sigma in (1, -1):
                G, _ = orc.green(M, s, lm, sigma)
                G2, _ = orc.green(M, s2, lm, sigma)
                d = np.exp(sigma * lm * (s2 - s)) - 1.0
                rhs = G + (G - np.eye(L)) @ (d[:, None] * G2)
                assert np.max(np.abs(G2 - rhs)) < 1e-10 * max(1.0, np.max(np.abs(G2))), (L, nflip, sigma)
                # the relation is not empty: the two fields' matrices differ
                assert np.max(np.abs(G2 - G)) > 1e-3


@pytest.mark.parametrize("beta,L,U", [(8.0, 16, 4.0), (20.0, 100, 5.0)])
def test_ratio_equals_determinant_ratio(orc, beta, L, U):
    g0 = inputs.bethe_G0_tau(beta, L)
    M = orc.bath_matrix(g0)
    lm = orc.lam(beta / L, U)
    s = orc.init_field(L, 11, 0, 0)
    rng = np.random.default_rng(0)
    for l in rng.choice(L, 5, replace=False):
        s2 = s.copy()
        s2[l] = -s2[l]
        R = 1.0
        for sigma in (1, -1):
            G, _ = orc.green(M, s, lm, sigma)
            delta = np.exp(-2 * sigma * lm * s[l]) - 1.0
            R *= 1.0 + (1.0 - G[l, l]) * delta
        dets = 1.0
        for sigma in (1, -1):
            a1 = np.linalg.slogdet(orc.build_A(M, s2, lm, sigma))
            a0 = np.linalg.slogdet(orc.build_A(M, s, lm, sigma))
            dets *= a1[0] * a0[0] * np.exp(a1[1] - a0[1])
        assert abs(R - dets) <= 1e-11 * abs(dets)


def test_rank1_updates_match_fresh_inversion(orc):
    """The chain's own rank-1 path (no recompute) against a fresh LU."""
    for beta, L, U in [(8.0, 16, 4.0), (20.0, 100, 5.0)]:
        g0 = inputs.bethe_G0_tau(beta, L)
        M = orc.bath_matrix(g0)
        lm = orc.lam(beta / L, U)
        ch = orc.Chain.new(M, lm, 1, 0, 0)
        orc.run_chain(ch, 3, 0, n_wrap=0)
        assert ch.stats[1] > 10
        for sigma, G in ((1, ch.Gup), (-1, ch.Gdn)):
            ref, _ = orc.green(M, ch.s, lm, sigma)
            assert np.max(np.abs(G - ref)) < 1e-10


def test_particle_hole_identity(orc):
    g0 = inputs.bethe_G0_tau(20.0, 100)
    M = orc.bath_matrix(g0)
    lm = orc.lam(0.2, 5.0)
    s = orc.init_field(100, 5, 2, 0)
    Gu, du = orc.green(M, s, lm, 1)
    Gd, dd = orc.green(M, s, lm, -1)
    # exact identity; the residual is LU rounding amplified by cond(A) ~ 1e4
    assert np.max(np.abs(Gd - (np.eye(100) - Gu.T))) < 1e-10
    assert du > 0 and dd > 0


def test_recompute_drift_is_rounding_level(orc):
    g0 = inputs.bethe_G0_tau(20.0, 100)
    M = orc.bath_matrix(g0)
    ch = orc.Chain.new(M, orc.lam(0.2, 5.0), 1, 0, 0)
    orc.run_chain(ch, 5, 0, n_wrap=16)
    assert ch.stats[2] >= 1
    assert 0.0 < ch.drift < 1e-10
