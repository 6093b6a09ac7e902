"""The measurement of the sweep that keeps G_up only (k_delayed.cu, kMirror),
restated in numpy: for G_dn = 1 - G_up^T (every field of a particle-hole
symmetric bath) the signed diagonal sums of G_dn, which the measurement
needs, follow from G_up's: a_dn(0) = L - a_up(0) and a_dn(k) = a_up(L - k)
for k > 0, with a(k) = sum_l sgn(l, k) G_{(l+k) mod L, l} and sgn = -1 where
the antiperiodic wrap l + k >= L applies.  The double occupancy's summand
(1 - G_up,ll)(1 - G_dn,ll) becomes (1 - G_up,ll) G_up,ll.  Checked against
the sums taken on G_dn directly, on random matrices and on the oracle's
Green matrices of a field, where 1 - G_up^T = G_dn holds to rounding."""
import numpy as np
import pytest


def diag_sums(G):
    L = G.shape[0]
    a = np.zeros(L)
    for k in range(L):
        for l in range(L):
            r = l + k
            a[k] += G[r, l] if r < L else -G[r - L, l]
    return a


def derived_dn(a_up):
    L = a_up.shape[0]
    out = np.empty(L)
    out[0] = L - a_up[0]
    out[1:] = a_up[L - np.arange(1, L)]
    return out


@pytest.mark.parametrize("L", [1, 2, 7, 16, 37])
def test_spin_down_sums_from_spin_up(L):
    rng = np.random.default_rng(L)
    Gu = rng.standard_normal((L, L))
    Gd = np.eye(L) - Gu.T
    np.testing.assert_allclose(derived_dn(diag_sums(Gu)), diag_sums(Gd), rtol=0, atol=1e-12)
    # D's summand
    np.testing.assert_allclose((1 - np.diag(Gu)) * (1 - np.diag(Gd)), (1 - np.diag(Gu)) * np.diag(Gu), atol=1e-15)


def test_a_planted_sign_or_index_mistake_fails():
    """The derivation is not vacuous: the sign of the wrap left unflipped, or
    the diagonal index k taken for L - k, miss by O(1) on a random matrix."""
    L = 16
    rng = np.random.default_rng(3)
    Gu = rng.standard_normal((L, L))
    a_dn = diag_sums(np.eye(L) - Gu.T)
    a_up = diag_sums(Gu)
    wrong_sign = derived_dn(a_up).copy()
    wrong_sign[1:] = -wrong_sign[1:]
    wrong_index = a_up.copy()
    wrong_index[0] = L - a_up[0]
    assert np.abs(wrong_sign - a_dn).max() > 0.5
    assert np.abs(wrong_index - a_dn).max() > 0.5


def test_on_the_oracles_green_matrices(orc):
    """For a field of the half-filled Bethe bath the oracle's G_dn equals
    1 - G_up^T to rounding, so its measured sums follow from G_up's."""
    from paper_0801_1222_gb300 import inputs
    beta, U, L = 10.0, 4.0, 40
    M = orc.bath_matrix(inputs.bethe_G0_tau(beta, L))
    lam = orc.lam(beta / L, U)
    s = orc.init_field(L, 9, 2, 0)
    Gu, _ = orc.green(M, s, lam, 1)
    Gd, _ = orc.green(M, s, lam, -1)
    assert np.abs(Gd - (np.eye(L) - Gu.T)).max() < 1e-10
    np.testing.assert_allclose(derived_dn(diag_sums(Gu)), diag_sums(Gd), rtol=0, atol=1e-9)
