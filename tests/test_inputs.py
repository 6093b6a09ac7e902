"""Pins for the Bethe-lattice bath G0(tau) (the synthetic input recipe).

The Matsubara-sum construction is checked against the closed form as an
integral over the semicircular density of states,
    G0(tau) = -int rho(e) exp(-e tau) / (1 + exp(-beta e)) de,
    rho(e) = sqrt(4 - e^2) / (2 pi),
and against particle-hole symmetry at half filling."""
import numpy as np
import pytest
from scipy import integrate

from paper_0801_1222_gb300 import inputs


def _dos_integral(tau, beta):
    def f(e):
        # exp(-e tau)/(1+exp(-beta e)) written without overflow for either sign of e
        if e >= 0:
            return np.exp(-e * tau) / (1.0 + np.exp(-beta * e))
        return np.exp(e * (beta - tau)) / (np.exp(beta * e) + 1.0)
    val, _ = integrate.quad(f, -2.0, 2.0, weight="alg", wvar=(0.5, 0.5), epsabs=1e-13,
                            epsrel=1e-13, limit=400)
    return -val / (2.0 * np.pi)


@pytest.mark.parametrize("beta,L", [(8.0, 16), (20.0, 100), (40.0, 240)])
def test_bethe_G0_matches_dos_integral(beta, L):
    g0 = inputs.bethe_G0_tau(beta, L)
    ks = sorted(set([1, 2, L // 7, L // 3, L // 2, L - 1]))
    for k in ks:
        tau = k * beta / L
        assert abs(g0[k] - _dos_integral(tau, beta)) < 2e-9, (k, g0[k])
    assert g0[0] == -0.5
    assert abs(_dos_integral(1e-12, beta) + 0.5) < 1e-9


def test_bethe_G0_particle_hole_and_bath_matrix(orc):
    beta, L = 20.0, 100
    g0 = inputs.bethe_G0_tau(beta, L)
    assert np.max(np.abs(g0[1:] - g0[1:][::-1])) < 1e-13
    M = orc.bath_matrix(g0)
    # half filling: 1 - M^T = M
    assert np.max(np.abs((np.eye(L) - M.T) - M)) < 1e-13
    assert np.all(np.diag(M) == 0.5)


def test_grid_size():
    assert inputs.grid_size(40.0, 40.0 / 240) == 240
    with pytest.raises(ValueError):
        inputs.grid_size(40.0, 0.33)
