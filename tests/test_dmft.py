"""DMFT glue (Fig. 1(c) cycle, Bethe lattice): transform pins against the
analytic semicircle, product-vs-oracle parity of the transform, the U = 0
fixed point (the non-interacting semicircle is self-consistent from the first
iteration), and a short GPU-driven DMFT run."""
import numpy as np
import pytest

from paper_0801_1222_gb300 import dmft, inputs


def test_spline_ft_of_the_semicircle():
    beta = 20.0
    tau = np.linspace(0.0, beta, 2001)
    g = inputs.bethe_G0_at(beta, tau)
    G_iw = dmft.spline_ft(beta, tau, g, 200)
    exact = inputs.bethe_G0_iw(1j * dmft.matsubara(beta, 200))
    assert np.max(np.abs(G_iw - exact)) < 2e-6
    # particle-hole symmetry: purely imaginary
    assert np.max(np.abs(G_iw.real)) < 1e-7


def test_bath_tau_round_trip():
    beta = 20.0
    G0_iw = inputs.bethe_G0_iw(1j * dmft.matsubara(beta, 1 << 14))
    tau = np.linspace(0.0, beta, 37)
    assert np.max(np.abs(dmft.bath_tau(beta, tau, G0_iw) - inputs.bethe_G0_at(beta, tau))) < 1e-9


def test_ft_matches_oracle_quadrature():
    from oracle import dmft as od
    beta = 10.0
    tau = np.linspace(0.0, beta, 4001)
    g = inputs.bethe_G0_at(beta, tau)
    a = dmft.spline_ft(beta, tau, g, 64)
    b = od.ft_trapezoid(beta, tau, g, 64)
    assert np.max(np.abs(a - b)) < 1e-6
    assert np.max(np.abs(dmft.bethe_update(a, beta) - od.bethe_update(a, beta))) < 1e-14


def test_U0_fixed_point_of_the_update():
    beta = 20.0
    tau = np.linspace(0.0, beta, 2001)
    g = inputs.bethe_G0_at(beta, tau)
    n_iw = 4096
    new = dmft.bethe_update(dmft.spline_ft(beta, tau, g, n_iw), beta)
    exact = inputs.bethe_G0_iw(1j * dmft.matsubara(beta, n_iw))
    assert np.max(np.abs(new - exact)) < 5e-6
    tk = np.linspace(0.0, beta, 41)
    assert np.max(np.abs(dmft.bath_tau(beta, tk, new) - inputs.bethe_G0_at(beta, tk))) < 5e-6


@pytest.mark.gpu
def test_gpu_dmft_loop_U0_is_stationary_and_U4_runs():
    from gpu_common import lib
    h = lib()
    beta = 8.0
    dtaus = [0.5, 0.4, 0.25]
    solver = h.HFQMC(beta, 0.0, dtaus, [4, 4, 4], seed=1, precision="f32_delayed", n_wrap=64,
                     drift_fail=1.0)
    loop = dmft.MultigridDMFT(solver, beta, dtaus, n_fine=801, n_iw=2048)
    g0_before = loop.G0_iw.copy()
    rec = loop.iterate(2, 20)
    assert np.max(np.abs(loop.G0_iw - g0_before)) < 1e-4
    assert abs(rec["D"] - 0.25) < 1e-4   # U = 0: <n_up n_dn> = 1/4 at half filling
    solver.close()
    solver = h.HFQMC(beta, 4.0, dtaus, [32, 32, 32], seed=1, precision="f32_delayed",
                     drift_fail=1.0)
    loop = dmft.MultigridDMFT(solver, beta, dtaus, n_fine=801, n_iw=2048, mix=0.7)
    for it in range(2):
        rec = loop.iterate(100 if it == 0 else 20, 400)
    assert np.all(np.isfinite(rec["G_fine"])) and 0.0 < rec["D"] < 0.25
    assert abs(rec["G_fine"][0] + 0.5) < 1e-4
