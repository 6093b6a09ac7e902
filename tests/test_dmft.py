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


@pytest.mark.parametrize("M,K", [(80, 80), (320, 320), (1000, 1001), (240, 241), (7, 8)])
def test_bath_tau_on_a_uniform_grid_by_dft_equals_the_direct_sum(M, K):
    """On tau_k = k beta / M the Matsubara sum is taken as one DFT of the
    frequencies folded onto n mod M; in any other order of the same points it
    is summed term by term.  Both agree (a bath with noise in every
    frequency, more frequencies than points and fewer)."""
    beta = 40.0
    rng = np.random.default_rng(3)
    for n_iw in (4096, 5):
        iw = 1j * dmft.matsubara(beta, n_iw)
        G0_iw = inputs.bethe_G0_iw(iw) + 1e-3 * (rng.standard_normal(n_iw) + 1j * rng.standard_normal(n_iw)) / (1 + iw.imag ** 2)
        tau = np.arange(K) * (beta / M)
        fast = dmft.bath_tau(beta, tau, G0_iw)
        direct = dmft.bath_tau(beta, tau[::-1], G0_iw)[::-1]  # not ascending from 0: summed directly
        # the direct sum's phases w_n tau reach 2 pi n_iw: its own rounding is ~1e-13
        assert np.max(np.abs(fast - direct)) < 1e-12


def test_spline_ft_third_derivative_sum_by_dft():
    """The sum over intervals of e^{iw_n tau_k} s3_k taken by one inverse DFT
    equals the explicit phase matrix, for more frequencies than intervals and
    fewer."""
    from scipy.interpolate import CubicSpline
    beta = 10.0
    rng = np.random.default_rng(5)
    for N, n_iw in ((100, 4096), (1000, 64)):
        tau = np.linspace(0.0, beta, N + 1)
        g = inputs.bethe_G0_at(beta, tau, 1 << 12) + 1e-3 * rng.standard_normal(N + 1)
        h = tau[1] - tau[0]
        sp = CubicSpline(tau, g, bc_type="not-a-knot")
        d1, d2, d3 = sp.derivative(1), sp.derivative(2), sp.derivative(3)
        iw = 1j * dmft.matsubara(beta, n_iw)
        ref = (-(g[-1] + g[0]) / iw + (d1(tau[-1]) + d1(tau[0])) / iw ** 2 - (d2(tau[-1]) + d2(tau[0])) / iw ** 3
               - (np.exp(iw * h) - 1.0) / iw ** 4 * (np.exp(np.outer(iw, tau[:-1])) @ d3(tau[:-1] + 0.5 * h)))
        got = dmft.spline_ft(beta, tau, g, n_iw)
        # rounding of either way of summing: a few N eps of sum |s3|, times the
        # factor |(e^{iw h} - 1) / (iw)^4| (large at the lowest frequencies)
        s3 = d3(tau[:-1] + 0.5 * h)
        tol = 8 * N * np.finfo(float).eps * np.sum(np.abs(s3)) * np.abs((np.exp(iw * h) - 1.0) / iw ** 4) + 1e-14
        assert np.all(np.abs(got - ref) <= tol)


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


def test_one_grid_fit_is_the_grid_value():
    """The conventional (fixed-dtau) procedure: a single grid's values are the
    estimate, with their own error bars (product and oracle agree)."""
    from paper_0801_1222_gb300 import multigrid as mg
    from oracle import multigrid as om
    vals = np.array([[0.3, -0.2, 0.11]])
    errs = np.array([[1e-3, 2e-3, 5e-4]])
    a, sa, b = mg.extrapolate([0.25], vals, errs)
    np.testing.assert_allclose(a, vals[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(sa, errs[0], rtol=1e-12)
    assert np.all(b == 0.0)
    np.testing.assert_allclose(om.extrapolate([0.25], vals, errs), vals[0], rtol=0, atol=1e-15)
    D, E = dmft.extrapolate_scalar([0.4], [0.2], [0.01])
    assert D == 0.2 and abs(E - 0.01) < 1e-15


def _oracle_solver(beta, U, dtau, chains=2, seed=3):
    from oracle import OracleHFQMC
    return OracleHFQMC(beta, [(U, dtau)], [chains], seed=seed, n_wrap=16)


def test_fixed_dtau_dmft_U0_is_stationary_with_the_oracle_solver():
    """Conventional loop at U = 0: G = G0 on the grid, the spline of G - G0 is
    zero, so the updated bath is the semicircle again and D = 1/4."""
    beta, dtau = 4.0, 0.5
    loop = dmft.FixedDtauDMFT(_oracle_solver(beta, 0.0, dtau), beta, dtau, n_fine=401, n_iw=1024)
    g0 = loop.G0_iw.copy()
    rec = loop.iterate(2, 20)
    # round-off of the bath's Matsubara sum and the spline transform only
    assert np.max(np.abs(loop.G0_iw - g0)) < 1e-10
    assert abs(rec["D"] - 0.25) < 1e-12


def test_fixed_dtau_sequence_with_the_oracle_solver():
    """D(dtau) from converged fixed-dtau loops and its dtau^2 extrapolation:
    physical range, the extrapolation a weighted fit through the points."""
    beta, U = 2.0, 2.0
    dtaus = [0.5, 0.4, 0.25]
    Ds, Es, D0, E0, loops = dmft.fixed_dtau_sequence(
        lambda dt: _oracle_solver(beta, U, dt, chains=4), beta, dtaus, n_iter=2, n_warm=50,
        n_meas=400, n_fine=201, n_iw=512, mix=1.0)
    assert len(Ds) == 3 and all(0.0 < d < 0.25 for d in Ds)
    assert all(e > 0 for e in Es) and np.isfinite(D0) and E0 > 0
    # the quadratic fit through three points reproduces them
    x = np.array(dtaus) ** 2
    c = np.polyfit(x, Ds, 2)
    assert abs(c[-1] - D0) < 1e-12
    for lp in loops:
        assert abs(lp.history[-1]["G_fine"][0] + 0.5) < 0.05


@pytest.mark.gpu
def test_gpu_fixed_dtau_sequence_U4():
    from gpu_common import lib
    h = lib()
    beta, U = 4.0, 4.0
    dtaus = [0.5, 0.4, 0.25]

    def make(dt):
        return h.HFQMC(beta, U, [dt], [32], seed=2, precision="f32_delayed", drift_fail=1.0)

    Ds, Es, D0, E0, loops = dmft.fixed_dtau_sequence(make, beta, dtaus, n_iter=2, n_warm=100,
                                                     n_meas=400, n_fine=401, n_iw=1024, mix=0.8)
    assert all(0.0 < d < 0.25 for d in Ds) and np.isfinite(D0) and 0.0 < D0 < 0.25
    for lp in loops:
        assert np.all(np.isfinite(lp.history[-1]["G_fine"]))
        lp.solver.close()


def test_ph_symmetrize_is_exact_and_keeps_a_symmetric_bath(orc):
    """ph_symmetrize makes G0(tau_k) and G0(tau_{L-k}) the same double and
    G0(0+) = -1/2 (the library's particle-hole test then finds a deviation of
    exactly 0); on the Bethe bath, symmetric already up to its Matsubara-sum
    rounding, it changes nothing beyond 1e-12.  A multigrid DMFT iteration
    with the oracle as the solver and ph_symmetric=True samples symmetric
    baths from the updated G0(iw) as well."""
    from paper_0801_1222_gb300 import dmft, inputs
    for beta, L in ((8.0, 16), (40.0, 240), (10.0, 37)):
        g = inputs.bethe_G0_tau(beta, L)
        s = dmft.ph_symmetrize(g)
        assert s[0] == -0.5 and all(s[k] == s[L - k] for k in range(1, L))
        assert np.abs(s - g).max() < 1e-12
        noisy = g + 1e-4 * np.sin(np.arange(L) * 2.3)
        s2 = dmft.ph_symmetrize(noisy)
        assert all(s2[k] == s2[L - k] for k in range(1, L))
    beta, U = 4.0, 4.0
    dtaus = [0.5, 0.25]
    q = orc.OracleHFQMC(beta, [(U, d) for d in dtaus], [3, 3], seed=2, n_wrap=16)
    loop = dmft.MultigridDMFT(q, beta, dtaus, n_fine=401, n_iw=1024, ph_symmetric=True)
    loop.iterate(5, 40)
    for L in loop.Ls:
        g = loop.bath_on_grid(L)
        assert g[0] == -0.5 and all(g[k] == g[L - k] for k in range(1, L))
