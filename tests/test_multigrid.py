"""Multigrid dtau -> 0 estimate (the paper's "Multigrid HF-QMC method"
section): oracle pins, product-vs-oracle parity, and the whole pipeline on
the GPU against the same estimate from exact enumeration."""
import numpy as np
import pytest

from paper_0801_1222_gb300 import inputs
from paper_0801_1222_gb300 import multigrid as mg


def _atomic_closed_form(beta, U, tau):
    return -(np.exp(tau * U / 2) + np.exp((beta - tau) * U / 2)) / (2 * (1 + np.exp(beta * U / 2)))


def _exact_grid_G(orc, beta, U, L, atomic=False):
    """Exact discrete-dtau G(tau_k), k = 0..L (physical sign) by enumeration."""
    g0 = inputs.atomic_G0_tau(L) if atomic else inputs.bethe_G0_tau(beta, L)
    g, D, _ = orc.brute_force(orc.bath_matrix(g0), orc.lam(beta / L, U))
    return np.concatenate([-g, [-1.0 + g[0]]])


def test_oracle_spline_pins():
    from oracle import multigrid as omg
    x = np.linspace(0.0, 3.0, 9)
    xq = np.linspace(0.0, 3.0, 101)
    assert np.max(np.abs(omg.natural_spline_eval(x, 2 * x - 1, xq) - (2 * xq - 1))) < 1e-13
    y = np.sin(x)
    assert np.max(np.abs(omg.natural_spline_eval(x, y, x) - y)) < 1e-14
    xf = np.linspace(0.0, np.pi, 65)
    err = np.abs(omg.natural_spline_eval(xf, np.sin(xf), xq[xq <= np.pi]) - np.sin(xq[xq <= np.pi]))
    assert err.max() < 1e-6


def test_oracle_extrapolation_recovers_exact_quadratic_in_dtau2():
    from oracle import multigrid as omg
    dt = np.array([0.5, 0.4, 0.3, 0.25])
    a = np.array([0.3, -1.2, 2.0])
    b = np.array([1.0, 0.5, -3.0])
    c = np.array([-0.7, 2.0, 0.1])
    G = a[None, :] + b[None, :] * dt[:, None] ** 2 + c[None, :] * dt[:, None] ** 4
    assert np.max(np.abs(omg.extrapolate(dt, G) - a)) < 1e-12
    assert np.max(np.abs(mg.extrapolate(dt, G)[0] - a)) < 1e-12


def test_oracle_atomic_limit_estimate_converges_to_the_continuum(orc):
    """Atomic limit: HF-QMC is Trotter-exact, so every grid samples the
    continuum g(tau) exactly (checked by enumeration at Lambda = 8, 12, 16);
    without a reference model the estimate carries only the spline's
    interpolation error, which must shrink as the grids refine."""
    from oracle import multigrid as omg
    beta, U = 4.0, 3.0
    Ls = [8, 12, 16]
    Gs = [_exact_grid_G(orc, beta, U, L, atomic=True) for L in Ls]
    for L, G in zip(Ls, Gs):
        tk = np.arange(L + 1) * beta / L
        assert np.max(np.abs(G - _atomic_closed_form(beta, U, tk))) < 1e-12
    tf = np.linspace(0.0, beta, 41)
    cf = _atomic_closed_form(beta, U, tf)
    err_coarse = np.max(np.abs(omg.multigrid_estimate(beta, [beta / L for L in Ls], Gs, None, tf) - cf))
    fine = [32, 48, 64]
    Gf = [_atomic_closed_form(beta, U, np.arange(L + 1) * beta / L) for L in fine]
    err_fine = np.max(np.abs(omg.multigrid_estimate(beta, [beta / L for L in fine], Gf, None, tf) - cf))
    assert err_coarse < 5e-3 and err_fine < err_coarse / 3
    # with the continuum itself as reference model the estimate is exact
    ref = lambda t: _atomic_closed_form(beta, U, t)
    assert np.max(np.abs(omg.multigrid_estimate(beta, [beta / L for L in Ls], Gs, None, tf, ref) - cf)) < 1e-11


def test_product_matches_oracle(orc):
    from oracle import multigrid as omg
    beta, U = 8.0, 4.0
    Ls = [8, 10, 12, 16]
    Gs = [_exact_grid_G(orc, beta, U, L) for L in Ls]
    Es = [np.full(L + 1, 1e-3) * (1 + 0.1 * i) for i, L in enumerate(Ls)]
    tf = np.linspace(0.0, beta, 57)
    ref = lambda t: inputs.bethe_G0_at(beta, t)
    dts = [beta / L for L in Ls]
    a_p, sa, _ = mg.multigrid_estimate(beta, dts, Gs, Es, tf, ref)
    a_o = omg.multigrid_estimate(beta, dts, Gs, Es, tf, ref)
    assert np.max(np.abs(a_p - a_o)) < 1e-10
    assert np.all(np.isfinite(sa))
    # half filling: G(0+) = G(beta-) = -1/2 survives interpolation and fit
    assert abs(a_p[0] + 0.5) < 1e-10 and abs(a_p[-1] + 0.5) < 1e-10


@pytest.mark.gpu
def test_gpu_multigrid_pipeline_matches_enumeration(orc):
    """GPU Monte Carlo on Lambda = 8, 12, 16 (Bethe bath, U = 4, beta = 8),
    then the multigrid estimate, against the estimate built from the exact
    discrete G of each grid."""
    from gpu_common import lib
    h = lib()
    beta, U = 8.0, 4.0
    Ls = [8, 12, 16]
    dts = [beta / L for L in Ls]
    ctx = h.HFQMC(beta, U, dts, [64] * 3, seed=2, precision="f64_rank1", n_wrap=64)
    for i, L in enumerate(Ls):
        ctx.set_G0(i, inputs.bethe_G0_tau(beta, L))
    ctx.sweep(500, 4000)
    Gs, Es = zip(*[ctx.get_G(i) for i in range(3)])
    tf = np.linspace(0.0, beta, 33)
    ref = lambda t: inputs.bethe_G0_at(beta, t)
    a, sa, _ = mg.multigrid_estimate(beta, dts, list(Gs), list(Es), tf, ref)
    exact = [_exact_grid_G(orc, beta, U, L) for L in Ls]
    a_ex, _, _ = mg.multigrid_estimate(beta, dts, exact, list(Es), tf, ref)
    assert np.all(np.abs(a - a_ex)[1:-1] <= 4 * sa[1:-1] + 1e-6), np.max(np.abs(a - a_ex) / sa)


def test_extrapolation_coefficients_and_error_propagation():
    """The per-point weighted fit, solved for all fine points at once: with as
    many grids as coefficients it interpolates, so a(tau) is the Lagrange
    value at dtau = 0 and sigma_a^2 = sum_i (l_i(0) e_i)^2 with the Lagrange
    basis l_i in x = dtau^2; with more grids a, b and sigma_a equal numpy's
    weighted polyfit and its unscaled covariance, point by point; error
    bars <= 0 take the smallest positive one of their point."""
    rng = np.random.default_rng(11)
    m = 7
    for dts in ([0.5, 0.4], [0.5, 0.4, 0.25]):
        x = np.asarray(dts) ** 2
        n = len(dts)
        G = rng.standard_normal((n, m))
        E = rng.uniform(1e-4, 1e-3, (n, m))
        a, sa, b = mg.extrapolate(dts, G, E)
        ell0 = [np.prod([(0.0 - x[j]) / (x[i] - x[j]) for j in range(n) if j != i]) for i in range(n)]
        np.testing.assert_allclose(a, sum(ell0[i] * G[i] for i in range(n)), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(sa, np.sqrt(sum((ell0[i] * E[i]) ** 2 for i in range(n))), rtol=1e-9)
    dts = [0.5, 0.4, 0.3, 0.25, 0.2, 1 / 6]
    x = np.asarray(dts) ** 2
    G = rng.standard_normal((6, m))
    E = rng.uniform(1e-4, 1e-3, (6, m))
    E[2, 3] = 0.0
    a, sa, b = mg.extrapolate(dts, G, E)
    for t in range(m):
        e = E[:, t].copy()
        e[e <= 0] = e[e > 0].min()
        coef, cov = np.polyfit(x, G[:, t], 2, w=1.0 / e, cov="unscaled")
        assert abs(a[t] - coef[-1]) < 1e-10 and abs(b[t] - coef[-2]) < 1e-8
        assert abs(sa[t] - np.sqrt(cov[-1, -1])) < 1e-10 * max(1.0, sa[t])
    a1, sa1, b1 = mg.extrapolate(dts, G, None)
    assert np.all(np.isnan(sa1))
    np.testing.assert_allclose(a1, [np.polyfit(x, G[:, t], 2)[-1] for t in range(m)], atol=1e-10)
