"""DMFT self-consistency around the multigrid HF-QMC impurity solver (host glue).

The cycle of the paper's Fig. 1(c) for the Bethe lattice with semi-elliptic
DOS (W = 4, t = 1) at half filling: the impurity problem defined by the bath
G0 is solved by HF-QMC on every dtau grid at once (the CUDA library), the
grids' G(tau) are combined into the dtau -> 0 estimate on a fine tau grid
(multigrid.py), transformed to Matsubara frequencies, and the bath is updated
by the Bethe self-consistency G0^{-1}(iw) = iw - t^2 G(iw); the new bath is
sampled on every grid for the next iteration.

Fourier transforms:
  tau -> iw: G(iw) = int_0^beta e^{iw tau} G(tau) dtau of the cubic spline
  through the fine-grid values, integrated exactly by parts (boundary terms
  with the spline's derivatives at 0+ and beta-, then the piecewise-constant
  third derivative), which builds in the 1/(iw) jump G(0+) + G(beta-) = -1.
  iw -> tau: G0(tau) = -1/2 + tau(beta - tau)/4
             + (2/beta) sum_n Re[e^{-iw_n tau}(G0(iw_n) - 1/(iw_n) - 1/(iw_n)^3)],
  the bath's high-frequency tail being 1/(iw) + t^2/(iw)^3.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import CubicSpline

from . import inputs
from . import multigrid as mg


def matsubara(beta: float, n_iw: int) -> np.ndarray:
    return (2 * np.arange(n_iw) + 1) * np.pi / float(beta)


def _uniform_steps(beta, tau):
    """M when tau_k = k beta / M for k = 0..len(tau)-1 (len(tau) <= M + 1), else 0."""
    if tau.shape[0] < 2 or tau[0] != 0.0:
        return 0
    M = int(round(beta / (tau[1] - tau[0])))
    if M < 1 or tau.shape[0] > M + 1:
        return 0
    dev = np.max(np.abs(tau - np.arange(tau.shape[0]) * (beta / M)))
    return M if dev <= 1e-12 * beta else 0


def spline_ft(beta, tau, G, n_iw):
    """G(iw_n), n = 0..n_iw-1, from G on the uniform grid tau[0] = 0+ .. tau[-1] = beta-.

    The piecewise-constant third derivative s3_k on interval k enters as
    sum_k e^{iw_n tau_k} s3_k; with tau_k = k h, h = beta / N, the phase is
    e^{i pi k / N} e^{2 pi i n k / N}, so the sum over k is one inverse DFT of
    length N of s3_k e^{i pi k / N}, read at n mod N."""
    tau = np.asarray(tau, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    N = tau.shape[0] - 1
    h = tau[1] - tau[0]
    sp = CubicSpline(tau, G, bc_type="not-a-knot")
    d1, d2, d3 = sp.derivative(1), sp.derivative(2), sp.derivative(3)
    s3 = d3(tau[:-1] + 0.5 * h)  # constant third derivative on each interval
    iw = 1j * matsubara(beta, n_iw)
    S0, Sb = G[0], G[-1]
    out = (-(Sb + S0) / iw + (d1(tau[-1]) + d1(tau[0])) / iw ** 2
           - (d2(tau[-1]) + d2(tau[0])) / iw ** 3)
    k = np.arange(N)
    q = s3 * np.exp(1j * np.pi * k / N)
    phs3 = N * np.fft.ifft(q)[np.arange(n_iw) % N]   # sum_k e^{iw_n tau_k} s3_k
    out -= (np.exp(iw * h) - 1.0) / iw ** 4 * phs3
    return out


def bath_tau(beta, tau, G0_iw):
    """G0(tau) at the given tau values from its Matsubara values.

    The sum over n of Re[e^{-iw_n tau} r_n] (r_n the Matsubara values less the
    1/(iw) and 1/(iw)^3 tails) on a uniform grid tau_k = k beta / M: the phase
    is e^{-i pi k / M} e^{-2 pi i n k / M}, so folding r_n onto n mod M turns
    the sum into one DFT of length M; other tau are summed directly."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    wn = matsubara(beta, G0_iw.shape[0])
    iw = 1j * wn
    rest = G0_iw - 1.0 / iw - 1.0 / iw ** 3
    M = _uniform_steps(float(beta), tau)
    if M:
        folded = np.bincount(np.arange(rest.shape[0]) % M, weights=rest.real, minlength=M) \
            + 1j * np.bincount(np.arange(rest.shape[0]) % M, weights=rest.imag, minlength=M)
        F = np.fft.fft(folded)
        k = np.arange(tau.shape[0])
        out = (2.0 / beta) * np.real(np.exp(-1j * np.pi * k / M) * F[k % M])
    else:
        out = np.empty(tau.shape[0])
        for a in range(0, tau.shape[0], 64):
            t = tau[a:a + 64, None]
            out[a:a + 64] = (2.0 / beta) * np.real(np.exp(-1j * wn[None, :] * t) * rest[None, :]).sum(axis=1)
    out += -0.5 + tau * (beta - tau) / 4.0
    out[tau == 0.0] = -0.5
    out[tau == beta] = -0.5
    return out


def bethe_update(G_iw, beta):
    """Bethe self-consistency at half filling, t = 1: G0(iw) = 1 / (iw - G(iw))."""
    iw = 1j * matsubara(beta, G_iw.shape[0])
    return 1.0 / (iw - G_iw)


def extrapolate_scalar(dtaus, values, errors=None):
    """Quadratic-in-dtau^2 least-squares extrapolation of a scalar (e.g. D)."""
    a, sa, _ = mg.extrapolate(dtaus, np.asarray(values)[:, None],
                              None if errors is None else np.asarray(errors)[:, None])
    return float(a[0]), float(sa[0])


def ph_symmetrize(g):
    """A bath sampled at tau_k = k beta / L made exactly particle-hole
    symmetric: G0(tau_k) and G0(tau_{L-k}) replaced by their mean (the same
    floating-point value for both), G0(0+) = -1/2.  At half filling the exact
    bath has this symmetry; the Monte Carlo noise of a DMFT update breaks it
    slightly."""
    g = np.array(g, dtype=np.float64)
    L = g.shape[0]
    k = np.arange(1, L)
    out = g.copy()
    out[k] = 0.5 * (g[k] + g[L - k])
    out[0] = -0.5
    return out


class MultigridDMFT:
    """Multigrid HF-QMC DMFT on the Bethe lattice.  ``solver`` is an
    ``hfqmc.HFQMC`` context (or anything with its set_G0 / sweep / get_G /
    get_D calls, e.g. the oracle) over the grids ``dtaus`` of one U, starting
    at grid index ``grid0`` of the solver.  ``ph_symmetric``: every bath
    sampled on a grid is made exactly particle-hole symmetric (half filling;
    the library then keeps G_up only)."""

    def __init__(self, solver, beta, dtaus, n_fine=1001, n_iw=4096, mix=1.0, grid0=0, ph_symmetric=False):
        self.solver = solver
        self.beta = float(beta)
        self.dtaus = list(dtaus)
        self.Ls = [inputs.grid_size(beta, d) for d in self.dtaus]
        self.tau_fine = np.linspace(0.0, self.beta, n_fine)
        self.n_iw = n_iw
        self.mix = mix
        self.grid0 = int(grid0)
        self.G0_iw = inputs.bethe_G0_iw(1j * matsubara(self.beta, n_iw))
        self.ph_symmetric = bool(ph_symmetric)
        self.history = []

    def bath_on_grid(self, L):
        g = bath_tau(self.beta, np.arange(L) * self.beta / L, self.G0_iw)
        return ph_symmetrize(g) if self.ph_symmetric else g

    def set_baths(self):
        """The current bath, sampled on every grid of this loop."""
        for i, L in enumerate(self.Ls):
            self.solver.set_G0(self.grid0 + i, self.bath_on_grid(L))

    def iterate(self, n_warm, n_meas):
        self.set_baths()
        self.solver.sweep(n_warm, n_meas)
        return self.collect()

    def collect(self):
        """After the sweeps: the multigrid estimate, its transform and the
        Bethe update of the bath."""
        idx = [self.grid0 + i for i in range(len(self.Ls))]
        Gs, Es = zip(*[self.solver.get_G(i) for i in idx])
        Ds = [self.solver.get_D(i) for i in idx]
        ref = lambda t: bath_tau(self.beta, t, self.G0_iw)
        G_fine, G_err, _ = mg.multigrid_estimate(self.beta, self.dtaus, list(Gs), list(Es),
                                                 self.tau_fine, ref)
        G_iw = spline_ft(self.beta, self.tau_fine, G_fine, self.n_iw)
        new = bethe_update(G_iw, self.beta)
        self.G0_iw = self.mix * new + (1.0 - self.mix) * self.G0_iw
        D, D_err = extrapolate_scalar(self.dtaus, [d[0] for d in Ds], [d[1] for d in Ds])
        rec = dict(G_fine=G_fine, G_err=G_err, G_iw=G_iw, D_grids=[d[0] for d in Ds], D=D, D_err=D_err)
        self.history.append(rec)
        return rec


class BatchedMultigridDMFT:
    """Several independent multigrid DMFT loops -- one per interaction U --
    whose impurity problems share one solver context (grid index u * n_dtau +
    i for U[u] and dtau[i], created with a per-grid U): every iteration sets
    all baths, runs one sweep call over every chain of every (U, dtau) grid,
    then updates each U's bath from its own grids."""

    def __init__(self, solver, beta, Us, dtaus, n_fine=1001, n_iw=4096, mix=1.0, ph_symmetric=False):
        self.solver = solver
        self.Us = list(Us)
        self.loops = [MultigridDMFT(solver, beta, dtaus, n_fine=n_fine, n_iw=n_iw, mix=mix,
                                    grid0=u * len(dtaus), ph_symmetric=ph_symmetric)
                      for u in range(len(self.Us))]

    def iterate(self, n_warm, n_meas):
        for lp in self.loops:
            lp.set_baths()
        self.solver.sweep(n_warm, n_meas)
        return [lp.collect() for lp in self.loops]


class FixedDtauDMFT(MultigridDMFT):
    """Conventional HF-QMC DMFT at one fixed dtau (the paper's Fig. 1(a) loop):
    the impurity G on the grid is splined onto the fine tau grid and used as
    it is, without a dtau -> 0 extrapolation.  ``solver`` holds that one grid."""

    def __init__(self, solver, beta, dtau, n_fine=1001, n_iw=4096, mix=1.0):
        super().__init__(solver, beta, [dtau], n_fine=n_fine, n_iw=n_iw, mix=mix)


def fixed_dtau_sequence(make_solver, beta, dtaus, n_iter, n_warm, n_meas, n_fine=1001, n_iw=4096,
                        mix=1.0):
    """Conventional runs for the dtau -> 0 comparison of the "Benchmark
    results" section: a converged fixed-dtau DMFT loop per dtau (make_solver(dtau)
    returns a one-grid solver context), then the double occupancy D(dtau)
    extrapolated quadratically in dtau^2.  Returns (D per dtau, D error per
    dtau, D extrapolated, its error, the loops)."""
    loops, Ds, Es = [], [], []
    for dt in dtaus:
        solver = make_solver(dt)
        loop = FixedDtauDMFT(solver, beta, dt, n_fine=n_fine, n_iw=n_iw, mix=mix)
        for it in range(n_iter):
            rec = loop.iterate(n_warm, n_meas)
        Ds.append(rec["D_grids"][0])
        Es.append(rec["D_err"])
        loops.append(loop)
    D0, E0 = extrapolate_scalar(dtaus, Ds, Es)
    return Ds, Es, D0, E0, loops

