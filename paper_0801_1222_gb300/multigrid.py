"""Multigrid dtau -> 0 estimate of the impurity Green function (host glue).

The paper's "Multigrid HF-QMC method" section obtains an unbiased G from the
HF-QMC results G_dtau_i of several grids in two steps: (i) each discrete
estimate is interpolated onto a common fine tau grid with the help of a
reference model; (ii) at every fine tau point a least-squares fit quadratic
in dtau^2 is extrapolated to dtau = 0.

Reference model: the paper points to another work for it.  Here the
reference is a continuous-tau function supplied by the caller -- by default
the bath G0(tau) of the same impurity problem, which carries the steep
structure near tau = 0 and beta -- and the difference G_dtau - ref, smooth,
is interpolated by a natural cubic spline through the grid points tau_k,
k = 0..Lambda (the last point is beta-).  The fit is
    G(tau; dtau) = a(tau) + b(tau) dtau^2 + c(tau) dtau^4
weighted by the error bars, and a(tau) with its standard error is the
estimate (fewer than three grids: the fit drops to a + b dtau^2).
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import CubicSpline


def grid_taus(beta: float, L: int) -> np.ndarray:
    """tau_k = k beta / L, k = 0..L (k = L is beta-)."""
    return np.arange(L + 1) * (float(beta) / L)


def interpolate_to_fine(beta, G_grid, tau_fine, ref=None, ref_fine=None):
    """G_grid: the Lambda+1 values G(tau_k), k = 0..Lambda, of one grid.
    ref: callable ref(tau) -> array, or None (no reference); ref_fine: ref at
    tau_fine when the caller has it already."""
    G_grid = np.asarray(G_grid, dtype=np.float64)
    L = G_grid.shape[0] - 1
    tk = grid_taus(beta, L)
    r_k = ref(tk) if ref is not None else 0.0
    spline = CubicSpline(tk, G_grid - r_k, bc_type="natural")
    if ref is None:
        r_f = 0.0
    else:
        r_f = ref_fine if ref_fine is not None else ref(tau_fine)
    return spline(tau_fine) + r_f


def extrapolate(dtaus, G_fine, err_fine=None):
    """Weighted least squares in x = dtau^2 at every fine tau point.

    dtaus: n grids; G_fine: n x m values on the fine grid; err_fine: n x m
    error bars (None: equal weights).  Returns (a, sigma_a, b); sigma_a is
    propagated from the error bars through the fit, (X^T W X)^{-1}, which
    stays defined when the fit has no residual degrees of freedom (NaN when
    no error bars are given).  All points are solved at once: a QR
    factorisation of the weighted design matrix per point, stacked."""
    x = np.asarray(dtaus, dtype=np.float64) ** 2
    G_fine = np.asarray(G_fine, dtype=np.float64)
    n, m = G_fine.shape
    # a + b x + c x^2 for three or more grids, a + b x for two; one grid is
    # the conventional fixed-dtau estimate itself (no extrapolation)
    deg = 2 if n >= 3 else (1 if n == 2 else 0)
    X = np.vander(x, deg + 1)  # x^deg ... x^0
    if err_fine is None:
        w = np.ones((n, m))
    else:
        e = np.asarray(err_fine, dtype=np.float64)
        pos = e > 0
        # a non-positive error bar takes the smallest positive one of its point
        floor = np.where(pos, e, np.inf).min(axis=0)
        floor = np.where(np.isfinite(floor), floor, 1.0)
        w = 1.0 / np.where(pos, e, floor[None, :])
    Xw = X[None, :, :] * w.T[:, :, None]          # m x n x (deg+1)
    yw = (G_fine * w).T[:, :, None]               # m x n x 1
    Q, R = np.linalg.qr(Xw)                       # R: m x (deg+1) x (deg+1)
    coef = np.linalg.solve(R, np.swapaxes(Q, 1, 2) @ yw)[:, :, 0]
    a = coef[:, -1].copy()
    b = coef[:, -2].copy() if deg > 0 else np.zeros(m)
    sa = np.full(m, np.nan)
    if err_fine is not None:
        # (X^T W X)^{-1} = R^{-1} R^{-T}: its last diagonal entry is the squared
        # norm of the last row of R^{-1}
        Rinv = np.linalg.inv(R)
        sa = np.sqrt(np.sum(Rinv[:, -1, :] ** 2, axis=1))
    return a, sa, b


def multigrid_estimate(beta, dtaus, G_list, err_list, tau_fine, ref=None):
    """The dtau -> 0 estimate on tau_fine from the per-grid G(tau_k) (each of
    length Lambda_i + 1) and their error bars (interpolated the same way)."""
    ref_fine = ref(tau_fine) if ref is not None else None  # the same for every grid
    Gf = np.array([interpolate_to_fine(beta, G, tau_fine, ref, ref_fine) for G in G_list])
    Ef = None
    if err_list is not None:
        Ef = np.array([np.abs(interpolate_to_fine(beta, E, tau_fine, None)) for E in err_list])
        Ef = np.maximum(Ef, 1e-15)
    return extrapolate(dtaus, Gf, Ef)
