"""Oracle of the multigrid dtau -> 0 estimate (test infrastructure).

Written independently of the product glue from the paper's "Multigrid
HF-QMC method" section: per grid, the difference from the reference model is
interpolated by a natural cubic spline (second derivatives from the textbook
tridiagonal system, solved densely), evaluated on the fine tau grid and the
reference added back; at every fine point G = a + b dtau^2 + c dtau^4 is
fitted by weighted least squares (numpy lstsq on the weighted design
matrix); a is the estimate.
"""
from __future__ import annotations

import numpy as np


def natural_spline_eval(x, y, xq):
    """Natural cubic spline through (x_i, y_i), evaluated at xq."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    h = np.diff(x)
    A = np.zeros((n, n))
    r = np.zeros(n)
    A[0, 0] = 1.0
    A[-1, -1] = 1.0
    for i in range(1, n - 1):
        A[i, i - 1] = h[i - 1]
        A[i, i] = 2.0 * (h[i - 1] + h[i])
        A[i, i + 1] = h[i]
        r[i] = 6.0 * ((y[i + 1] - y[i]) / h[i] - (y[i] - y[i - 1]) / h[i - 1])
    M = np.linalg.solve(A, r)  # second derivatives at the knots
    xq = np.asarray(xq, dtype=np.float64)
    out = np.empty(xq.shape[0])
    for q, t in enumerate(xq):
        i = min(max(int(np.searchsorted(x, t, side="right")) - 1, 0), n - 2)
        hi = h[i]
        u0 = x[i + 1] - t
        u1 = t - x[i]
        out[q] = (M[i] * u0 ** 3 / (6 * hi) + M[i + 1] * u1 ** 3 / (6 * hi)
                  + (y[i] / hi - M[i] * hi / 6) * u0 + (y[i + 1] / hi - M[i + 1] * hi / 6) * u1)
    return out


def interpolate(beta, G_grid, tau_fine, ref=None):
    G_grid = np.asarray(G_grid, dtype=np.float64)
    L = G_grid.shape[0] - 1
    tk = np.arange(L + 1) * (float(beta) / L)
    rk = ref(tk) if ref is not None else np.zeros(L + 1)
    rf = ref(np.asarray(tau_fine)) if ref is not None else 0.0
    return natural_spline_eval(tk, G_grid - rk, tau_fine) + rf


def extrapolate(dtaus, G_fine, err_fine=None):
    x = np.asarray(dtaus, dtype=np.float64) ** 2
    G_fine = np.asarray(G_fine, dtype=np.float64)
    n, m = G_fine.shape
    # one grid: the fixed-dtau value itself (the conventional procedure)
    deg = 2 if n >= 3 else (1 if n == 2 else 0)
    X = np.vander(x, deg + 1, increasing=True)  # 1, x, x^2
    a = np.empty(m)
    for t in range(m):
        w = np.ones(n) if err_fine is None else 1.0 / np.asarray(err_fine)[:, t]
        coef, *_ = np.linalg.lstsq(X * w[:, None], G_fine[:, t] * w, rcond=None)
        a[t] = coef[0]
    return a


def multigrid_estimate(beta, dtaus, G_list, err_list, tau_fine, ref=None):
    Gf = np.array([interpolate(beta, G, tau_fine, ref) for G in G_list])
    Ef = None
    if err_list is not None:
        Ef = np.maximum(np.array([np.abs(interpolate(beta, E, tau_fine, None)) for E in err_list]), 1e-15)
    return extrapolate(dtaus, Gf, Ef)
