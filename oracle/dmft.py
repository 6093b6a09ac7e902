"""Oracle of the DMFT glue's transforms (test infrastructure).

tau -> iw by the trapezoid rule on the fine grid with the Euler-Maclaurin
endpoint correction h^2/12 [f'(beta-) e^{iw beta} - f'(0+)] (derivatives from
one-sided second-order differences) -- an independent quadrature of the same
integral the product evaluates through its spline; the Bethe update is the
formula G0 = 1/(iw - G) written out again.
"""
from __future__ import annotations

import numpy as np


def ft_trapezoid(beta, tau, G, n_iw):
    tau = np.asarray(tau, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    h = tau[1] - tau[0]
    wn = (2 * np.arange(n_iw) + 1) * np.pi / beta
    out = np.empty(n_iw, dtype=complex)
    d0 = (-3 * G[0] + 4 * G[1] - G[2]) / (2 * h)
    db = (3 * G[-1] - 4 * G[-2] + G[-3]) / (2 * h)
    for n, w in enumerate(wn):
        f = np.exp(1j * w * tau) * G
        s = h * (f.sum() - 0.5 * (f[0] + f[-1]))
        # derivative of e^{iw tau} G at the ends, e^{iw beta} = -1
        fp0 = 1j * w * G[0] + d0
        fpb = -(1j * w * G[-1] + db)
        out[n] = s - h * h / 12.0 * (fpb - fp0)
    return out


def bethe_update(G_iw, beta):
    wn = (2 * np.arange(G_iw.shape[0]) + 1) * np.pi / beta
    return np.array([1.0 / (1j * w - g) for w, g in zip(wn, G_iw)])
