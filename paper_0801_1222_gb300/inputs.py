"""Synthetic inputs for the HF-QMC sweep (shared by the tests, bench and smoke).

This module holds the input recipes only -- no step of the Monte Carlo method.
Both the CUDA library and the CPU oracle are fed the arrays it returns.

Benchmark model (the paper's "Benchmark results" section): the half-filled
one-band Hubbard model with a semi-elliptic density of states of bandwidth
W = 4 (hopping t = 1).  Before any DMFT iteration the bath is the
non-interacting one:

    G(iw) = (iw - i sgn(w) sqrt(w^2 + 4)) / 2,       G0(iw) = 1 / (iw - G(iw)),

which equals G(iw) itself for this lattice.  G0(tau) follows from the
Matsubara sum with the 1/(iw) and 1/(iw)^3 tails subtracted and added back
analytically (1/(iw) -> -1/2, 1/(iw)^3 -> tau (beta - tau) / 4 on 0 < tau < beta):

    G0(tau) = -1/2 + tau(beta - tau)/4
              + (2/beta) sum_{n>=0} Re[exp(-i w_n tau) (G0(iw_n) - 1/(iw_n) - 1/(iw_n)^3)].

Each dtau grid receives the Lambda samples G0(k dtau), k = 0..Lambda-1, with
G0_tau[0] = G0(0+) = -1/2.

Also here: the zero-hybridisation ("atomic limit") bath G0(tau) = -1/2, and the
five workload shapes (Lambda, U, beta, chains, sweeps) used by tests and bench.
"""
from __future__ import annotations

import numpy as np

N_MATSUBARA = 1 << 16


def bethe_G0_iw(iw: np.ndarray) -> np.ndarray:
    """Non-interacting bath of the W = 4 semicircle at half filling."""
    w = iw.imag
    G = 0.5 * (iw - 1j * np.sign(w) * np.sqrt(w * w + 4.0))
    return 1.0 / (iw - G)


def bethe_G0_at(beta: float, tau: np.ndarray, n_matsubara: int = N_MATSUBARA) -> np.ndarray:
    """Non-interacting Bethe bath G0(tau) at arbitrary 0 <= tau <= beta
    (tau = 0 means 0+, tau = beta means beta-)."""
    beta = float(beta)
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    n = np.arange(n_matsubara)
    wn = (2 * n + 1) * np.pi / beta
    iw = 1j * wn
    rest = bethe_G0_iw(iw) - 1.0 / iw - 1.0 / iw ** 3
    out = np.empty(tau.shape[0])
    chunk = 64
    for a in range(0, tau.shape[0], chunk):
        t = tau[a:a + chunk, None]
        ph = np.exp(-1j * wn[None, :] * t)
        out[a:a + chunk] = (2.0 / beta) * np.real(ph * rest[None, :]).sum(axis=1)
    out += -0.5 + tau * (beta - tau) / 4.0
    out[tau == 0.0] = -0.5
    out[tau == beta] = -0.5
    return out


def bethe_G0_tau(beta: float, L: int, n_matsubara: int = N_MATSUBARA) -> np.ndarray:
    """G0(tau_k), tau_k = k beta / L, k = 0..L-1 (physical sign, G0(0+) = -1/2)."""
    return bethe_G0_at(beta, np.arange(L) * (float(beta) / L), n_matsubara)


def atomic_G0_tau(L: int) -> np.ndarray:
    """Bath without hybridisation at half filling: G0(tau) = -1/2 on (0, beta)."""
    return np.full(L, -0.5)


def grid_size(beta: float, dtau: float) -> int:
    L = int(round(beta / dtau))
    if L < 1 or abs(beta / dtau - L) > 1e-9:
        raise ValueError(f"beta/dtau = {beta / dtau} is not an integer")
    return L


# Workload shapes of the paper's Mott-transition regime (U = 4..5.2,
# T = 1/8 .. 1/50, Bethe DOS).  Sweeps as (warm-up, measured).
WORKLOADS = {
    "single_L16": dict(U=[4.0], beta=8.0, L=[16], chains=[1], sweeps=(10_000, 100_000),
                       precision="f64"),
    "fixed_L100": dict(U=[5.0], beta=20.0, L=[100], chains=[256], sweeps=(1_000, 10_000),
                       precision="f32_delayed", k=16),
    "multigrid_L100_240": dict(U=[5.0], beta=40.0, L=[100, 120, 140, 160, 200, 240],
                               chains=[64] * 6, sweeps=(1_000, 10_000), precision="f32_delayed"),
    "large_L500": dict(U=[4.8], beta=50.0, L=[500], chains=[128], sweeps=(1_000, 10_000),
                       precision="f32_delayed", k=64, n_wrap=64),
    # the multigrid DMFT loop: four U values x six grids, 1024 chains (42 per
    # (U, dtau) pair, the 16 left over on the largest Lambda), 15 iterations;
    # sweeps (warm-up, measured) of the first and of the later iterations
    "dmft_c5": dict(U=[4.6, 4.8, 5.0, 5.2], beta=40.0, L=[80, 120, 160, 200, 240, 320],
                    chains=[42, 42, 42, 42, 42, 46], sweeps=(1_000, 10_000), sweeps_later=(200, 10_000),
                    iterations=15, precision="f32_delayed"),
}


def workload_grids(name: str):
    """(U, dtau, L, chains) for every grid of a named workload."""
    w = WORKLOADS[name]
    out = []
    for U in w["U"]:
        for L, c in zip(w["L"], w["chains"]):
            out.append((U, w["beta"] / L, L, c))
    return out
