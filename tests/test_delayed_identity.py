"""The delayed (rank-k) form of the Hirsch-Fye update, restated in numpy and
checked against the rank-1 form it replaces: after j accepted flips the
current Green matrix is G + U W^T, an accepted flip at slice l appends
u = G_cur[:, l] - e_l and w = (Delta / R) G_cur[l, :] (each entry the base
entry plus a length-j dot product with the panels), and a flush adds U W^T
to G.  In exact arithmetic this is the rank-1 update applied flip by flip;
in FP64 the two agree to rounding.  The sweep kernels use this identity
(FP32 panels, tensor-core flush); their decisions and G are held to the
oracle on the GPU."""
import numpy as np
import pytest

import oracle


def rank1(G, l, f):
    col = G[:, l].copy()
    col[l] -= 1.0
    return G + np.outer(col, f * G[l, :])


def delayed(G, flips, k):
    L = G.shape[0]
    U = np.zeros((L, 0))
    W = np.zeros((L, 0))
    for l, f in flips:
        col = G[:, l] + U @ W[l, :]
        row = G[l, :] + U[l, :] @ W.T
        u = col.copy()
        u[l] -= 1.0
        U = np.hstack([U, u[:, None]])
        W = np.hstack([W, (f * row)[:, None]])
        if U.shape[1] == k:
            G = G + U @ W.T
            U = np.zeros((L, 0))
            W = np.zeros((L, 0))
    return G + U @ W.T


@pytest.mark.parametrize("k", [1, 3, 8, 32])
def test_delayed_equals_rank1(k):
    from paper_0801_1222_gb300 import inputs
    beta, U_, L = 4.0, 3.0, 20
    lam = np.arccosh(np.exp(beta / L * U_ / 2))
    q = oracle.OracleHFQMC(beta, [(U_, beta / L)], [1], seed=3, n_wrap=1 << 30)
    q.set_G0(0, inputs.bethe_G0_tau(beta, L))
    G = q.chains[0][0].Gup.copy()
    s = q.chains[0][0].s.astype(int).copy()
    rng = np.random.default_rng(k)
    flips = []
    Gr = G.copy()
    for _ in range(45):
        l = int(rng.integers(L))
        d = np.exp(-2 * lam * s[l]) - 1.0  # spin up
        R = 1.0 + (1.0 - Gr[l, l]) * d
        flips.append((l, d / R))
        Gr = rank1(Gr, l, d / R)
        s[l] = -s[l]
    Gd = delayed(G, flips, k)
    assert np.max(np.abs(Gd - Gr)) < 1e-9 * max(1.0, np.abs(Gr).max())
