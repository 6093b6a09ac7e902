"""The panel form of the FP64 Gauss-Jordan inversion used by the delayed
sweep and the initialisation, restated step by step in numpy and checked
against the library inverse: implicit pivoting (rows never move, the pivot of
column k is the largest |entry| among the rows not used yet, ties to the
lowest row), each panel of b columns reduced on its own, the other columns
updated once per panel by x <- x + (V - E) x_P, and the result read out as
(B^-1)_{km} = B'_{p_k, pos(m)}.  The GPU kernel runs the same steps; its
results are held to the oracle's LU solve on the GPU."""
import numpy as np
import pytest


def panel_inverse(B, b):
    B = np.array(B, dtype=np.float64)
    L = B.shape[0]
    pos = -np.ones(L, dtype=int)
    perm = np.zeros(L, dtype=int)
    for k0 in range(0, L, b):
        bb = min(b, L - k0)
        pan = B[:, k0:k0 + bb].copy()
        for t in range(bb):
            k = k0 + t
            free = np.flatnonzero(pos < 0)
            mags = np.abs(pan[free, t])
            p = free[np.flatnonzero(mags == mags.max())[0]]
            perm[k], pos[p] = p, k
            inv = 1.0 / pan[p, t]
            row = pan[p] * inv
            row[t] = inv
            for i in range(L):
                if i != p:
                    c = pan[i, t]
                    pan[i] -= c * row
                    pan[i, t] = -c * inv
            pan[p] = row
        rest = [j for j in range(L) if not k0 <= j < k0 + bb]
        slab = B[perm[k0:k0 + bb]][:, rest]
        pivots = (pos >= k0) & (pos < k0 + bb)
        upd = pan @ slab
        B[np.ix_(~pivots, rest)] += upd[~pivots]
        B[np.ix_(pivots, rest)] = upd[pivots]
        B[:, k0:k0 + bb] = pan
    return B[np.ix_(perm, pos)]


@pytest.mark.parametrize("L,b", [(1, 16), (5, 16), (16, 16), (37, 16), (40, 4), (64, 16)])
def test_panel_inverse_matches_inverse(L, b):
    rng = np.random.default_rng(L * 7 + b)
    A = rng.standard_normal((L, L)) + 0.5 * np.eye(L)
    G = panel_inverse(A, b)
    np.testing.assert_allclose(G @ A, np.eye(L), atol=1e-9)


def test_panel_inverse_needs_pivoting():
    # a zero leading entry: without pivoting the first step would divide by 0
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    np.testing.assert_allclose(panel_inverse(A, 2), np.linalg.inv(A), atol=1e-14)


def test_panel_width_does_not_change_the_inverse():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((48, 48)) + 0.5 * np.eye(48)
    ref = panel_inverse(A, 1)
    for b in (4, 16, 48):
        np.testing.assert_allclose(panel_inverse(A, b), ref, atol=1e-10)
