"""The measurement walk of the delayed sweep (G in HBM) keeps its bins in
registers: a warp walks a contiguous range of rows, lane t holds the slots
j = 128 c + 4 t + q, slot j holds bin (r - j) mod L after row r, and from one
row to the next every bin moves one slot up (slot L - 1 to slot 0): within a
lane by register shifts, across lanes by shuffles (lane 0 takes slot 127 of
lane 31, or slot L - 1).  Restated here lane by lane for 16 warps and checked
against the plain diagonal sums sum_l sgn G[(l + k) mod L][l]."""
import numpy as np
import pytest

NW, RB = 16, 4


def slot_walk(G):
    L = G.shape[0]
    part = np.zeros((NW, L))
    lastc, lastl = (L - 1) >> 7, ((L - 1) & 127) >> 2
    lanes = np.arange(32)
    below = (lanes + 31) & 31
    cols = 128 * np.arange(2)[None, :, None] + 4 * lanes[:, None, None] + np.arange(4)[None, None, :]
    valid = cols < L
    for warp in range(NW):
        rb, re = (warp * L) // NW, ((warp + 1) * L) // NW
        acc = np.zeros((32, 2, 4))
        for r in range(rb, re):
            if r > rb:
                t0 = acc[below, 0, 3]
                t1 = acc[below, 1, 3]
                t2 = np.full(32, acc[lastl, lastc, 3])
                acc[:, :, 1:] = acc[:, :, :3].copy()
                acc[:, 0, 0] = np.where(lanes > 0, t0, t2)
                acc[:, 1, 0] = np.where(lanes > 0, t1, t0)
            x = np.where(valid, G[r, np.minimum(cols, L - 1)], 0.0)
            acc += np.where(r >= cols, x, -x)
        if re > rb:
            k = (re - 1 - cols[valid]) % L
            part[warp, k] = acc[valid]
    return part.sum(axis=0)


def diagonal_sums(G):
    L = G.shape[0]
    r, l = np.indices((L, L))
    out = np.zeros(L)
    np.add.at(out, (r - l) % L, np.where(r >= l, G, -G))
    return out


@pytest.mark.parametrize("L", [4, 8, 16, 60, 100, 120, 128, 132, 160, 200, 240, 256])
def test_slot_walk_equals_diagonal_sums(L):
    G = np.random.default_rng(L).standard_normal((L, L))
    np.testing.assert_allclose(slot_walk(G), diagonal_sums(G), atol=1e-10)


def test_wrap_through_slot_L_minus_1_matters():
    # closing the ring through slot 255 instead of slot L - 1 is wrong
    # unless L = 256
    L = 240
    G = np.random.default_rng(7).standard_normal((L, L))
    good = slot_walk(G)
    Gp = np.zeros((256, 256))
    Gp[:L, :L] = G
    ring256 = slot_walk(Gp)[:L]
    assert not np.allclose(ring256, good)
    np.testing.assert_allclose(good, diagonal_sums(G), atol=1e-10)
