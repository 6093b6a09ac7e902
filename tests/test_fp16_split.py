"""The delayed flush's operand split, restated in numpy: each panel (U or W
of one spin) is scaled by 2^(141 - E), E the largest biased FP32 exponent in
it, so that its largest magnitude lies in [2^14, 2^15); every scaled entry x
is split into hi = fp16(x) and lo = fp16(x - hi) (round to nearest); the
tensor cores form hi*hi + hi*lo + lo*hi, and the scaling is undone by a
power of two.  The product then carries the split's relative error
(~2^-21 per term, as a TF32 split would), whatever the panels' magnitudes:
no FP16 overflow, and the subnormal range only below 2^-29 of a panel's
largest entry."""
import numpy as np
import pytest


def scale_exponent(P):
    bits = np.abs(P.astype(np.float32)).view(np.uint32)
    E = int((bits >> 23).max())
    return 0 if E == 0 else min(141 - E, 127)


def split(P, a):
    x = (P.astype(np.float32) * np.float32(2.0 ** a)).astype(np.float32)
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float64), lo.astype(np.float64)


def flush_product(U, W):
    aU, aW = scale_exponent(U), scale_exponent(W)
    uh, ul = split(U, aU)
    wh, wl = split(W, aW)
    return (uh @ wh.T + uh @ wl.T + ul @ wh.T) * 2.0 ** -(aU + aW)


@pytest.mark.parametrize("scale_u,scale_w", [(1.0, 1.0), (17.0, 200.0), (1e-3, 1e4), (1e-30, 1e-20), (3e4, 3e4)])
def test_split_product_error(scale_u, scale_w):
    rng = np.random.default_rng(int(scale_u * 1e3) % 97 + 5)
    L, k = 96, 16
    # magnitudes spread over six decades inside each panel
    U = (rng.standard_normal((L, k)) * 10.0 ** rng.uniform(-6, 0, (L, k)) * scale_u).astype(np.float32)
    W = (rng.standard_normal((L, k)) * 10.0 ** rng.uniform(-6, 0, (L, k)) * scale_w).astype(np.float32)
    exact = U.astype(np.float64) @ W.astype(np.float64).T
    got = flush_product(U, W)
    assert np.all(np.isfinite(got))
    bound = np.abs(U.astype(np.float64)) @ np.abs(W.astype(np.float64)).T
    # 3 * 2^-22 per term from the two roundings of lo and the dropped lo*lo,
    # plus the subnormal floor relative to the panels' largest entries
    floor = 2.0 ** -38 * np.abs(U).max() * np.abs(W).max() * k
    assert np.all(np.abs(got - exact) <= 3 * 2.0 ** -22 * bound + floor)


def test_zero_panel_has_scale_one_and_adds_zero():
    U = np.ones((8, 4), np.float32)
    W = np.zeros((8, 4), np.float32)
    assert scale_exponent(W) == 0
    assert np.all(flush_product(U, W) == 0.0)


def test_scaled_largest_entry_below_fp16_max():
    rng = np.random.default_rng(1)
    for mag in (1e-12, 1.0, 7.0, 1e9):
        P = (rng.standard_normal((32, 8)) * mag).astype(np.float32)
        a = scale_exponent(P)
        top = np.abs(P).max() * 2.0 ** a
        assert 2.0 ** 14 <= top < 2.0 ** 15
        hi, lo = split(P, a)
        assert np.all(np.isfinite(hi)) and np.all(np.isfinite(lo))


def test_without_scaling_the_split_fails():
    # the same split with the scale exponents forced to 0: large panels
    # overflow FP16, small ones fall into its subnormal range
    rng = np.random.default_rng(2)
    for mag in (3e4, 1e-6):
        U = (rng.standard_normal((64, 16)) * mag).astype(np.float32)
        W = (rng.standard_normal((64, 16)) * mag).astype(np.float32)
        with np.errstate(over="ignore", invalid="ignore"):
            uh, ul = split(U, 0)
            wh, wl = split(W, 0)
            got = uh @ wh.T + uh @ wl.T + ul @ wh.T
            exact = U.astype(np.float64) @ W.astype(np.float64).T
            bound = np.abs(U.astype(np.float64)) @ np.abs(W.astype(np.float64)).T
            ok = np.isfinite(got) & (np.abs(got - exact) <= 3 * 2.0 ** -22 * bound)
        assert not np.all(ok)
