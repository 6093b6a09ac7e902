"""The arithmetic of the Newton-refinement recompute (hfq_refine.cuh, the
slice table of hfq_setup's k_refine_prep), restated in numpy with exact
integers, against the FP64 residual and inverse of the Hirsch-Fye Dyson
equation built by the oracle.

The steps restated, for one spin and field:
  * A = M^{-1} - diag(1 - e^{-sigma lambda s_j}), cut into six signed 7-bit
    slices under one scale 2^ea (rint of the running remainder times 2^7);
  * H = fl32(fl32(e^{sigma lambda s_j}) G_jn) and H' = rint(H 2^{28-eh})
    2^{eh-28}, which equals the sum of its four 7-bit slices;
  * the products of slices p, q with p + q = l summed over the contraction
    index (a tensor core's FP32 accumulation: every partial sum an integer
    below 2^24 in magnitude), the six level sums combined as
    V = sum_l S_l 2^{7(5-l)} and E = delta 2^{sh} - V, sh = 49 - ea - eh;
  * G_new = e^{-sigma lambda s_j} (H' + H' E).
It checks the partial-sum bound that makes the accumulation exact, that E
matches 1 - B G' to ~1e-10 of the terms, and that one step from a drifted G
lands on the FP64 inverse to within a few FP32 roundings."""
import numpy as np
import pytest

BITS, SA, SH, LEVELS = 7, 6, 4, 6


def slices(x, scale_exp, n):
    """Signed 7-bit slices of x / 2^scale_exp (|x| < 2^scale_exp), as the kernels cut them."""
    y = np.ldexp(np.asarray(x, dtype=np.float64), BITS - scale_exp)
    out = []
    for _ in range(n):
        r = np.rint(y)
        out.append(r)
        y = (y - r) * (1 << BITS)
    return out


def refine_step(Minv, G32, s, lam, sig):
    """One Newton step in the kernel's order; returns (G_new, E, E_exact, partial-sum max)."""
    L = G32.shape[0]
    v = np.where(sig * s > 0, 0, 1)
    a = Minv[0, 0] - (1.0 - np.exp(-lam * np.array([1.0, -1.0])))  # A_jj for v = 0, 1
    A = Minv.copy()
    A[np.arange(L), np.arange(L)] = a[v]
    m = max(np.abs(Minv[:, 0]).max(), np.abs(a).max())
    ea = int(np.frexp(m)[1])
    assert m < 2.0 ** ea
    As = slices(Minv, ea, SA)
    ds = slices(a, ea, SA)
    for p in range(SA):
        As[p][np.arange(L), np.arange(L)] = ds[p][v]
    cplus = np.array([np.float32(np.exp(lam)), np.float32(np.exp(-lam))])
    H = (G32.astype(np.float32) * cplus[v][:, None].astype(np.float32)).astype(np.float64)
    eh = int(np.frexp(np.abs(H).max())[1])
    Hs = slices(H, eh, SH)
    Hp = np.rint(np.ldexp(H, 28 - eh)) * 2.0 ** (eh - 28)
    assert np.array_equal(sum(Hs[q] * 2.0 ** (eh - BITS * (q + 1)) for q in range(SH)), Hp)
    # level sums with every partial sum along the contraction index
    S = []
    pmax = 0
    for lv in range(LEVELS):
        terms = [(p, lv - p) for p in range(SA) if 0 <= lv - p < SH]
        prod = sum(As[p].astype(np.int64)[:, :, None] * Hs[q].astype(np.int64)[None, :, :] for p, q in terms)
        part = np.cumsum(prod, axis=1)
        pmax = max(pmax, int(np.abs(part).max()))
        S.append(part[:, -1, :])
    V = np.zeros((L, L), dtype=object)
    for lv in range(LEVELS):
        V = V * (1 << BITS) + S[lv].astype(object)
    sh = 49 - ea - eh
    Eint = np.where(np.eye(L, dtype=bool), 1 << sh, 0).astype(object) - V
    E = np.array([[float(x) for x in row] for row in Eint]) * 2.0 ** -sh
    # the FP64 residual of G' = (1 + D)^{-1} H' for the same B
    d = np.exp(sig * lam * s) - 1.0
    B = Minv * (1.0 + d)[None, :] - np.diag(d)
    Gp = Hp / (1.0 + d)[:, None]
    E_exact = np.eye(L) - B @ Gp
    cminus = np.exp(-sig * lam * s)
    G_new = (cminus[:, None] * (Hp + Hp @ E.astype(np.float32).astype(np.float64))).astype(np.float32)
    return G_new.astype(np.float64), E, E_exact, pmax, B


@pytest.fixture(scope="module")
def chain(orc):
    from paper_0801_1222_gb300 import inputs
    beta, U, L = 20.0, 5.0, 64
    M = orc.bath_matrix(inputs.bethe_G0_tau(beta, L))
    lam = orc.lam(beta / L, U)
    ch = orc.Chain.new(M, lam, 1, 0, 0)
    orc.run_chain(ch, 30, 0, n_wrap=16)
    return M, lam, ch


@pytest.mark.parametrize("sig", [1, -1])
def test_newton_step_from_a_drifted_G_lands_on_the_fp64_inverse(chain, sig):
    M, lam, ch = chain
    G = ch.Gup if sig == 1 else ch.Gdn
    Minv = np.linalg.inv(M)
    rng = np.random.default_rng(3)
    drifted = G + 1e-5 * np.abs(G).max() * rng.standard_normal(G.shape) / np.sqrt(G.shape[0])
    G_new, E, E_exact, pmax, B = refine_step(Minv, drifted.astype(np.float32).astype(np.float64), ch.s, lam,
                                             sig)
    assert pmax < 2 ** 24                      # exact FP32 accumulation of every level
    assert 1e-6 < np.abs(E).max() < 2.0 ** -8  # a step is taken, and it is needed
    assert np.abs(E - E_exact).max() < 1e-9
    G_exact = np.linalg.inv(B)
    rounding = np.abs(G_exact.astype(np.float32).astype(np.float64) - G_exact).max()
    assert np.abs(G_new - G_exact).max() <= 4 * rounding


def test_partial_sum_bound_at_the_largest_slices():
    """Worst case: every slice at its largest magnitude (128 for the first,
    64 after) with equal signs, contraction length 512.  The level sums stay
    below 2^24, so FP32 accumulates them exactly."""
    K = 512
    worst = 0
    for lv in range(LEVELS):
        t = sum((128 if p == 0 else 64) * (128 if lv - p == 0 else 64)
                for p in range(SA) if 0 <= lv - p < SH)
        worst = max(worst, t * K)
    assert worst < 2 ** 24


def test_h_prime_equals_its_slices_at_ties():
    """rint(H 2^{28-eh}) 2^{eh-28} (the kernels' H' in the update) equals the
    sum of the four slices (the residual's H'), ties included."""
    rng = np.random.default_rng(5)
    eh = 5
    H = rng.uniform(-32, 32, 20000).astype(np.float32).astype(np.float64)
    ties = (np.arange(-2000, 2000) + 0.5) * 2.0 ** (eh - 28)
    H = np.concatenate([H, ties, ties * 3, [31.999999, -31.999999, 0.0]])
    Hs = slices(H, eh, SH)
    direct = np.rint(np.ldexp(H, 28 - eh)) * 2.0 ** (eh - 28)
    assert np.array_equal(sum(Hs[q] * 2.0 ** (eh - BITS * (q + 1)) for q in range(SH)), direct)
    assert all(np.abs(Hs[0]).max() <= 128 and np.abs(Hs[q]).max() <= 64 for q in range(1, SH))


def test_rounding_to_fp16_by_magic_constant():
    """The H' slicing's rounding (hfq_refine.cuh rf_round_h2), restated in
    numpy: in FP32, y + 1.5 * 2^23 - 1.5 * 2^23 is the nearest integer of y
    (ties to even) for |y| <= 2^7; the integer is the FP32 sum's bit pattern
    minus that of 1.5 * 2^23; 0x6600 + v are the FP16 bits of 1536 + v, and
    1536 subtracted in FP16 leaves v.  Every multiple of 1/64 in [-128, 128]
    (ties included) against numpy's rint and float16 (as values: rint keeps
    the sign of a zero, the subtraction gives +0; the products are the same)."""
    y = (np.arange(-128 * 64, 128 * 64 + 1) / 64.0).astype(np.float32)
    magic = np.float32(12582912.0)
    t = (y + magic).astype(np.float32)
    r = (t - magic).astype(np.float32)
    np.testing.assert_array_equal(r, np.rint(y))
    v = t.view(np.int32).astype(np.int64) - 0x4B400000
    np.testing.assert_array_equal(v, np.rint(y).astype(np.int64))
    bits = ((0x6600 + v) & 0xFFFF).astype(np.uint16)
    h = (bits.view(np.float16) - np.float16(1536.0)).astype(np.float16)
    np.testing.assert_array_equal(h.astype(np.float64), np.rint(y))
    nz = np.rint(y) != 0
    np.testing.assert_array_equal(h.view(np.uint16)[nz], np.rint(y).astype(np.float16).view(np.uint16)[nz])
