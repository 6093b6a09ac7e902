"""Philox4x32-10 pinned from outside this repository: cuRAND's header-only
device function curand_Philox4x32_10 (a library implementation of the same
published generator, Salmon et al., SC'11) against the generator the sweep
kernels use and the CPU oracle's independently written one, bit for bit, on
10^5 counters under several keys; and the 53-bit proposal uniform of the
sweep against the oracle's, on the same outputs.

A wrong round multiplier, a swapped output word or a wrong key schedule in
either of this repository's two implementations would show here, which the
statistical checks of tests/test_oracle_philox.py cannot promise."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = [0, 1, 0xFFFFFFFF, 0x9E3779B97F4A7C15, 0x0123456789ABCDEF, (1 << 64) - 1]


def _probe():
    import build_probe
    from gpu_common import require_cuda
    require_cuda()
    lib = ctypes.CDLL(build_probe.build())
    P = ctypes.c_void_p
    lib.philox_probe.argtypes = [P, P, ctypes.c_int, P, P, P]
    lib.philox_probe.restype = ctypes.c_int
    return lib


def _counters(n, rng):
    c = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[:64] = 0                                     # edge words: zeros, all-ones, the proposal shape
    c[64:128] = 0xFFFFFFFF
    c[128:256, 0] = np.arange(128)                 # slice l, sweep, chain, grid as in the sweep
    c[128:256, 1] = 7
    c[128:256, 2] = 3
    c[128:256, 3] = 1
    return np.ascontiguousarray(c)


def test_philox_matches_curand_and_oracle(orc):
    lib = _probe()
    rng = np.random.default_rng(2024)
    n = 100_000
    for key in KEYS:
        c = _counters(n, rng)
        k = np.full(n, key, dtype=np.uint64)
        out_lib = np.empty((n, 4), dtype=np.uint32)
        out_hfq = np.empty((n, 4), dtype=np.uint32)
        u = np.empty(n)
        rc = lib.philox_probe(c.ctypes.data, k.ctypes.data, n, out_lib.ctypes.data,
                              out_hfq.ctypes.data, u.ctypes.data)
        assert rc == 0, rc
        np.testing.assert_array_equal(out_hfq, out_lib)
        np.testing.assert_array_equal(orc.philox(c, key), out_lib)
        # the 53-bit uniform: ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53, exact in FP64
        x0 = out_lib[:, 0].astype(np.uint64) >> np.uint64(5)
        x1 = out_lib[:, 1].astype(np.uint64) >> np.uint64(6)
        ref = ((x0 << np.uint64(26)) + x1).astype(np.float64) * 2.0 ** -53
        np.testing.assert_array_equal(u, ref)
        assert np.all((u >= 0.0) & (u < 1.0))
        for i in range(128, 160):  # the oracle's proposal uniform on the sweep's counters
            l, t, ch, g = (int(v) for v in c[i])
            assert orc.uniform(l, t, ch, g, key) == u[i]
