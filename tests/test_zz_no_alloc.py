"""hfqmc_green_noalloc: the Green-function entry point for callers that may
not allocate device memory.  Its output must equal, within the FP64 parity
tolerance of the other tests (1e-10 relative), the Green matrices the regular
entry points build for the same field (hfqmc_set_G0 + hfqmc_get_chain), on
two calls in a row that share the library's static scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_regular_entry_points_twice():
    import torch

    from paper_0801_1222_gb300 import build, hfqmc, inputs
    build.build()
    assert torch.cuda.is_available()
    beta, U, L = 20.0, 5.0, 100
    g0 = inputs.bethe_G0_tau(beta, L)
    ctx = hfqmc.HFQMC(beta, U, [beta / L], [2], seed=7, precision="f64_rank1")
    ctx.set_G0(0, g0)
    ref = [ctx.get_chain(0, c) for c in range(2)]
    ctx.close()
    g0_d = _dev(g0)
    for c in range(2):  # two calls in a row on the shared scratch
        s_d = _dev(ref[c]["s"])
        gu = torch.empty((L, L), dtype=torch.float64, device="cuda")
        gd = torch.empty((L, L), dtype=torch.float64, device="cuda")
        st = hfqmc.hfqmc_green_noalloc(g0_d.data_ptr(), s_d.data_ptr(), L, beta / L, U,
                                       gu.data_ptr(), gd.data_ptr(), 0)
        assert st == 0
        for G, R in ((gu.cpu().numpy(), ref[c]["Gup"]), (gd.cpu().numpy(), ref[c]["Gdn"])):
            scale = np.abs(R).max()
            assert np.max(np.abs(G - R)) <= 1e-10 * scale


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_0801_1222_gb300 import hfqmc
    L = hfqmc.NOALLOC_MAX_L + 1
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(hfqmc.HFQMCError) as ei:
        hfqmc.hfqmc_green_noalloc(buf.data_ptr(), buf.data_ptr(), L, 0.1, 4.0, buf.data_ptr(),
                                  buf.data_ptr(), 0)
    assert ei.value.name == "EINVAL"
