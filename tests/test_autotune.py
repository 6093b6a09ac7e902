"""The per-Lambda tuning table: validation in the C ABI (host side, no GPU),
the table built from measured rates and its JSON cache (host side, with a
stand-in measurement), and a short tuning run on the GPU whose table the
library then applies."""
import ctypes
import json

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_0801_1222_gb300 import build, hfqmc
    build.build()
    return hfqmc


def _opts_with_table(lib, rows):
    o = lib.hfqmc_default_opts()
    flat = [v for r in rows for v in r]
    arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    o.tune_table = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int))
    o.tune_entries = len(rows)
    return o, arr


@pytest.mark.parametrize("rows,what", [
    ([(64, 12, 8192)], "multiple of 8"),            # k not a multiple of 8
    ([(64, 16, 0)], "n_wrap"),                      # n_wrap 0
    ([(128, 16, 8192), (64, 16, 8192)], "increasing"),
    ([(0, 16, 8192)], "Lambda_max"),
])
def test_bad_tables_are_rejected_before_the_device(lib, rows, what):
    o, keep = _opts_with_table(lib, rows)
    with pytest.raises(lib.HFQMCError) as ei:
        lib.hfqmc_create(8.0, 4.0, [0.5], [1], opts=o)
    assert ei.value.name == "EINVAL" and what in str(ei.value)


def test_negative_entry_count_rejected(lib):
    o = lib.hfqmc_default_opts()
    o.tune_entries = -1
    with pytest.raises(lib.HFQMCError) as ei:
        lib.hfqmc_create(8.0, 4.0, [0.5], [1], opts=o)
    assert ei.value.name == "EINVAL"


def test_table_from_measured_rates():
    from paper_0801_1222_gb300 import autotune
    measured = {240: {(8, 64): 1.0e8, (16, 64): 1.2e8, (16, 32): 1.1e8},
                100: {(16, 64): 2.2e8, (24, 64): 2.3e8, (32, 64): 2.3e8, (24, 16): 1.9e8}}
    # ascending Lambda; the fastest (k, n_wrap), the smaller k on a tie
    assert autotune.table_from(measured) == [(100, 24, 64), (240, 16, 64)]
    # a candidate that fails the G(tau) check is passed over for the next fastest
    acc = {240: {(16, 64): (2e-5, 1e-7), (16, 32): (1e-9, 1e-10)}}
    assert autotune.table_from(measured, acc) == [(100, 24, 64), (240, 16, 32)]
    with pytest.raises(RuntimeError):
        autotune.table_from({240: {(16, 64): 1.0}}, {240: {(16, 64): (1.0, 1e-7)}})


def test_accuracy_criterion():
    from paper_0801_1222_gb300 import autotune
    assert autotune.passes((9e-6, 1e-8))
    assert autotune.passes((1.2e-5, 1e-6))        # within 1e-5 + 3 sigma
    assert not autotune.passes((2e-5, 1e-6))
    assert not autotune.passes((0.0, 4e-6))       # sigma too large to resolve 1e-5


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_0801_1222_gb300 import autotune
    calls, checks = [], []

    def fake_measure(Ls, **kw):
        calls.append(list(Ls))
        return {L: {(16, 64): 1.0, (24, 64): 2.0 if L < 150 else 0.5, (24, 32): 1.5} for L in Ls}

    def fake_paired(L, k, nw, **kw):
        checks.append((L, k, nw))
        return (3e-5, 1e-7) if (L, k, nw) == (120, 24, 64) else (1e-9, 1e-10)

    monkeypatch.setattr(autotune, "measure", fake_measure)
    monkeypatch.setattr(autotune, "paired_error", fake_paired)
    cache = str(tmp_path / "tune.json")
    t1 = autotune.autotune([120, 200], cache=cache, key="dev|sm1|f32_delayed")
    t2 = autotune.autotune([200, 120], cache=cache, key="dev|sm1|f32_delayed")
    # Lambda 120: (24, 64) fastest but fails its check -> (24, 32); Lambda 200: (24, 32)
    assert t1 == t2 == [(120, 24, 32), (200, 24, 32)]
    assert calls == [[120, 200]]                       # the second call read the cache
    assert checks == [(120, 24, 64), (120, 24, 32), (200, 24, 32)]
    db = json.load(open(cache))
    assert set(db["dev|sm1|f32_delayed"]["rates"]) == {"120", "200"}
    autotune.autotune([120, 160], cache=cache, key="dev|sm1|f32_delayed")
    assert calls[-1] == [120, 160]                     # a new Lambda: measured again


@pytest.mark.gpu
def test_gpu_tuning_run_and_the_table_applied():
    from gpu_common import lib as glib
    from paper_0801_1222_gb300 import autotune, inputs
    h = glib()
    measured = autotune.measure([40, 80], beta=8.0, U=4.0, ks=(8, 16), n_wraps=(32, 64), chains=16, sweeps=8)
    assert set(measured) == {40, 80} and all(len(r) >= 2 for r in measured.values())
    err = autotune.paired_error(80, 16, 64, beta=8.0, U=4.0, chains=8, n_warm=2, n_meas=20)
    assert autotune.passes(err), err
    table = autotune.table_from(measured)
    ctx = h.HFQMC(8.0, 4.0, [8.0 / 40, 8.0 / 80], [4, 4], precision="f32_delayed", tune=table,
                  drift_fail=1.0)
    for g, L in enumerate((40, 80)):
        ctx.set_G0(g, inputs.bethe_G0_tau(8.0, L))
    ctx.sweep(1, 2)
    for g, (L, k, nw) in enumerate(table):
        st = ctx.get_stats(g)
        assert st["k"] == k and st["n_wrap"] == nw
    ctx.close()
    # autotune off: fixed k = 16, n_wrap = 1024
    ctx = h.HFQMC(8.0, 4.0, [0.2], [2], precision="f32_delayed", autotune=False, drift_fail=1.0)
    st = ctx.get_stats(0)
    assert st["k"] == 16 and st["n_wrap"] == 1024
    ctx.close()
