"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/hfqmc.h declares, and rejects bad arguments
before touching the device."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_0801_1222_gb300 import build, hfqmc
    build.build()
    return hfqmc


def test_exports_every_declared_symbol(lib):
    names = lib.header_functions()
    assert {"hfqmc_create", "hfqmc_set_G0", "hfqmc_sweep", "hfqmc_get_G"} <= set(names)
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n


def test_default_opts(lib):
    o = lib.hfqmc_default_opts()
    assert o.precision == lib.PRECISION["f32_delayed"]
    assert o.accept_rule == 0 and o.use_graph == 1 and o.drift_fail == 1e-1


@pytest.mark.parametrize("beta,dtau,chains,what", [
    (8.0, [0.33], [1], "integer"),
    (-1.0, [0.5], [1], "beta"),
    (8.0, [0.5], [0], "chains"),
    (8.0, [8.0 / 2000], [1], "integer Lambda in [1, 1024]"),
])
def test_create_rejects_bad_arguments(lib, beta, dtau, chains, what):
    with pytest.raises(lib.HFQMCError) as ei:
        lib.hfqmc_create(beta, 4.0, dtau, chains)
    assert ei.value.name == "EINVAL" and what in str(ei.value)


def test_bad_k_rejected(lib):
    o = lib.hfqmc_default_opts()
    o.k = 12
    with pytest.raises(lib.HFQMCError) as ei:
        lib.hfqmc_create(8.0, 4.0, [0.5], [1], opts=o)
    assert ei.value.name == "EINVAL"


def test_null_ctx_calls_fail_cleanly(lib):
    so = lib.load()
    assert so.hfqmc_sweep(None, 1, 1) == -1
    assert so.hfqmc_set_G0(None, 0, None) == -1
    so.hfqmc_destroy(None)
    assert b"NULL" in so.hfqmc_last_error(None)


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_0801_1222_gb300 import hfqmc
    monkeypatch.setattr(hfqmc, "_lib", None)
    monkeypatch.setattr(hfqmc, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        hfqmc.load()


def test_trace_and_chain_calls_reject_a_null_context(lib):
    so = lib.load()
    assert so.hfqmc_set_trace(None, 1, 10) == -1
    assert so.hfqmc_get_trace(None, 0, None, 0) == -1
    assert so.hfqmc_put_trace(None, 0, None, 0) == -1
    assert so.hfqmc_get_chain_D(None, 0, 0, None, None) == -1
