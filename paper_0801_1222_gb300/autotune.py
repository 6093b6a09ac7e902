"""Per-Lambda tuning of the delay depth k on the current GPU.

The FP32 delayed sweep has one free performance parameter per grid: the
delay depth k (accepted flips gathered into one rank-k flush).  A larger k
means fewer flushes of G but longer panel dot products per accepted flip and
more shared memory (k is lowered by the library when the panels or the flush
buffers do not fit).  This module measures the sweep rate of each candidate k
at each Lambda on the GPU it runs on and returns the table that
``hfqmc_opts.tune_table`` takes: (Lambda_max, k, n_wrap) triples.

N_wrap is not tuned here: it is an accuracy choice (the FP32 G(tau) has to
stay within 1e-5 of FP64 on top of the statistical error), so the table keeps
the validated values, 8192 accepted flips for Lambda <= 128 and 16384 above.

The measurement uses the Bethe bath of the benchmark model and n_wrap = -1
(no recompute), so that only k changes the work.  Results can be cached in a
JSON file keyed by the device name, its SM count and the precision.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hfqmc, inputs


def validated_n_wrap(L: int) -> int:
    """The recompute interval validated against the G(tau) accuracy criterion."""
    return 8192 if L <= 128 else 16384


def measure(Ls, beta=40.0, U=5.0, ks=(8, 16, 24, 32), chains=None, sweeps=40, seed=1):
    """Sweep rate (proposals/s) of every candidate k at every Lambda:
    {L: {k_effective: rate}} (the library may lower a requested k; the
    effective value is the key, the best rate kept)."""
    import torch
    if chains is None:
        chains = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for L in Ls:
        g0 = inputs.bethe_G0_tau(beta, L)
        rates = {}
        for k in ks:
            ctx = hfqmc.HFQMC(beta, U, [beta / L], [chains], seed=seed, precision="f32_delayed", k=k,
                              n_wrap=-1, drift_fail=1e30)
            try:
                ctx.set_G0(0, g0)
                ctx.sweep(0, max(2, sweeps // 8))
                ctx.sweep(0, sweeps)
                st = ctx.get_stats(0)
                rate = L * chains * sweeps / (st["last_sweep_ms"] * 1e-3)
                keff = int(st["k"])
                rates[keff] = max(rate, rates.get(keff, 0.0))
            finally:
                ctx.close()
        out[int(L)] = rates
    return out


def table_from(measured) -> list:
    """(Lambda_max, k, n_wrap) entries from measure()'s result: for each
    measured Lambda (ascending) the fastest k; a grid takes the entry of the
    smallest measured Lambda >= its own (the last entry beyond)."""
    table = []
    for L in sorted(measured):
        rates = measured[L]
        k = max(rates, key=lambda kk: (rates[kk], -kk))
        table.append((int(L), int(k), validated_n_wrap(int(L))))
    return table


def device_key(precision="f32_delayed") -> str:
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name}|sm{p.multi_processor_count}|{precision}"


def autotune(Ls, cache=None, key=None, **kw) -> list:
    """The tuning table for these Lambdas: from the JSON cache when it holds
    an entry for this device (and every Lambda), else measured (and stored)."""
    key = key or device_key()
    Ls = sorted(int(L) for L in Ls)
    db = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            db = json.load(f)
    ent = db.get(key)
    if ent and all(str(L) in ent["rates"] for L in Ls):
        measured = {L: {int(k): v for k, v in ent["rates"][str(L)].items()} for L in Ls}
        return table_from(measured)
    measured = measure(Ls, **kw)
    if cache:
        ent = db.setdefault(key, {"rates": {}})
        for L, r in measured.items():
            ent["rates"][str(L)] = {str(k): v for k, v in r.items()}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return table_from(measured)
