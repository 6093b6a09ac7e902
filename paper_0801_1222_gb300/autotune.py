"""Per-Lambda tuning of the delay depth k and the recompute interval N_wrap on
the current GPU.

The FP32 delayed sweep has two free parameters per grid:
  * k, the accepted flips gathered into one rank-k flush: a larger k means
    fewer flushes of G but longer panel dot products per accepted flip and
    more shared memory (the library lowers a k whose panels or flush buffers
    do not fit);
  * N_wrap, the accepted flips between recomputes of G: a shorter interval
    costs more recomputes and keeps the FP32 drift smaller.
This module measures the sweep rate of every candidate (k, N_wrap) at each
Lambda on the GPU it runs on (Bethe bath of the benchmark model, the
library's recompute), and picks per Lambda the fastest candidate whose G(tau)
passes the accuracy criterion on a short calibration run: the FP32 run's
flips replayed by the FP64 rank-1 path (hfqmc_set_trace), chain-paired
difference of the measured G(tau) within 1e-5 + 3 sigma, sigma <= 3e-6.  It
returns the table that ``hfqmc_opts.tune_table`` takes: (Lambda_max, k,
n_wrap) triples.  The candidate intervals default to {16, 32, 64}, the
multigrid configuration's set.

Results can be cached in a JSON file keyed by the device name, its SM count
and the precision.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hfqmc, inputs

NWRAP_SET = (16, 32, 64)
TOL, SIG_MAX = 1e-5, 3e-6


def measure(Ls, beta=40.0, U=5.0, ks=(16, 24, 32), n_wraps=NWRAP_SET, chains=None, sweeps=40, seed=1):
    """Sweep rate (proposals/s) of every candidate at every Lambda:
    {L: {(k_effective, n_wrap): rate}} (the library may lower a requested k;
    the effective value is the key, the best rate kept).  The measurement
    starts from a fresh field after a few unmeasured sweeps."""
    import torch
    if chains is None:
        chains = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for L in Ls:
        g0 = inputs.bethe_G0_tau(beta, L)
        rates = {}
        for k in ks:
            for nw in n_wraps:
                ctx = hfqmc.HFQMC(beta, U, [beta / L], [chains], seed=seed, precision="f32_delayed", k=k,
                                  n_wrap=nw, drift_fail=1e30)
                try:
                    ctx.set_G0(0, g0)
                    ctx.sweep(0, max(2, sweeps // 8))
                    ctx.sweep(0, sweeps)
                    st = ctx.get_stats(0)
                    rate = L * chains * sweeps / (st["last_sweep_ms"] * 1e-3)
                    key = (int(st["k"]), int(nw))
                    rates[key] = max(rate, rates.get(key, 0.0))
                finally:
                    ctx.close()
        out[int(L)] = rates
    return out


def paired_error(L, k, n_wrap, beta=40.0, U=5.0, chains=16, n_warm=10, n_meas=120, seed=7):
    """(max_k |mean_c dG_c(tau_k)|, max_k sigma_paired) of the FP32 delayed run
    against the FP64 rank-1 run that replays its flips."""
    g0 = inputs.bethe_G0_tau(beta, L)
    S = n_warm + n_meas
    ctx = hfqmc.HFQMC(beta, U, [beta / L], [chains], seed=seed, precision="f32_delayed", k=k, n_wrap=n_wrap,
                      drift_fail=1e30)
    ref = hfqmc.HFQMC(beta, U, [beta / L], [chains], seed=seed, precision="f64_rank1", n_wrap=4096,
                      drift_fail=1e30)
    try:
        ctx.set_G0(0, g0)
        ctx.set_trace("record", S)
        ctx.sweep(n_warm, n_meas)
        ref.set_G0(0, g0)
        ref.set_trace("replay", S)
        ref.put_trace(0, ctx.get_trace(0, chains))
        ref.sweep(n_warm, n_meas)
        d = np.empty((chains, L))
        for c in range(chains):
            a, b = ctx.get_chain(0, c)["acc"], ref.get_chain(0, c)["acc"]
            d[c] = -((a[:L] + a[L:]) - (b[:L] + b[L:])) / (2.0 * n_meas)
    finally:
        ctx.close()
        ref.close()
    return float(np.max(np.abs(d.mean(0)))), float(np.max(d.std(0, ddof=1) / np.sqrt(chains)))


def passes(err) -> bool:
    dg, sig = err
    return sig <= SIG_MAX and dg <= TOL + 3.0 * sig


def table_from(measured, accuracy=None) -> list:
    """(Lambda_max, k, n_wrap) entries: for each measured Lambda (ascending)
    the fastest candidate (the smaller k, then the longer interval, on a tie)
    among those that pass the accuracy check when ``accuracy`` ({L: {(k,
    n_wrap): (dG, sigma)}}) has an entry for them; a grid takes the entry of
    the smallest measured Lambda >= its own (the last entry beyond)."""
    table = []
    for L in sorted(measured):
        rates = measured[L]
        order = sorted(rates, key=lambda c: (-rates[c], c[0], -c[1]))
        acc = (accuracy or {}).get(L, {})
        pick = next((c for c in order if c not in acc or passes(acc[c])), None)
        if pick is None:
            raise RuntimeError(f"no candidate at Lambda = {L} passes the G(tau) accuracy check")
        table.append((int(L), int(pick[0]), int(pick[1])))
    return table


def device_key(precision="f32_delayed") -> str:
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name}|sm{p.multi_processor_count}|{precision}"


def _enc(c):
    return f"{c[0]}:{c[1]}"


def _dec(s):
    k, nw = s.split(":")
    return int(k), int(nw)


def autotune(Ls, cache=None, key=None, check_accuracy=True, beta=40.0, U=5.0, **kw) -> list:
    """The tuning table for these Lambdas: from the JSON cache when it holds
    an entry for this device (and every Lambda), else measured (and stored).
    With check_accuracy the fastest candidate of each Lambda is calibrated
    (paired_error), and the next one tried while it fails."""
    key = key or device_key()
    Ls = sorted(int(L) for L in Ls)
    db = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            db = json.load(f)
    ent = db.get(key)
    if ent and all(str(L) in ent["rates"] for L in Ls):
        measured = {L: {_dec(c): v for c, v in ent["rates"][str(L)].items()} for L in Ls}
        accuracy = {L: {_dec(c): tuple(v) for c, v in ent.get("accuracy", {}).get(str(L), {}).items()} for L in Ls}
        return table_from(measured, accuracy)
    measured = measure(Ls, beta=beta, U=U, **kw)
    accuracy = {}
    if check_accuracy:
        for L in Ls:
            accuracy[L] = {}
            for c in sorted(measured[L], key=lambda c: (-measured[L][c], c[0], -c[1])):
                accuracy[L][c] = paired_error(L, c[0], c[1], beta=beta, U=U)
                if passes(accuracy[L][c]):
                    break
    if cache:
        ent = db.setdefault(key, {"rates": {}, "accuracy": {}})
        for L, r in measured.items():
            ent["rates"][str(L)] = {_enc(c): v for c, v in r.items()}
            ent.setdefault("accuracy", {})[str(L)] = {_enc(c): list(v) for c, v in accuracy.get(L, {}).items()}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return table_from(measured, accuracy)
