"""Plain FP64 CPU oracle for the Hirsch-Fye QMC sweep (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports it, and it never
imports the product: both sides are fed the same G0(tau) samples and seed.

The arithmetic lives in ``hfqmc_oracle.c`` (compiled with -ffp-contract=off);
this module compiles it with gcc, loads it with ctypes and adds the host steps
of the paper's impurity solve:

* ``OracleHFQMC`` -- the same call sequence as the C ABI (create, set_G0,
  sweep, get_G, stats): fixed-bath HF-QMC on several dtau grids with several
  independent chains per grid ("Multigrid HF-QMC method" section: 10-20
  impurity solutions per dtau, averaged).
* ``brute_force`` -- exact discrete-dtau G(tau) by enumerating all 2^Lambda
  HS fields (small Lambda).
* ``reduce_chains`` -- mean over chains and error bar (sample standard error
  over chains; 32 consecutive bins for a single chain).

Each chain's work is one C call, which releases the GIL, so ``run_chains``
spreads chains over host threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_BINS = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64, u32, u64, f64 = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_double)
            lib.orc_philox4x32_10.argtypes = [P, u64, P]
            lib.orc_philox_many.argtypes = [i64, P, u64, P]
            lib.orc_uniform.argtypes = [u32, u32, u32, u32, u64]
            lib.orc_uniform.restype = f64
            lib.orc_init_field.argtypes = [i32, u64, u32, u32, P]
            lib.orc_lambda.argtypes = [f64, f64]
            lib.orc_lambda.restype = f64
            lib.orc_bath_matrix.argtypes = [i32, P, P]
            lib.orc_build_A.argtypes = [i32, P, P, f64, i32, P]
            lib.orc_green.argtypes = [i32, P, P, f64, i32, P, P]
            lib.orc_green.restype = i32
            lib.orc_measure_g.argtypes = [i32, P, P]
            lib.orc_measure_D.argtypes = [i32, P, P]
            lib.orc_measure_D.restype = f64
            lib.orc_run_chain.argtypes = [i32, f64, P, u64, u32, u32, i64, i64, i64, i32, i32,
                                          P, P, P, P, P, P, P, P, P]
            lib.orc_run_chain.restype = i32
            lib.orc_brute_force.argtypes = [i32, f64, P, P, P, P, P]
            lib.orc_brute_force.restype = i64
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Small wrappers
# --------------------------------------------------------------------------
def philox(ctrs: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 of each row of ``ctrs`` (n x 4 uint32) under key ``seed``."""
    c = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    _load().orc_philox_many(c.shape[0], _p(c), ctypes.c_uint64(seed), _p(out))
    return out


def uniform(l: int, sweep: int, chain: int, grid: int, seed: int) -> float:
    return _load().orc_uniform(l, sweep, chain, grid, ctypes.c_uint64(seed))


def init_field(L: int, seed: int, chain: int, grid: int) -> np.ndarray:
    s = np.empty(L, dtype=np.int8)
    _load().orc_init_field(L, ctypes.c_uint64(seed), chain, grid, _p(s))
    return s


def lam(dtau: float, U: float) -> float:
    """lambda with cosh(lambda) = exp(dtau U / 2)."""
    return _load().orc_lambda(dtau, U)


def bath_matrix(G0_tau: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(G0_tau, dtype=np.float64)
    L = g.shape[0]
    M = np.empty((L, L))
    _load().orc_bath_matrix(L, _p(g), _p(M))
    return M


def build_A(M: np.ndarray, s: np.ndarray, lmbda: float, sigma: int) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    A = np.empty_like(M)
    _load().orc_build_A(M.shape[0], _p(M), _p(s), lmbda, sigma, _p(A))
    return A


def green(M: np.ndarray, s: np.ndarray, lmbda: float, sigma: int):
    """(G^sigma(s), det A^sigma(s)) by LU."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    G = np.empty_like(M)
    det = ctypes.c_double(0.0)
    rc = _load().orc_green(M.shape[0], _p(M), _p(s), lmbda, sigma, _p(G), ctypes.byref(det))
    if rc != 0:
        raise ArithmeticError("singular A in oracle green()")
    return G, det.value


def measure_g(G: np.ndarray) -> np.ndarray:
    G = np.ascontiguousarray(G, dtype=np.float64)
    g = np.empty(G.shape[0])
    _load().orc_measure_g(G.shape[0], _p(G), _p(g))
    return g


def measure_D(Gup: np.ndarray, Gdn: np.ndarray) -> float:
    Gup = np.ascontiguousarray(Gup, dtype=np.float64)
    Gdn = np.ascontiguousarray(Gdn, dtype=np.float64)
    return _load().orc_measure_D(Gup.shape[0], _p(Gup), _p(Gdn))


FNV_OFFSET = 0xcbf29ce484222325


# --------------------------------------------------------------------------
# Chains
# --------------------------------------------------------------------------
@dataclass
class Chain:
    """Full state of one Markov chain (field, both Green matrices, counters)."""
    L: int
    lmbda: float
    M: np.ndarray
    seed: int
    chain: int
    grid: int
    s: np.ndarray
    Gup: np.ndarray
    Gdn: np.ndarray
    t: int = 0                              # global sweep index of the next sweep
    stats: np.ndarray = field(default=None)  # proposals, accepted, recomputes, hash, bad R
    acc: np.ndarray = field(default=None)    # 2L sums of g^sigma(tau_k)
    accD: np.ndarray = field(default=None)   # 1 sum of D
    bins: np.ndarray = field(default=None)   # 32 x L sums of (g^up+g^dn)/2
    bin_counts: np.ndarray = field(default=None)
    n_meas: int = 0
    drift: float = 0.0

    @classmethod
    def new(cls, M, lmbda, seed, chain, grid):
        L = M.shape[0]
        s = init_field(L, seed, chain, grid)
        Gup, _ = green(M, s, lmbda, 1)
        Gdn, _ = green(M, s, lmbda, -1)
        st = np.zeros(5, dtype=np.int64)
        st[3] = np.array(FNV_OFFSET, dtype=np.uint64).view(np.int64)
        return cls(L=L, lmbda=lmbda, M=np.ascontiguousarray(M), seed=seed, chain=chain, grid=grid,
                   s=s, Gup=Gup, Gdn=Gdn, stats=st, acc=np.zeros(2 * L), accD=np.zeros(1),
                   bins=np.zeros((N_BINS, L)), bin_counts=np.zeros(N_BINS, dtype=np.int64))

    @property
    def decision_hash(self) -> int:
        return int(np.array(self.stats[3]).view(np.uint64))


def run_chain(ch: Chain, n_warm: int, n_meas: int, n_wrap: int = 64, accept_rule: int = 0,
              hist: np.ndarray | None = None) -> Chain:
    """Advance one chain by n_warm + n_meas sweeps (in place)."""
    drift = ctypes.c_double(ch.drift)
    h = _p(hist) if hist is not None else None
    rc = _load().orc_run_chain(ch.L, ch.lmbda, _p(ch.M), ctypes.c_uint64(ch.seed), ch.chain,
                               ch.grid, ch.t, n_warm, n_meas, n_wrap, accept_rule, _p(ch.s),
                               _p(ch.Gup), _p(ch.Gdn), _p(ch.stats), _p(ch.acc), _p(ch.accD),
                               _p(ch.bins) if n_meas > 0 else None, h, ctypes.byref(drift))
    if rc != 0:
        raise ArithmeticError("singular A during an oracle recompute")
    ch.drift = drift.value
    ch.t += n_warm + n_meas
    if n_meas > 0:
        m = np.arange(n_meas)
        ch.bin_counts += np.bincount((N_BINS * m) // n_meas, minlength=N_BINS)
    ch.n_meas += n_meas
    return ch


def run_chains(chains, n_warm, n_meas, n_wrap=64, accept_rule=0, threads=None):
    threads = threads or os.cpu_count() or 1
    if threads <= 1 or len(chains) <= 1:
        for ch in chains:
            run_chain(ch, n_warm, n_meas, n_wrap, accept_rule)
        return chains
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda c: run_chain(c, n_warm, n_meas, n_wrap, accept_rule), chains))
    return chains


def reduce_chains(chains):
    """Physical G(tau_k), k = 0..L-1, plus G(beta-) = -1 - G(0+), and error bars.

    Each chain gives its mean over measured sweeps of -(g^up + g^dn)/2.  With
    two or more chains the error is the sample standard deviation (n-1) of the
    chain means over sqrt(n); with one chain the measured sweeps are cut into
    32 consecutive bins and the same estimator is applied to the bin means.
    Also returns D and its error the same way."""
    L = chains[0].L
    means = np.array([-(c.acc[:L] + c.acc[L:]) / (2.0 * c.n_meas) for c in chains])
    Dm = np.array([c.accD[0] / c.n_meas for c in chains])
    if len(chains) >= 2:
        n = len(chains)
        G = means.mean(axis=0)
        err = means.std(axis=0, ddof=1) / np.sqrt(n)
        D = Dm.mean()
        Derr = Dm.std(ddof=1) / np.sqrt(n)
    else:
        c = chains[0]
        ok = c.bin_counts > 0
        bm = -c.bins[ok] / c.bin_counts[ok, None]
        G = means[0]
        nb = bm.shape[0]
        err = bm.std(axis=0, ddof=1) / np.sqrt(nb) if nb >= 2 else np.full(L, np.nan)
        D = Dm[0]
        Derr = float("nan")
    G_out = np.concatenate([G, [-1.0 - G[0]]])
    err_out = np.concatenate([err, [err[0]]])
    return G_out, err_out, D, Derr


def brute_force(M: np.ndarray, lmbda: float, return_weights: bool = False):
    """Exact discrete-dtau g(tau_k) (positive convention, spin-averaged), D, Z.

    Enumerates all 2^L fields with weight det A^up det A^dn.  Raises if any
    weight is not positive."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    L = M.shape[0]
    if L > 20:
        raise ValueError("brute force limited to L <= 20")
    g = np.empty(L)
    D = ctypes.c_double(0.0)
    Z = ctypes.c_double(0.0)
    w = np.empty(1 << L) if return_weights else None
    n_bad = _load().orc_brute_force(L, lmbda, _p(M), _p(g), ctypes.byref(D), ctypes.byref(Z),
                                    _p(w) if w is not None else None)
    if n_bad != 0:
        raise ArithmeticError(f"brute force: {n_bad} non-positive weights or singular A")
    if return_weights:
        return g, D.value, Z.value, w
    return g, D.value, Z.value


# --------------------------------------------------------------------------
# The C-ABI call sequence, on the oracle
# --------------------------------------------------------------------------
class OracleHFQMC:
    """Oracle with the same call sequence as the CUDA library's C ABI.

    grids are (U, dtau) pairs; beta/dtau must be an integer Lambda.  Chain c of
    grid i uses Philox counters (l, sweep, c, i) under key ``seed``."""

    def __init__(self, beta, grids, chains_per_grid, seed=1, n_wrap=64, accept_rule=0, threads=None):
        self.beta = float(beta)
        self.grids = []
        for (U, dtau) in grids:
            L = int(round(self.beta / dtau))
            if abs(self.beta / dtau - L) > 1e-9 or L < 1:
                raise ValueError("beta/dtau must be an integer")
            d = self.beta / L
            self.grids.append(dict(U=float(U), L=L, dtau=d, lmbda=lam(d, float(U))))
        self.chains_per_grid = list(chains_per_grid)
        self.seed = int(seed)
        self.n_wrap = int(n_wrap)
        self.accept_rule = int(accept_rule)
        self.threads = threads
        self.chains = [None] * len(self.grids)

    def set_G0(self, grid, G0_tau):
        """First call: fresh chains (field from Philox).  Later calls keep each
        chain's field, sweep index and flip counters, rebuild G from the new
        bath and zero the measurement sums (the library's semantics)."""
        g = self.grids[grid]
        G0_tau = np.asarray(G0_tau, dtype=np.float64)
        assert G0_tau.shape == (g["L"],)
        M = bath_matrix(G0_tau)
        if self.chains[grid] is None:
            self.chains[grid] = [Chain.new(M, g["lmbda"], self.seed, c, grid)
                                 for c in range(self.chains_per_grid[grid])]
            return
        for ch in self.chains[grid]:
            ch.M = np.ascontiguousarray(M)
            ch.Gup, _ = green(M, ch.s, ch.lmbda, 1)
            ch.Gdn, _ = green(M, ch.s, ch.lmbda, -1)
            ch.acc[:] = 0.0
            ch.accD[:] = 0.0
            ch.bins[:] = 0.0
            ch.bin_counts[:] = 0
            ch.n_meas = 0
            ch.drift = 0.0

    def sweep(self, n_warm, n_meas):
        allc = [c for cs in self.chains for c in cs]
        run_chains(allc, n_warm, n_meas, self.n_wrap, self.accept_rule, self.threads)

    def get_G(self, grid):
        G, err, _, _ = reduce_chains(self.chains[grid])
        return G, err

    def get_D(self, grid):
        _, _, D, Derr = reduce_chains(self.chains[grid])
        return D, Derr
