"""Python binding of libhfqmc.so (include/hfqmc.h): argument marshalling only.

Every step of the sweep runs in the library's CUDA kernels; this module
converts numpy arrays to pointers, passes PyTorch's current CUDA stream and
(optionally) PyTorch's caching allocator to the library, and raises on any
non-zero status.  If the library has not been built the import of the
binding still works, but the first call raises -- there is no CPU fallback.

Function names follow the C ABI (hfqmc_create, hfqmc_set_G0, hfqmc_sweep,
hfqmc_get_G, ...); ``HFQMC`` wraps them as methods of one context.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhfqmc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hfqmc.h")

HFQMC_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "EDRIFT", -6: "ENUMERIC",
          -7: "ETIMEOUT"}
PRECISION = {"f64_rank1": 0, "f32_rank1": 1, "f32_delayed": 2}
TRACE = {"off": 0, "record": 1, "replay": 2}
N_BINS = 32
ACCEPT = {"metropolis": 0, "heat_bath": 1}
FLUSH = {"auto": 0, "tcgen05": 1, "ffma": 2}
RECOMPUTE = {"auto": 0, "gj": 1, "refine": 2}

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class HFQMCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hfqmc {ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class hfqmc_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("k", ctypes.c_int), ("n_wrap", ctypes.c_int),
                ("accept_rule", ctypes.c_int), ("drift_warn", ctypes.c_double),
                ("drift_fail", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("autotune", ctypes.c_int), ("flush", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("alloc", _ALLOC_FN), ("free", _FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("resident_kb", ctypes.c_int), ("gj_smem", ctypes.c_int), ("gtile", ctypes.c_int),
                ("tune_table", ctypes.POINTER(ctypes.c_int)), ("tune_entries", ctypes.c_int),
                ("recompute", ctypes.c_int), ("refine_max", ctypes.c_double), ("ph_symmetry", ctypes.c_int)]


class hfqmc_stats(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("chains", ctypes.c_int), ("k", ctypes.c_int),
                ("n_wrap", ctypes.c_int), ("sweeps", ctypes.c_int64),
                ("proposals", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("recomputes", ctypes.c_int64), ("numeric_errors", ctypes.c_int64),
                ("accept_rate", ctypes.c_double), ("drift_max", ctypes.c_double),
                ("last_sweep_ms", ctypes.c_double), ("recompute_fallbacks", ctypes.c_int64),
                ("ph_symmetric", ctypes.c_int)]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/hfqmc.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(hfqmc_\w+)\s*\(", txt, flags=re.M)))


def load():
    """Loads libhfqmc.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the sweep has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.hfqmc_default_opts.argtypes = [ctypes.POINTER(hfqmc_opts)]
    lib.hfqmc_default_opts.restype = None
    lib.hfqmc_create.argtypes = [ctypes.POINTER(P), D, D, P, I, P, ctypes.c_uint64,
                                 ctypes.POINTER(hfqmc_opts)]
    lib.hfqmc_create_ex.argtypes = [ctypes.POINTER(P), D, P, P, I, P, ctypes.c_uint64,
                                    ctypes.POINTER(hfqmc_opts)]
    lib.hfqmc_set_G0.argtypes = [P, I, P]
    lib.hfqmc_sweep.argtypes = [P, I64, I64]
    lib.hfqmc_get_G.argtypes = [P, I, P, P]
    lib.hfqmc_get_D.argtypes = [P, I, P, P]
    lib.hfqmc_get_stats.argtypes = [P, I, ctypes.POINTER(hfqmc_stats)]
    lib.hfqmc_grid_size.argtypes = [P, I, ctypes.POINTER(I)]
    lib.hfqmc_get_chain.argtypes = [P, I, I, P, P, P, P, P]
    lib.hfqmc_last_error.argtypes = [P]
    lib.hfqmc_last_error.restype = ctypes.c_char_p
    lib.hfqmc_destroy.argtypes = [P]
    lib.hfqmc_destroy.restype = None
    lib.hfqmc_green_noalloc.argtypes = [P, P, I, D, D, P, P, P, ctypes.POINTER(I)]
    lib.hfqmc_get_chain_D.argtypes = [P, I, I, P, P]
    lib.hfqmc_set_trace.argtypes = [P, I, I64]
    lib.hfqmc_get_trace.argtypes = [P, I, P, I64]
    lib.hfqmc_put_trace.argtypes = [P, I, P, I64]
    for name in ("hfqmc_create", "hfqmc_create_ex", "hfqmc_set_G0", "hfqmc_sweep", "hfqmc_get_G",
                 "hfqmc_get_D", "hfqmc_get_stats", "hfqmc_grid_size", "hfqmc_get_chain",
                 "hfqmc_green_noalloc", "hfqmc_get_chain_D", "hfqmc_set_trace", "hfqmc_get_trace",
                 "hfqmc_put_trace"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, ctx):
    if rc != HFQMC_OK:
        msg = load().hfqmc_last_error(ctx)
        raise HFQMCError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C-ABI-named functions
# ---------------------------------------------------------------------------
def hfqmc_default_opts() -> hfqmc_opts:
    o = hfqmc_opts()
    load().hfqmc_default_opts(ctypes.byref(o))
    return o


def hfqmc_create(beta, U, dtau, chains_per_grid, seed=1, opts: hfqmc_opts | None = None):
    """U: a scalar (one U for all grids) or one value per grid (hfqmc_create_ex)."""
    lib = load()
    dt = np.ascontiguousarray(dtau, dtype=np.float64)
    ch = np.ascontiguousarray(chains_per_grid, dtype=np.int32)
    out = ctypes.c_void_p()
    o = opts if opts is not None else hfqmc_default_opts()
    if np.ndim(U) == 0:
        rc = lib.hfqmc_create(ctypes.byref(out), float(beta), float(U), _p(dt), len(dt), _p(ch),
                              ctypes.c_uint64(seed), ctypes.byref(o))
    else:
        Ua = np.ascontiguousarray(U, dtype=np.float64)
        rc = lib.hfqmc_create_ex(ctypes.byref(out), float(beta), _p(Ua), _p(dt), len(dt), _p(ch),
                                 ctypes.c_uint64(seed), ctypes.byref(o))
    _check(rc, None)
    return out


def hfqmc_set_G0(ctx, grid, G0_tau):
    g = np.ascontiguousarray(G0_tau, dtype=np.float64)
    _check(load().hfqmc_set_G0(ctx, grid, _p(g)), ctx)


def hfqmc_sweep(ctx, n_warm, n_meas):
    _check(load().hfqmc_sweep(ctx, int(n_warm), int(n_meas)), ctx)


def hfqmc_grid_size(ctx, grid) -> int:
    L = ctypes.c_int(0)
    _check(load().hfqmc_grid_size(ctx, grid, ctypes.byref(L)), ctx)
    return L.value


def hfqmc_get_G(ctx, grid, G_tau: np.ndarray | None = None, G_err: np.ndarray | None = None):
    L = hfqmc_grid_size(ctx, grid)
    G = G_tau if G_tau is not None else np.empty(L + 1)
    E = G_err if G_err is not None else np.empty(L + 1)
    _check(load().hfqmc_get_G(ctx, grid, _p(G), _p(E)), ctx)
    return G, E


def hfqmc_get_D(ctx, grid):
    D = ctypes.c_double()
    E = ctypes.c_double()
    _check(load().hfqmc_get_D(ctx, grid, ctypes.byref(D), ctypes.byref(E)), ctx)
    return D.value, E.value


def hfqmc_get_stats(ctx, grid) -> dict:
    s = hfqmc_stats()
    _check(load().hfqmc_get_stats(ctx, grid, ctypes.byref(s)), ctx)
    return {f: getattr(s, f) for f, _ in hfqmc_stats._fields_}


def hfqmc_get_chain(ctx, grid, chain) -> dict:
    L = hfqmc_grid_size(ctx, grid)
    s = np.empty(L, dtype=np.int8)
    Gu = np.empty((L, L))
    Gd = np.empty((L, L))
    cnt = np.empty(6, dtype=np.int64)
    acc = np.empty(2 * L)
    _check(load().hfqmc_get_chain(ctx, grid, chain, _p(s), _p(Gu), _p(Gd), _p(cnt), _p(acc)), ctx)
    return dict(s=s, Gup=Gu, Gdn=Gd, proposals=int(cnt[0]), accepted=int(cnt[1]),
                recomputes=int(cnt[2]), hash=int(np.array(cnt[3]).view(np.uint64)),
                bad=int(cnt[4]), t=int(cnt[5]), acc=acc)


def hfqmc_get_chain_D(ctx, grid, chain):
    """(sum of D over the measured sweeps since set_G0, its 32 bin sums)."""
    D = ctypes.c_double(0.0)
    bins = np.empty(N_BINS)
    _check(load().hfqmc_get_chain_D(ctx, grid, chain, ctypes.byref(D), _p(bins)), ctx)
    return D.value, bins


def hfqmc_set_trace(ctx, mode, max_sweeps):
    """mode: "off", "record" or "replay" (see include/hfqmc.h)."""
    _check(load().hfqmc_set_trace(ctx, TRACE[mode], int(max_sweeps)), ctx)


def hfqmc_get_trace(ctx, grid, n_words):
    bits = np.empty(int(n_words), dtype=np.uint32)
    _check(load().hfqmc_get_trace(ctx, grid, _p(bits), int(n_words)), ctx)
    return bits


def hfqmc_put_trace(ctx, grid, bits):
    b = np.ascontiguousarray(bits, dtype=np.uint32)
    _check(load().hfqmc_put_trace(ctx, grid, _p(b), b.size), ctx)


NOALLOC_MAX_L = 256


def hfqmc_green_noalloc(G0_tau_dev: int, s_dev: int, L: int, dtau: float, U: float, G_up_dev: int,
                        G_dn_dev: int, stream: int = 0) -> int:
    """FP64 G^up, G^dn of one field from caller-owned device buffers (integer
    device addresses), without any device allocation; returns the status bits."""
    st = ctypes.c_int(0)
    rc = load().hfqmc_green_noalloc(ctypes.c_void_p(G0_tau_dev), ctypes.c_void_p(s_dev), int(L),
                                    float(dtau), float(U), ctypes.c_void_p(G_up_dev),
                                    ctypes.c_void_p(G_dn_dev), ctypes.c_void_p(stream),
                                    ctypes.byref(st))
    if rc != HFQMC_OK:
        raise HFQMCError(rc, f"hfqmc_green_noalloc (L={L}, status bits {st.value})")
    return st.value


def hfqmc_last_error(ctx) -> str:
    m = load().hfqmc_last_error(ctx)
    return m.decode() if m else ""


def hfqmc_destroy(ctx):
    if ctx:
        load().hfqmc_destroy(ctx)


# ---------------------------------------------------------------------------
# PyTorch plumbing: device memory through the caching allocator, current stream
# ---------------------------------------------------------------------------
class _TorchAllocator:
    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.stream = torch.cuda.current_stream(device)
        self._a = _ALLOC_FN(self._alloc)
        self._f = _FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:  # reported by the library as HFQMC_ENOMEM
            return None

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


class HFQMC:
    """One context: several (U, dtau) grids x chains, fixed beta.  The
    keyword options map one to one onto hfqmc_opts (include/hfqmc.h); among
    them recompute ("auto" = "refine" on the FP32 delayed path, "gj"),
    refine_max (the Newton step's largest residual, 0 = 2^-8) and
    ph_symmetry (0: with every grid's bath particle-hole symmetric the sweep
    keeps G_up only; 1: only the recompute uses the symmetry; -1: never)."""

    def __init__(self, beta, U, dtau, chains_per_grid, seed=1, precision="f32_delayed", k=0,
                 n_wrap=0, accept_rule="metropolis", drift_fail=1e-1, flush="auto",
                 use_graph=True, stream=None, torch_alloc=True, resident_kb=0, gj_smem=0,
                 gtile=0, tune=None, autotune=True, recompute="auto", refine_max=0.0, ph_symmetry=0):
        o = hfqmc_default_opts()
        o.precision = PRECISION[precision]
        o.k = int(k)
        o.n_wrap = int(n_wrap)
        o.accept_rule = ACCEPT[accept_rule]
        o.drift_fail = float(drift_fail)
        o.flush = FLUSH[flush]
        o.use_graph = 1 if use_graph else 0
        o.resident_kb = int(resident_kb)
        o.gj_smem = int(gj_smem)
        o.gtile = int(gtile)
        o.autotune = 1 if autotune else 0
        o.recompute = RECOMPUTE[recompute]
        o.refine_max = float(refine_max)
        o.ph_symmetry = int(ph_symmetry)
        if tune is not None:  # [(Lambda_max, k, n_wrap), ...] (see autotune.py)
            flat = [int(v) for e in tune for v in e]
            self._tune = (ctypes.c_int * len(flat))(*flat)
            o.tune_table = ctypes.cast(self._tune, ctypes.POINTER(ctypes.c_int))
            o.tune_entries = len(flat) // 3
        self._allocator = None
        try:
            import torch
            if torch.cuda.is_available():
                dev = torch.cuda.current_device()
                st = stream if stream is not None else torch.cuda.current_stream(dev)
                o.cuda_stream = ctypes.c_void_p(st.cuda_stream)
                self.torch_stream = st
                if torch_alloc:
                    self._allocator = _TorchAllocator(dev)
                    o.alloc = self._allocator._a
                    o.free = self._allocator._f
        except ImportError:
            pass
        self._opts = o
        self.ctx = hfqmc_create(beta, U, dtau, chains_per_grid, seed, o)
        self.n_grids = len(np.atleast_1d(dtau))

    def set_G0(self, grid, G0_tau):
        hfqmc_set_G0(self.ctx, grid, G0_tau)

    def sweep(self, n_warm, n_meas):
        hfqmc_sweep(self.ctx, n_warm, n_meas)

    def get_G(self, grid):
        return hfqmc_get_G(self.ctx, grid)

    def get_D(self, grid):
        return hfqmc_get_D(self.ctx, grid)

    def get_stats(self, grid):
        return hfqmc_get_stats(self.ctx, grid)

    def get_chain(self, grid, chain):
        return hfqmc_get_chain(self.ctx, grid, chain)

    def grid_size(self, grid):
        return hfqmc_grid_size(self.ctx, grid)

    def get_chain_D(self, grid, chain):
        return hfqmc_get_chain_D(self.ctx, grid, chain)

    def set_trace(self, mode, max_sweeps=1):
        hfqmc_set_trace(self.ctx, mode, max_sweeps)
        self._trace_sweeps = int(max_sweeps)

    def trace_words(self, grid, chains):
        return chains * self._trace_sweeps * ((self.grid_size(grid) + 31) // 32)

    def get_trace(self, grid, chains):
        """One grid's trace as [chain][sweep][word] uint32."""
        w = (self.grid_size(grid) + 31) // 32
        return hfqmc_get_trace(self.ctx, grid, self.trace_words(grid, chains)).reshape(
            chains, self._trace_sweeps, w)

    def put_trace(self, grid, bits):
        hfqmc_put_trace(self.ctx, grid, bits)

    def close(self):
        if getattr(self, "ctx", None):
            hfqmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
