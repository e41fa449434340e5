"""Thin ctypes binding of libsrmra.so (C ABI in include/srmra.h).

The functions ``srmra_create``, ``srmra_em_iter``, ... carry the C names and only
marshal arguments; every step of the computation runs in the CUDA library.  The
:class:`Solver` class is a small convenience wrapper over the same calls.

The library is loaded on first use.  If it has not been built (``python -m
paper_2204_04754_gb300.build``) a RuntimeError is raised; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, byref, c_char_p, c_double, c_float,
                    c_int32, c_int64, c_uint32, c_void_p)

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsrmra.so")

SRMRA_OK, SRMRA_EINVAL, SRMRA_ENOMEM, SRMRA_ECUDA, SRMRA_ETIMEOUT, SRMRA_ENUMERIC, \
    SRMRA_EBUSY = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT",
                5: "ENUMERIC", 6: "EBUSY"}
SRMRA_FP32, SRMRA_BF16, SRMRA_BF16X3, SRMRA_FFT32 = 0, 1, 2, 3
PRECISIONS = {"fp32": SRMRA_FP32, "bf16": SRMRA_BF16, "bf16x3": SRMRA_BF16X3,
              "fft32": SRMRA_FFT32}
SRMRA_FLAG_CHECK_NUMERIC = 1
SRMRA_FLAG_NO_CLUSTER = 2
SRMRA_FLAG_MSTEP_COMP = 4
SRMRA_FLAG_MSTEP_FP16 = 8
SRMRA_FLAG_P1_TILE128 = 16
SRMRA_FLAG_P2_PAIR = 32
SRMRA_SERVER_AUTO = 4  # srmra_server_create: the form picked per request


class srmra_params(Structure):
    _fields_ = [("L_high", c_int32), ("K", c_int32), ("N", c_int64), ("sigma", c_double),
                ("prec", c_int32), ("flags", c_uint32)]


DENOISER_FN = CFUNCTYPE(c_int32, POINTER(c_float), c_int32, c_double, c_void_p, c_void_p)


class SrmraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsrmra.so (once) and declare the C prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                           "`python -m paper_2204_04754_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = POINTER
    sig = {
        "srmra_create": (c_int32, [P(srmra_params), c_void_p, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_void_p, P(c_void_p)]),
        "srmra_em_iter": (c_int32, [c_void_p, c_int32, c_void_p]),
        "srmra_project": (c_int32, [c_void_p, c_double, c_void_p, c_void_p]),
        "srmra_solve": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_double, c_void_p,
                                  c_void_p, c_void_p]),
        "srmra_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
        "srmra_set_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_double,
                                      c_int32]),
        "srmra_get_estep": (c_int32, [c_void_p, c_void_p, c_void_p]),
        "srmra_launch_count": (c_int32, [c_void_p, P(c_int64)]),
        "srmra_get_plan": (c_int32, [c_void_p, c_void_p, c_int32]),
        "srmra_set_wait_limit": (c_int32, [c_void_p, c_int64, c_int32]),
        "srmra_sync": (c_int32, [c_void_p]),
        "srmra_profile": (c_int32, [c_void_p, c_int32]),
        "srmra_profile_read": (c_int32, [c_void_p, c_void_p, c_void_p]),
        "srmra_destroy": (None, [c_void_p]),
        "srmra_batch_create": (c_int32, [c_void_p, c_int32, c_uint32, P(c_void_p)]),
        "srmra_batch_solve": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_double,
                                        c_void_p]),
        "srmra_batch_tuning": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "srmra_batch_tiles": (c_int32, [c_void_p, c_void_p]),
        "srmra_batch_destroy": (None, [c_void_p]),
        "srmra_batch_pass_ms": (c_int32, [c_void_p, c_void_p, c_void_p]),
        "srmra_batch_last_error": (c_char_p, [c_void_p]),
        "srmra_em_iter_batch": (c_int32, [c_void_p, c_int32, c_int32]),
        "srmra_set_schedule": (c_int32, [c_void_p, c_int32, c_double, c_double]),
        "srmra_set_denoiser": (c_int32, [c_void_p, c_int32, c_double, c_int32]),
        "srmra_estimate_device_bytes": (c_int32, [P(srmra_params), P(c_int64)]),
        "srmra_device_bytes": (c_int32, [c_void_p, P(c_int64)]),
        "srmra_server_create": (c_int32, [c_int64, c_int32, c_int32, c_void_p, P(c_void_p)]),
        "srmra_server_submit": (c_int32, [c_void_p, P(srmra_params), c_void_p, c_void_p,
                                          c_int32, c_int32, c_double, c_double, P(c_int64)]),
        "srmra_server_step": (c_int32, [c_void_p, P(c_int32), P(c_int32), P(c_int32)]),
        "srmra_server_result": (c_int32, [c_void_p, c_int64, P(c_int32), c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p]),
        "srmra_server_memory": (c_int32, [c_void_p, P(c_int64), P(c_int64)]),
        "srmra_server_destroy": (None, [c_void_p]),
        "srmra_server_last_error": (c_char_p, [c_void_p]),
        "srmra_online_create": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                          P(c_void_p)]),
        "srmra_online_step": (c_int32, [c_void_p, c_int32, c_double, c_void_p]),
        "srmra_online_project": (c_int32, [c_void_p, c_double]),
        "srmra_online_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p,
                                             P(c_int64)]),
        "srmra_online_destroy": (None, [c_void_p]),
        "srmra_online_last_error": (c_char_p, [c_void_p]),
        "srmra_stats_length": (c_int32, [c_void_p, P(c_int64)]),
        "srmra_estep_stats": (c_int32, [c_void_p, c_void_p, c_int32]),
        "srmra_mstep_stats": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
        "srmra_mom_create": (c_int32, [c_void_p, P(c_void_p)]),
        "srmra_mom_moments": (c_int32, [c_void_p, c_void_p, c_void_p]),
        "srmra_mom_eval": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "srmra_mom_run": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_double, c_double,
                                    c_double, c_void_p, c_void_p, c_void_p]),
        "srmra_mom_recompute_moments": (c_int32, [c_void_p]),
        "srmra_mom_destroy": (None, [c_void_p]),
        "srmra_mom_last_error": (c_char_p, [c_void_p]),
        "srmra_last_error": (c_char_p, [c_void_p]),
        "srmra_version": (c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a) -> int | None:
    """Address of a numpy array / torch tensor / None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


def _check(st: int, ctx=None):
    if st != SRMRA_OK:
        msg = lib().srmra_last_error(ctx)
        raise SrmraError(st, msg.decode() if msg else "")


# ----------------------------------------------------------------------------- C names

def srmra_create(params: srmra_params, y, y_is_device: bool, x0=None, rho1_0=None,
                 rho2_0=None, stream: int = 0) -> int:
    ctx = c_void_p()
    st = lib().srmra_create(byref(params), _ptr(y), int(bool(y_is_device)), _ptr(x0),
                            _ptr(rho1_0), _ptr(rho2_0), c_void_p(stream or None), byref(ctx))
    _check(st, None)
    return ctx.value


def srmra_em_iter(ctx: int, n_iters: int, loglik_out=None) -> None:
    _check(lib().srmra_em_iter(ctx, n_iters, _ptr(loglik_out)), ctx)


def srmra_project(ctx: int, sigma_bm: float, fn=None, user=None) -> None:
    _check(lib().srmra_project(ctx, sigma_bm, fn, user), ctx)


def srmra_solve(ctx: int, iters: int, F: int, sigma_bm1: float, decay: float,
                fn=None, user=None, loglik_out=None) -> None:
    _check(lib().srmra_solve(ctx, iters, F, sigma_bm1, decay, fn, user, _ptr(loglik_out)), ctx)


def srmra_get_state(ctx: int, x=None, rho1=None, rho2=None):
    sbm = c_double()
    t = c_int32()
    _check(lib().srmra_get_state(ctx, _ptr(x), _ptr(rho1), _ptr(rho2), byref(sbm), byref(t)),
           ctx)
    return sbm.value, t.value


def srmra_set_state(ctx: int, x, rho1, rho2, sigma_bm: float, t: int) -> None:
    _check(lib().srmra_set_state(ctx, _ptr(x), _ptr(rho1), _ptr(rho2), sigma_bm, t), ctx)


def srmra_get_estep(ctx: int, lse=None, c=None) -> None:
    _check(lib().srmra_get_estep(ctx, _ptr(lse), _ptr(c)), ctx)


def srmra_launch_count(ctx: int) -> int:
    n = c_int64()
    _check(lib().srmra_launch_count(ctx, byref(n)), ctx)
    return n.value


P2_FORMS = {0: "per_chunk", 1: "ring", 2: "interleaved", 3: "fp32", 4: "fft",
            5: "per_chunk_comp", 6: "pair"}


def srmra_set_wait_limit(ctx: int, limit_ns: int, test_hook: int = 0) -> None:
    _check(lib().srmra_set_wait_limit(ctx, int(limit_ns), int(test_hook)), ctx)


def srmra_get_plan(ctx: int) -> dict:
    v = np.zeros(7, np.int32)
    _check(lib().srmra_get_plan(ctx, v.ctypes.data, 7), ctx)
    return {"p1_groups": int(v[0]), "p1_tiles_per_group": int(v[1]), "p2_cluster": int(v[2]),
            "p2_chunk_groups": int(v[3]), "p2_form": P2_FORMS[int(v[4])],
            "p2_splits": int(v[5]), "p1_shift_tile": int(v[6])}


PHASES = ["prep", "pass1", "combine", "pass2", "final", "denoise"]


def srmra_profile(ctx: int, enable: bool) -> None:
    _check(lib().srmra_profile(ctx, int(bool(enable))), ctx)


def srmra_profile_read(ctx: int):
    ms = np.zeros(len(PHASES))
    n = np.zeros(len(PHASES), np.int64)
    _check(lib().srmra_profile_read(ctx, ms.ctypes.data, n.ctypes.data), ctx)
    return ms, n


def srmra_sync(ctx: int) -> None:
    _check(lib().srmra_sync(ctx), ctx)


def srmra_destroy(ctx: int) -> None:
    lib().srmra_destroy(ctx)


def srmra_version() -> str:
    return lib().srmra_version().decode()


SRMRA_BATCH_AUTOTUNE = 1
SRMRA_BATCH_NO_GRAPH = 2


def _bcheck(st: int, batch=None):
    if st != SRMRA_OK:
        msg = lib().srmra_batch_last_error(batch)
        raise SrmraError(st, msg.decode() if msg else "")


def _ctx_array(ctxs):
    arr = (c_void_p * len(ctxs))(*ctxs)
    return arr


def srmra_batch_create(ctxs, flags: int = 0) -> int:
    out = c_void_p()
    arr = _ctx_array(ctxs)
    _bcheck(lib().srmra_batch_create(arr, len(ctxs), flags, byref(out)), None)
    return out.value


def srmra_batch_solve(batch: int, iters: int, F: int, sigma_bm1: float, decay: float,
                      loglik_last=None) -> None:
    _bcheck(lib().srmra_batch_solve(batch, iters, F, sigma_bm1, decay, _ptr(loglik_last)),
            batch)


def srmra_batch_tuning(batch: int):
    a, b, c = c_int32(), c_int32(), c_int32()
    ms = c_double()
    _bcheck(lib().srmra_batch_tuning(batch, byref(a), byref(b), byref(c), byref(ms)), batch)
    bn = c_int32()
    _bcheck(lib().srmra_batch_tiles(batch, byref(bn)), batch)
    return dict(p1_scale=a.value, p2_scale=b.value, order=c.value, ms=ms.value,
                p1_shift_tile=bn.value)


def srmra_batch_destroy(batch: int) -> None:
    lib().srmra_batch_destroy(batch)


def srmra_em_iter_batch(ctxs, n_iters: int) -> None:
    arr = _ctx_array(ctxs)
    _bcheck(lib().srmra_em_iter_batch(arr, len(ctxs), n_iters), None)


# ----------------------------------------------------------------------------- wrapper

class Solver:
    """One SR-MRA problem held on the GPU.

    y: (N, l, l) float32 numpy array (host) or CUDA tensor (device, C-contiguous).
    prec: 'fp32' | 'bf16' | 'bf16x3'.  stream: cudaStream_t as an int (0 = default).
    """

    def __init__(self, L: int, K: int, sigma: float, y, prec: str = "fp32", x0=None,
                 rho1=None, rho2=None, stream: int = 0, flags: int = 0,
                 y_on_device: bool | None = None):
        if y_on_device is None:
            y_on_device = bool(getattr(y, "is_cuda", False))
        on_device = y_on_device
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=np.float32)
        self.L, self.K, self.N = int(L), int(K), int(y.shape[0])
        self.l = self.L // self.K
        p = srmra_params(self.L, self.K, self.N, float(sigma), PRECISIONS[prec], flags)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float32)
        r1 = None if rho1 is None else np.ascontiguousarray(rho1, dtype=np.float64)
        r2 = None if rho2 is None else np.ascontiguousarray(rho2, dtype=np.float64)
        self._keep = (y,)
        self.ctx = srmra_create(p, y, on_device, x0, r1, r2, stream)

    def em_iter(self, n: int = 1, loglik: bool = True):
        out = np.empty(max(n, 1)) if loglik else None
        srmra_em_iter(self.ctx, n, out)
        return None if out is None else out[:n]

    def solve(self, iters: int, F: int, sigma_bm1: float = 1.0, decay: float = 2.0 ** -0.1,
              denoiser=None, loglik: bool = True):
        out = np.empty(max(iters, 1)) if loglik else None
        fn = None
        if denoiser is not None:
            fn = DENOISER_FN(denoiser)
            self._fn = fn
        srmra_solve(self.ctx, iters, F, sigma_bm1, decay, fn, None, out)
        return None if out is None else out[:iters]

    def project(self, sigma_bm: float, denoiser=None):
        fn = None
        if denoiser is not None:
            fn = DENOISER_FN(denoiser)
            self._fn = fn
        srmra_project(self.ctx, sigma_bm, fn, None)

    def set_schedule(self, F: int, sigma_bm: float, decay: float = 2.0 ** -0.1):
        """Algorithm 2 schedule applied by mstep_stats (and by batches solved with F < 0)."""
        _check(lib().srmra_set_schedule(self.ctx, int(F), float(sigma_bm), float(decay)),
               self.ctx)

    def set_denoiser(self, mode: str = "hard", threshold: float = 2.7, spin: bool = False):
        """Built-in denoiser: 'hard' or 'soft' threshold, optional cycle spinning."""
        m = {"hard": 0, "soft": 1}[mode]
        _check(lib().srmra_set_denoiser(self.ctx, m, float(threshold), int(bool(spin))), self.ctx)

    def state(self):
        x = np.empty((self.L, self.L), np.float32)
        r1 = np.empty(self.L)
        r2 = np.empty(self.L)
        sbm, t = srmra_get_state(self.ctx, x, r1, r2)
        return x, r1, r2, sbm, t

    def set_state(self, x, rho1, rho2, sigma_bm: float, t: int):
        srmra_set_state(self.ctx, np.ascontiguousarray(x, np.float32),
                        np.ascontiguousarray(rho1, np.float64),
                        np.ascontiguousarray(rho2, np.float64), sigma_bm, t)

    def estep(self):
        lse = np.empty(self.N)
        c = np.empty(self.L * self.L)
        srmra_get_estep(self.ctx, lse, c)
        return lse, c

    def stats_length(self) -> int:
        n = c_int64()
        _check(lib().srmra_stats_length(self.ctx, byref(n)), self.ctx)
        return n.value

    def estep_stats(self, out=None):
        """E-step statistics at the current estimate (see include/srmra.h): a float64
        numpy vector (host), or written into `out`, a float64 CUDA tensor (device, in
        stream order)."""
        if out is not None and getattr(out, "is_cuda", False):
            _check(lib().srmra_estep_stats(self.ctx, c_void_p(out.data_ptr()), 1), self.ctx)
            return out
        v = np.empty(self.stats_length())
        _check(lib().srmra_estep_stats(self.ctx, _ptr(v), 0), self.ctx)
        return v

    def mstep_stats(self, stats, loglik: bool = True):
        """M-step from a statistics vector (numpy float64, or a float64 CUDA tensor)."""
        out = np.empty(1) if loglik else None
        if getattr(stats, "is_cuda", False):
            _check(lib().srmra_mstep_stats(self.ctx, c_void_p(stats.data_ptr()), 1, _ptr(out)),
                   self.ctx)
        else:
            v = np.ascontiguousarray(stats, dtype=np.float64)
            _check(lib().srmra_mstep_stats(self.ctx, _ptr(v), 0, _ptr(out)), self.ctx)
        return None if out is None else float(out[0])

    @property
    def launches(self) -> int:
        return srmra_launch_count(self.ctx)

    def plan(self) -> dict:
        """Work decomposition of the context's kernels (srmra_get_plan)."""
        return srmra_get_plan(self.ctx)

    def set_wait_limit(self, limit_ns: int, test_hook: int = 0):
        """Limit of the bounded device waits, and the failure-path test hook."""
        srmra_set_wait_limit(self.ctx, limit_ns, test_hook)

    def sync(self):
        srmra_sync(self.ctx)

    def profile(self, enable: bool = True):
        srmra_profile(self.ctx, enable)

    def profile_read(self):
        """-> ({phase: ms}, {phase: launches}) accumulated since the last read."""
        ms, n = srmra_profile_read(self.ctx)
        return dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, n.tolist()))

    def close(self):
        if getattr(self, "ctx", None):
            srmra_destroy(self.ctx)
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


class Batch:
    """Several :class:`Solver` problems advanced together (grouped launches, CUDA graph)."""

    def __init__(self, solvers, autotune: bool = False, graph: bool = True):
        self.solvers = list(solvers)
        flags = (SRMRA_BATCH_AUTOTUNE if autotune else 0) | (0 if graph else SRMRA_BATCH_NO_GRAPH)
        self.handle = srmra_batch_create([s.ctx for s in self.solvers], flags)

    def solve(self, iters: int, F: int, sigma_bm1: float = 1.0, decay: float = 2.0 ** -0.1):
        out = np.empty(len(self.solvers))
        srmra_batch_solve(self.handle, iters, F, sigma_bm1, decay, out)
        return out

    def tuning(self):
        return srmra_batch_tuning(self.handle)

    def pass_ms(self):
        """Device ms of the grouped pass 1 and pass 2 of the most recent iteration."""
        a, b = c_double(), c_double()
        _bcheck(lib().srmra_batch_pass_ms(self.handle, byref(a), byref(b)), self.handle)
        return a.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            srmra_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srmra_estimate_device_bytes(L: int, K: int, N: int, sigma: float, prec: str = "fp32") -> int:
    out = c_int64()
    p = srmra_params(L, K, N, sigma, PRECISIONS[prec], 0)
    _check(lib().srmra_estimate_device_bytes(byref(p), byref(out)), None)
    return out.value


class Online:
    """Online (mini-batch) EM over shard :class:`Solver` objects (same L, K, sigma,
    precision, stream): each step runs the E-step on one shard, folds its statistics
    into the running ones with step size gamma, and runs the M-step on them."""

    def __init__(self, shards, x0=None, rho1=None, rho2=None):
        self.shards = list(shards)
        arr = _ctx_array([s.ctx for s in self.shards])
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float32)
        r1 = None if rho1 is None else np.ascontiguousarray(rho1, dtype=np.float64)
        r2 = None if rho2 is None else np.ascontiguousarray(rho2, dtype=np.float64)
        out = c_void_p()
        self._check(lib().srmra_online_create(arr, len(self.shards), _ptr(x0), _ptr(r1),
                                              _ptr(r2), byref(out)), None)
        self.handle = out.value
        self.L = self.shards[0].L

    @staticmethod
    def _check(st, h):
        if st != SRMRA_OK:
            msg = lib().srmra_online_last_error(h)
            raise SrmraError(st, msg.decode() if msg else "")

    def step(self, shard: int, gamma: float, loglik: bool = True):
        out = np.empty(1) if loglik else None
        self._check(lib().srmra_online_step(self.handle, shard, gamma, _ptr(out)), self.handle)
        return None if out is None else float(out[0])

    def project(self, sigma_bm: float):
        self._check(lib().srmra_online_project(self.handle, sigma_bm), self.handle)

    def state(self):
        x = np.empty((self.L, self.L), np.float32)
        r1 = np.empty(self.L)
        r2 = np.empty(self.L)
        n = c_int64()
        self._check(lib().srmra_online_get_state(self.handle, _ptr(x), _ptr(r1), _ptr(r2),
                                                 byref(n)), self.handle)
        return x, r1, r2, n.value

    def close(self):
        if getattr(self, "handle", None):
            lib().srmra_online_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mom:
    """Projected method of moments (Algorithm 1) on a :class:`Solver`'s observations:
    the empirical moments are computed once at construction; :meth:`run` updates the
    solver's estimate in place (read it with ``solver.state()``)."""

    def __init__(self, solver):
        self.solver = solver
        out = c_void_p()
        self._check(lib().srmra_mom_create(solver.ctx, byref(out)), None)
        self.handle = out.value
        self.L, self.l = solver.L, solver.l

    @staticmethod
    def _check(st, h):
        if st != SRMRA_OK:
            msg = lib().srmra_mom_last_error(h)
            raise SrmraError(st, msg.decode() if msg else "")

    def moments(self):
        n = self.l * self.l
        m1 = np.empty(n)
        m2 = np.empty((n, n))
        self._check(lib().srmra_mom_moments(self.handle, _ptr(m1), _ptr(m2)), self.handle)
        return m1, m2

    def eval(self):
        """(f, df/dx (L x L), df/drho1, df/drho2) at the solver's current estimate."""
        f = np.empty(1)
        gx = np.empty((self.L, self.L))
        g1 = np.empty(self.L)
        g2 = np.empty(self.L)
        self._check(lib().srmra_mom_eval(self.handle, _ptr(f), _ptr(gx), _ptr(g1), _ptr(g2)),
                    self.handle)
        return float(f[0]), gx, g1, g2

    def run(self, iters: int, F: int, mu_x: float, mu_rho: float, sigma_bm1: float = 1.0,
            decay: float = 2.0 ** -0.1, denoiser=None, objective: bool = True):
        out = np.empty(max(iters, 1)) if objective else None
        fn = None
        if denoiser is not None:
            fn = DENOISER_FN(denoiser)
            self._fn = fn
        self._check(lib().srmra_mom_run(self.handle, int(iters), int(F), float(mu_x),
                                        float(mu_rho), float(sigma_bm1), float(decay), fn, None,
                                        _ptr(out)), self.handle)
        return None if out is None else out[:iters]

    def recompute_moments(self):
        self._check(lib().srmra_mom_recompute_moments(self.handle), self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().srmra_mom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (see include/srmra.h).  prec: a form for every
    request, or "auto" (the polyphase-FFT form where L/K is 8, 16 or 32, else bf16x3)."""

    def __init__(self, budget_bytes: int, max_active: int, prec: str = "bf16x3",
                 stream: int = 0):
        out = c_void_p()
        self.prec = prec
        code = SRMRA_SERVER_AUTO if prec == "auto" else PRECISIONS[prec]
        st = lib().srmra_server_create(int(budget_bytes), int(max_active), code,
                                       c_void_p(stream or None), byref(out))
        self._scheck(st, None)
        self.handle = out.value

    def _scheck(self, st, h):
        if st != SRMRA_OK:
            msg = lib().srmra_server_last_error(h)
            raise SrmraError(st, msg.decode() if msg else "")

    def submit(self, L, K, sigma, y, iters: int, F: int = 1, sigma_bm1: float = 1.0,
               decay: float = 2.0 ** -0.1, x0=None) -> int:
        y = np.ascontiguousarray(y, np.float32)
        x0 = None if x0 is None else np.ascontiguousarray(x0, np.float32)
        # (the server replaces the form with its own, or with the one it picks)
        p = srmra_params(int(L), int(K), int(y.shape[0]), float(sigma),
                         PRECISIONS.get(self.prec, SRMRA_BF16X3), 0)
        rid = c_int64()
        self._scheck(lib().srmra_server_submit(self.handle, byref(p), _ptr(y), _ptr(x0),
                                               int(iters), int(F), float(sigma_bm1),
                                               float(decay), byref(rid)), self.handle)
        return rid.value

    def step(self):
        a, b, c = c_int32(), c_int32(), c_int32()
        self._scheck(lib().srmra_server_step(self.handle, byref(a), byref(b), byref(c)),
                     self.handle)
        return a.value, b.value, c.value

    def result(self, rid: int, L: int):
        state = c_int32()
        x = np.empty((L, L), np.float32)
        r1 = np.empty(L)
        r2 = np.empty(L)
        ll = c_double()
        t = np.empty(3)
        st = lib().srmra_server_result(self.handle, rid, byref(state), _ptr(x), _ptr(r1),
                                       _ptr(r2), byref(ll), _ptr(t))
        self._scheck(st, self.handle)
        return dict(state=state.value, x=x, rho1=r1, rho2=r2, loglik=ll.value,
                    queue_ms=t[0], run_ms=t[1], latency_ms=t[2])

    def memory(self):
        u, b = c_int64(), c_int64()
        self._scheck(lib().srmra_server_memory(self.handle, byref(u), byref(b)), self.handle)
        return u.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            lib().srmra_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
