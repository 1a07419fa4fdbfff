"""Thin ctypes binding of libtrstmi.so (include/trstmi.h); marshalling only.

Every step of the search runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or no CUDA device is usable, the
calls raise.  Frames are numpy complex128 arrays of shape (d, N).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtrstmi.so")

TRSTMI_OK, TRSTMI_PENDING = 0, 1
TRSTMI_EINVAL, TRSTMI_ENOMEM, TRSTMI_ECUDA, TRSTMI_ETIMEOUT = -1, -2, -3, -4
TRSTMI_ECANCELLED, TRSTMI_EBUSY, TRSTMI_EUNSUPPORTED, TRSTMI_ENOTFOUND = -5, -6, -7, -8
TRSTMI_ESIZE = -9
FP64, FP32, BF16_SCREEN, FP16_SCREEN = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16_SCREEN, "fp16": FP16_SCREEN}


class TrstmiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = lib().trstmi_last_error().decode() if status == TRSTMI_ECUDA else ""
        super().__init__(f"{what}: {strerror(status)} ({status}) {detail}".rstrip())


class Options(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("precision", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("trace_cap", ctypes.c_int32), ("delta0", ctypes.c_double),
                ("gamma_inc", ctypes.c_double), ("gamma_dec", ctypes.c_double),
                ("delta_min", ctypes.c_double), ("delta_max", ctypes.c_double),
                ("target_mu", ctypes.c_double), ("screen_min_delta", ctypes.c_double),
                ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class TraceRow(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint32), ("cstar", ctypes.c_uint32),
                ("mu2_best", ctypes.c_double), ("mu2_screen", ctypes.c_double),
                ("mu2_cur", ctypes.c_double), ("delta_used", ctypes.c_double),
                ("delta_next", ctypes.c_double), ("accepted", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


TRACE_DTYPE = np.dtype([("t", "<u4"), ("cstar", "<u4"), ("mu2_best", "<f8"),
                        ("mu2_screen", "<f8"), ("mu2_cur", "<f8"), ("delta_used", "<f8"),
                        ("delta_next", "<f8"), ("accepted", "<i4"), ("flags", "<i4")])
assert TRACE_DTYPE.itemsize == ctypes.sizeof(TraceRow)


class StepInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("accepts", ctypes.c_int32),
                ("mu", ctypes.c_double), ("delta", ctypes.c_double),
                ("pairs_scored", ctypes.c_uint64), ("elapsed_ns", ctypes.c_uint64),
                ("done", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/trstmi.h
SIGNATURES = {
    "trstmi_default_options": (None, [ctypes.POINTER(Options)]),
    "trstmi_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]),
    "trstmi_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    "trstmi_coherence": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "trstmi_get_phi": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "trstmi_set_phi": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "trstmi_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_size_t)]),
    "trstmi_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "trstmi_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TraceRow), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]),
    "trstmi_destroy": (None, [ctypes.c_void_p]),
    "trstmi_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "trstmi_last_error": (ctypes.c_char_p, []),
    "trstmi_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]),
    "trstmi_candidate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_double, ctypes.c_int, _dp]),
    "trstmi_mu2_frame": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]),
    "trstmi_profile_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_size_t, _dp]),
    "trstmi_mu2_frame_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
}


def lib():
    """Loads libtrstmi.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libtrstmi.so not built at {LIB_PATH}")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().trstmi_strerror(status).decode()


def _check(status: int, what: str):
    if status < 0:
        raise TrstmiError(status, what)
    return status


def _flat(phi: np.ndarray) -> np.ndarray:
    a = np.asarray(phi, dtype=np.complex128)
    return np.ascontiguousarray(a.T).view(np.float64).reshape(-1).copy()


def _unflat(buf: np.ndarray, d: int, N: int) -> np.ndarray:
    return buf.view(np.complex128).reshape(N, d).T.copy()


def default_options() -> Options:
    o = Options()
    lib().trstmi_default_options(ctypes.byref(o))
    return o


def make_options(**kw) -> Options:
    o = default_options()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Search:
    """One search instance (trstmi_create .. trstmi_destroy)."""

    def __init__(self, N: int, d: int, seed: int, **options):
        self.N, self.d, self.seed = N, d, seed
        self.options = make_options(**options)
        h = ctypes.c_void_p()
        _check(lib().trstmi_create(N, d, seed, ctypes.byref(self.options), ctypes.byref(h)),
               "trstmi_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().trstmi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, iters: int) -> StepInfo:
        info = StepInfo()
        _check(lib().trstmi_step(self._h, iters, ctypes.byref(info)), "trstmi_step")
        return info

    def coherence(self):
        mu, w = ctypes.c_double(), ctypes.c_double()
        _check(lib().trstmi_coherence(self._h, ctypes.byref(mu), ctypes.byref(w)),
               "trstmi_coherence")
        return mu.value, w.value

    def get_phi(self) -> np.ndarray:
        b = np.zeros(2 * self.d * self.N)
        _check(lib().trstmi_get_phi(self._h, b.ctypes.data_as(_dp)), "trstmi_get_phi")
        return _unflat(b, self.d, self.N)

    def set_phi(self, phi: np.ndarray):
        b = _flat(phi)
        _check(lib().trstmi_set_phi(self._h, b.ctypes.data_as(_dp)), "trstmi_set_phi")

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().trstmi_get_state(self._h, None, ctypes.byref(n)), "trstmi_get_state")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().trstmi_get_state(self._h, buf, ctypes.byref(n)), "trstmi_get_state")
        return buf.raw[: n.value]

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().trstmi_set_state(self._h, buf, len(blob)), "trstmi_set_state")

    def trace(self, n: int = 1 << 30) -> np.ndarray:
        cap = max(0, min(n, self.options.trace_cap))
        rows = (TraceRow * max(cap, 1))()
        got = ctypes.c_int()
        _check(lib().trstmi_get_trace(self._h, rows, cap, ctypes.byref(got)), "trstmi_get_trace")
        arr = np.frombuffer(bytes(rows), dtype=TRACE_DTYPE)[: got.value].copy()
        return arr

    def score(self, t: int, c0: int, count: int, delta: float, precision="fp64") -> np.ndarray:
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        out = np.zeros(count)
        _check(lib().trstmi_score(self._h, t, c0, count, delta, p, out.ctypes.data_as(_dp)),
               "trstmi_score")
        return out

    def candidate(self, t: int, c: int, delta: float, precision="fp64") -> np.ndarray:
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        b = np.zeros(2 * self.d * self.N)
        _check(lib().trstmi_candidate(self._h, t, c, delta, p, b.ctypes.data_as(_dp)),
               "trstmi_candidate")
        return _unflat(b, self.d, self.N)


    def profile_score(self, precision="fp32", launches=5, delta=0.1, flush_bytes=0) -> float:
        """Mean device ms of one launch of the scoring kernel (events around it alone)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        out = ctypes.c_double()
        _check(lib().trstmi_profile_score(self._h, p, launches, delta, flush_bytes,
                                          ctypes.byref(out)), "trstmi_profile_score")
        return out.value

    @property
    def handle(self) -> int:
        return self._h.value


def mu2_frame(phi: np.ndarray, precision="fp64") -> float:
    d, N = phi.shape
    p = PRECISIONS[precision] if isinstance(precision, str) else precision
    b = _flat(phi)
    out = ctypes.c_double()
    _check(lib().trstmi_mu2_frame(N, d, b.ctypes.data_as(_dp), p, ctypes.byref(out)),
           "trstmi_mu2_frame")
    return out.value
