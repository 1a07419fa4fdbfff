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
FP64, FP32, BF16_SCREEN, FP16_SCREEN, TF32_SCREEN = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16_SCREEN, "fp16": FP16_SCREEN,
              "tf32": TF32_SCREEN}


class TrstmiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = lib().trstmi_last_error().decode() if status == TRSTMI_ECUDA else ""
        super().__init__(f"{what}: {strerror(status)} ({status}) {detail}".rstrip())


# trstmi_options.dev_alloc / dev_free
DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("precision", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("trace_cap", ctypes.c_int32), ("delta0", ctypes.c_double),
                ("gamma_inc", ctypes.c_double), ("gamma_dec", ctypes.c_double),
                ("delta_min", ctypes.c_double), ("delta_max", ctypes.c_double),
                ("target_mu", ctypes.c_double), ("screen_min_delta", ctypes.c_double),
                ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class TorchAllocator:
    """Device memory for a handle from PyTorch's caching allocator.

    Passed as ``allocator=`` to Search, Batch or Server, it fills the options'
    dev_alloc / dev_free callbacks, so every device allocation of the handle
    comes from (and returns to) torch's pool on the handle's device instead
    of cudaMalloc / cudaFree.  The object must outlive the handle (the
    handle's Python wrapper keeps a reference).  ``allocs``, ``frees`` and
    ``live`` count what went through it.
    """

    def __init__(self, device: int = 0):
        import torch  # the binding itself does not need torch; this allocator does
        self._torch = torch
        self.device = device
        self.live = {}
        self.allocs = 0
        self.frees = 0

        def _alloc(nbytes, _ctx):
            try:
                p = int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device))
            except Exception:  # out of memory: the library reports TRSTMI_ENOMEM
                return None
            self.live[p] = int(nbytes)
            self.allocs += 1
            return p

        def _free(ptr, _ctx):
            if ptr is None:
                return
            self.live.pop(int(ptr), None)
            self.frees += 1
            self._torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = DEV_ALLOC_FN(_alloc)
        self._free = DEV_FREE_FN(_free)

    def install(self, o: "Options") -> None:
        o.dev_alloc = self._alloc
        o.dev_free = self._free
        o.alloc_ctx = None


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


class ServerOpts(ctypes.Structure):
    _fields_ = [("search", Options), ("hbm_budget", ctypes.c_size_t),
                ("max_slots", ctypes.c_int32), ("iters_per_round", ctypes.c_int32),
                ("queue_cap", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_resident_pairs", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("d", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("budget_iters", ctypes.c_int32), ("want_phi", ctypes.c_int32),
                ("target_mu", ctypes.c_double), ("target_rel_welch", ctypes.c_double),
                ("deadline_ms", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("accepts", ctypes.c_int32), ("reached_target", ctypes.c_int32),
                ("mu", ctypes.c_double), ("welch", ctypes.c_double),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("pairs_scored", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("pairs_scored", ctypes.c_uint64),
                ("gpu_busy_s", ctypes.c_double), ("hbm_in_use", ctypes.c_size_t),
                ("active_slots", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("worker_status", ctypes.c_int32), ("timed_out", ctypes.c_int32),
                ("kernel_launches", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)

class Certificates(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("mu_min", ctypes.c_double),
                ("welch", ctypes.c_double), ("orthoplex", ctypes.c_double),
                ("levenshtein", ctypes.c_double), ("lower_bound", ctypes.c_double),
                ("gap", ctypes.c_double), ("min_chordal", ctypes.c_double),
                ("distinct", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", ctypes.c_double), ("fp64_tflops", ctypes.c_double),
                ("tf32_tflops", ctypes.c_double), ("bf16_tflops", ctypes.c_double)]


class TrOptions(ctypes.Structure):
    _fields_ = [("n_delta", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("delta", ctypes.c_double * 16), ("max_cg", ctypes.c_int32),
                ("path", ctypes.c_int32), ("radius0", ctypes.c_double),
                ("radius_max", ctypes.c_double), ("eta", ctypes.c_double),
                ("gtol", ctypes.c_double), ("fd_step", ctypes.c_double),
                ("hessian", ctypes.c_int32), ("reserved", ctypes.c_int32)]


TR_ROW_DTYPE = np.dtype([("stage", "<i4"), ("iter", "<i4"), ("F", "<f8"), ("s", "<f8"),
                         ("gnorm", "<f8"), ("radius", "<f8"), ("rho", "<f8"),
                         ("step_norm", "<f8"), ("pred", "<f8"), ("cg_iters", "<i4"),
                         ("cg_status", "<i4"), ("accepted", "<i4"), ("reserved", "<i4")])


def tr_options(deltas=None, **kw) -> TrOptions:
    """hessian: "exact" (default) or "difference" (or the enum value)."""
    o = TrOptions()
    lib().trstmi_tr_default_options(ctypes.byref(o))
    h = kw.pop("hessian", None)
    if h is not None:
        o.hessian = {"exact": 0, "difference": 1}.get(h, h)
    if deltas is not None:
        o.n_delta = len(deltas)
        for i, x in enumerate(deltas):
            o.delta[i] = x
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class MultistartResult(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("best", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("best_seed", ctypes.c_uint64)]


# name -> (restype, argtypes); mirrors include/trstmi.h
SIGNATURES = {
    "trstmi_default_options": (None, [ctypes.POINTER(Options)]),
    "trstmi_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]),
    "trstmi_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    "trstmi_shard_score_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "trstmi_shard_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p]),
    "trstmi_shard_finish": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(StepInfo)]),
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
    "trstmi_last_ranking": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_uint32),
                                           _dp]),
    "trstmi_candidate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_double, ctypes.c_int, _dp]),
    "trstmi_mu2_frame": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]),
    "trstmi_profile_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_size_t, _dp]),
    "trstmi_lse_frames": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                         ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]),
    "trstmi_lse_scratch_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "trstmi_lse_frames_device": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "trstmi_frame_certificates": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp,
                                                 ctypes.c_double, ctypes.POINTER(Certificates)]),
    "trstmi_instance_certificates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double,
                                           ctypes.POINTER(Certificates)]),
    "trstmi_tr_default_options": (None, [ctypes.POINTER(TrOptions)]),
    "trstmi_tr_solve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(TrOptions),
                                       ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "trstmi_tr_multistart": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_int, ctypes.POINTER(TrOptions),
                                            ctypes.c_int, ctypes.POINTER(MultistartResult), _dp,
                                            _dp, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "trstmi_instance_tr_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TrOptions),
                                                ctypes.c_void_p, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_int)]),
    "trstmi_multistart": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options),
                                         ctypes.c_int, ctypes.POINTER(MultistartResult), _dp,
                                         _dp]),
    "trstmi_measure_peaks": (ctypes.c_int, [ctypes.POINTER(Peaks), ctypes.c_void_p]),
    "trstmi_screen_wait_test": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "trstmi_mu2_frame_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "trstmi_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(Options),
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "trstmi_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StepInfo)]),
    "trstmi_batch_mu": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_int32)]),
    "trstmi_batch_get_phi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "trstmi_batch_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                              ctypes.POINTER(TraceRow), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    "trstmi_batch_tile_widths": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "trstmi_batch_profile_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
                                                  _dp]),
    "trstmi_batch_destroy": (None, [ctypes.c_void_p]),
    "trstmi_default_server_opts": (None, [ctypes.POINTER(ServerOpts)]),
    "trstmi_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts),
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "trstmi_server_destroy": (None, [ctypes.c_void_p]),
    "trstmi_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "trstmi_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result), _dp]),
    "trstmi_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.POINTER(Result), _dp]),
    "trstmi_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "trstmi_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
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
    alloc = kw.pop("allocator", None)
    if alloc is not None:
        alloc.install(o)
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
        self.allocator = options.get("allocator")
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

    # candidate sharding (include/trstmi.h): scores is a device buffer of
    # shard_score_bytes() bytes given by its address (e.g. tensor.data_ptr())
    def shard_score_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().trstmi_shard_score_bytes(self._h, ctypes.byref(n)), "trstmi_shard_score_bytes")
        return n.value

    def shard_score(self, c_lo: int, c_hi: int, scores_ptr: int) -> None:
        _check(lib().trstmi_shard_score(self._h, c_lo, c_hi, ctypes.c_void_p(scores_ptr)),
               "trstmi_shard_score")

    def shard_finish(self, scores_ptr: int) -> StepInfo:
        info = StepInfo()
        _check(lib().trstmi_shard_finish(self._h, ctypes.c_void_p(scores_ptr), ctypes.byref(info)),
               "trstmi_shard_finish")
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

    def last_ranking(self):
        """(ranking scores of the last iteration's K candidates, survivor
        indices, their binary32 re-scores); the last two are None outside the
        screen modes."""
        K, k = self.options.K, self.options.topk
        mu2 = np.zeros(K)
        screen = self.options.precision in (BF16_SCREEN, FP16_SCREEN, TF32_SCREEN)
        if screen:
            idx = np.zeros(k, dtype=np.uint32)
            top = np.zeros(k)
            _check(lib().trstmi_last_ranking(self._h, mu2.ctypes.data_as(_dp),
                                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                             top.ctypes.data_as(_dp)), "trstmi_last_ranking")
            return mu2, idx, top
        _check(lib().trstmi_last_ranking(self._h, mu2.ctypes.data_as(_dp), None, None),
               "trstmi_last_ranking")
        return mu2, None, None

    def candidate(self, t: int, c: int, delta: float, precision="fp64") -> np.ndarray:
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        b = np.zeros(2 * self.d * self.N)
        _check(lib().trstmi_candidate(self._h, t, c, delta, p, b.ctypes.data_as(_dp)),
               "trstmi_candidate")
        return _unflat(b, self.d, self.N)


    def tr_solve(self, cap: int = 1 << 16, **options):
        """Polish the current frame with the trust-region procedure; returns the trace."""
        o = tr_options(**options)
        tr = np.zeros(max(cap, 1), dtype=TR_ROW_DTYPE)
        n = ctypes.c_int()
        _check(lib().trstmi_instance_tr_solve(self._h, ctypes.byref(o), tr.ctypes.data, cap,
                                              ctypes.byref(n)), "trstmi_instance_tr_solve")
        return tr[: min(n.value, cap)]

    def certificates(self, tol: float = 1e-6) -> dict:
        """Coherence, bounds and distinct distances of the current frame."""
        c = Certificates()
        _check(lib().trstmi_instance_certificates(self._h, tol, ctypes.byref(c)),
               "trstmi_instance_certificates")
        return c.as_dict()

    def profile_score(self, precision="fp32", launches=5, delta=0.1, flush_bytes=0) -> float:
        """Mean device ms of one launch of the scoring kernel (events around it alone)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        out = ctypes.c_double()
        _check(lib().trstmi_profile_score(self._h, p, launches, delta, flush_bytes,
                                          ctypes.byref(out)), "trstmi_profile_score")
        return out.value

    def screen_wait_test(self, precision="bf16", wait_limit_ms=20.0) -> int:
        """Status of a screen launch whose block producers are withheld, so its
        bounded wait runs out after wait_limit_ms (TRSTMI_ETIMEOUT expected)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else precision
        return lib().trstmi_screen_wait_test(self._h, p, wait_limit_ms)

    @property
    def handle(self) -> int:
        return self._h.value


def tr_solve(phi: np.ndarray, cap: int = 1 << 16, **options):
    """The paper's trust-region CG-Steihaug procedure over the smoothing
    stages on a frame (d, N), on the GPU in binary64.  Returns (the result,
    unit columns; the per-iteration trace)."""
    d, N = phi.shape
    o = tr_options(**options)
    b = _flat(phi)
    tr = np.zeros(max(cap, 1), dtype=TR_ROW_DTYPE)
    n = ctypes.c_int()
    _check(lib().trstmi_tr_solve(N, d, b.ctypes.data_as(_dp), ctypes.byref(o), tr.ctypes.data,
                                 cap, ctypes.byref(n)), "trstmi_tr_solve")
    return _unflat(b, d, N), tr[: min(n.value, cap)]


def tr_multistart(N: int, d: int, seed0: int, L: int = 0, batch_cap: int = 0,
                  want_phi: bool = True, trace_cap: int = 0, work=None, **options):
    """The paper's whole algorithm: L random initialisations (seeds seed0 ..,
    the frames trstmi_create draws; L <= 0: 2 d^2), each through the
    trust-region procedure, advanced together on the GPU; the minimum over
    the trials.  Returns (result, mu of every trial, the winning frame or
    None, the winning trial's trace).  `work`, an int32 array of shape
    (trials, 2), receives each trial's trust-region iterations and
    Hessian-vector products."""
    o = tr_options(**options)
    trials = L if L > 0 else 2 * d * d
    if work is not None and (work.dtype != np.int32 or work.shape != (trials, 2)
                             or not work.flags.c_contiguous):
        raise ValueError(f"work must be a C-contiguous int32 array of shape ({trials}, 2)")
    res = MultistartResult()
    mus = np.zeros(trials)
    phi = np.zeros(2 * d * N) if want_phi else None
    tr = np.zeros(max(trace_cap, 1), dtype=TR_ROW_DTYPE)
    n = ctypes.c_int()
    _check(lib().trstmi_tr_multistart(N, d, seed0, L, ctypes.byref(o), batch_cap,
                                      ctypes.byref(res), mus.ctypes.data_as(_dp),
                                      phi.ctypes.data_as(_dp) if want_phi else None,
                                      tr.ctypes.data if trace_cap > 0 else None, trace_cap,
                                      ctypes.byref(n),
                                      work.ctypes.data if work is not None else None),
           "trstmi_tr_multistart")
    return (res, mus, (_unflat(phi, d, N) if want_phi else None),
            tr[: min(n.value, trace_cap)] if trace_cap > 0 else None)


def certificates(phi: np.ndarray, tol: float = 1e-6) -> dict:
    """Coherence, bounds, smallest chordal distance and distinct distances of a
    frame (d, N) computed on the GPU in binary64."""
    d, N = phi.shape
    b = _flat(phi)
    c = Certificates()
    _check(lib().trstmi_frame_certificates(N, d, b.ctypes.data_as(_dp), tol, ctypes.byref(c)),
           "trstmi_frame_certificates")
    return c.as_dict()


def multistart(N: int, d: int, seed0: int, L: int, iters: int, batch_cap: int = 0,
               want_phi: bool = True, **options):
    """L random initialisations (seeds seed0 ..), each searched for `iters`
    iterations, and the minimum over the trials.  Returns (result, mu of every
    trial, the winning frame or None)."""
    o = make_options(**options)
    trials = L if L > 0 else 2 * d * d
    res = MultistartResult()
    mus = np.zeros(trials)
    phi = np.zeros(2 * d * N) if want_phi else None
    _check(lib().trstmi_multistart(N, d, seed0, L, iters, ctypes.byref(o), batch_cap,
                                   ctypes.byref(res), mus.ctypes.data_as(_dp),
                                   phi.ctypes.data_as(_dp) if want_phi else None),
           "trstmi_multistart")
    return res, mus, (_unflat(phi, d, N) if want_phi else None)


class Batch:
    """Many searches advanced together (trstmi_batch_create .. _destroy)."""

    def __init__(self, Ns, ds, seeds, **options):
        self.Ns, self.ds = [int(x) for x in Ns], [int(x) for x in ds]
        self.seeds = [int(x) for x in seeds]
        self.n = len(self.Ns)
        self.allocator = options.get("allocator")
        self.options = make_options(**options)
        Na = (ctypes.c_int * self.n)(*self.Ns)
        da = (ctypes.c_int * self.n)(*self.ds)
        sa = (ctypes.c_uint64 * self.n)(*self.seeds)
        h = ctypes.c_void_p()
        _check(lib().trstmi_batch_create(self.n, Na, da, sa, ctypes.byref(self.options),
                                         ctypes.byref(h)), "trstmi_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().trstmi_batch_destroy(self._h)
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
        _check(lib().trstmi_batch_step(self._h, iters, ctypes.byref(info)), "trstmi_batch_step")
        return info

    def mu(self):
        out = np.zeros(self.n)
        it = (ctypes.c_int32 * self.n)()
        _check(lib().trstmi_batch_mu(self._h, out.ctypes.data_as(_dp), it), "trstmi_batch_mu")
        return out, np.array(list(it))

    def get_phi(self, i: int) -> np.ndarray:
        b = np.zeros(2 * self.ds[i] * self.Ns[i])
        _check(lib().trstmi_batch_get_phi(self._h, i, b.ctypes.data_as(_dp)), "trstmi_batch_get_phi")
        return _unflat(b, self.ds[i], self.Ns[i])

    def trace(self, i: int, n: int = 1 << 30) -> np.ndarray:
        cap = max(0, min(n, self.options.trace_cap))
        rows = (TraceRow * max(cap, 1))()
        got = ctypes.c_int()
        _check(lib().trstmi_batch_get_trace(self._h, i, rows, cap, ctypes.byref(got)),
               "trstmi_batch_get_trace")
        return np.frombuffer(bytes(rows), dtype=TRACE_DTYPE)[: got.value].copy()

    def tile_widths(self):
        w = (ctypes.c_int * self.n)()
        _check(lib().trstmi_batch_tile_widths(self._h, w), "trstmi_batch_tile_widths")
        return list(w)

    def profile_score(self, launches=3, flush_bytes=0) -> float:
        out = ctypes.c_double()
        _check(lib().trstmi_batch_profile_score(self._h, launches, flush_bytes, ctypes.byref(out)),
               "trstmi_batch_profile_score")
        return out.value


class Server:
    """The serving loop (trstmi_server_create .. _destroy)."""

    def __init__(self, hbm_budget=4 << 30, max_slots=256, iters_per_round=20, queue_cap=1 << 16,
                 max_resident_pairs=None, **search):
        o = ServerOpts()
        lib().trstmi_default_server_opts(ctypes.byref(o))
        o.hbm_budget, o.max_slots = hbm_budget, max_slots
        o.iters_per_round, o.queue_cap = iters_per_round, queue_cap
        if max_resident_pairs is not None:
            o.max_resident_pairs = max_resident_pairs
        self.allocator = search.pop("allocator", None)
        if self.allocator is not None:
            self.allocator.install(o.search)
        for k, v in search.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            if not hasattr(o.search, k):
                raise TypeError(f"unknown option {k}")
            setattr(o.search, k, v)
        self.opts = o
        h = ctypes.c_void_p()
        _check(lib().trstmi_server_create(ctypes.byref(o), ctypes.byref(h)), "trstmi_server_create")
        self._h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().trstmi_server_destroy(self._h)
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

    def submit(self, N, d, seed, budget_iters, target_mu=0.0, target_rel_welch=0.0,
               want_phi=False, deadline_ms=0.0) -> int:
        r = Request(N, d, seed, budget_iters, int(bool(want_phi)), target_mu, target_rel_welch,
                    deadline_ms)
        t = ctypes.c_uint64()
        _check(lib().trstmi_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "trstmi_submit")
        self._shapes[t.value] = (d, N)
        return t.value

    def poll(self, ticket, with_phi=False):
        res = Result()
        phi = None
        buf = None
        if with_phi and ticket in self._shapes:
            d, N = self._shapes[ticket]
            buf = np.zeros(2 * d * N)
        st = lib().trstmi_poll(self._h, ticket, ctypes.byref(res),
                               buf.ctypes.data_as(_dp) if buf is not None else None)
        if buf is not None and st == TRSTMI_OK:
            phi = _unflat(buf, *self._shapes[ticket])
        return st, res, phi

    def wait(self, ticket, timeout_ms=600000, with_phi=False):
        res = Result()
        buf = None
        if with_phi and ticket in self._shapes:
            d, N = self._shapes[ticket]
            buf = np.zeros(2 * d * N)
        st = lib().trstmi_wait(self._h, ticket, timeout_ms, ctypes.byref(res),
                               buf.ctypes.data_as(_dp) if buf is not None else None)
        phi = _unflat(buf, *self._shapes[ticket]) if (buf is not None and st == TRSTMI_OK) else None
        return st, res, phi

    def cancel(self, ticket) -> int:
        return lib().trstmi_cancel(self._h, ticket)

    def stats(self) -> ServerStats:
        s = ServerStats()
        _check(lib().trstmi_server_stats(self._h, ctypes.byref(s)), "trstmi_server_stats")
        return s


def lse(v: np.ndarray, delta: float, precision="fp64", grad: bool = True):
    """The paper's smooth maximum F_{s,delta} of |G_jk|^2 (j < k) of the
    column-normalised frame of V, s = max |G_jk|^2, and the real gradient in
    V (dF/dRe V + i dF/dIm V).  v: (d, N) or a stack (count, d, N) of complex
    frames; returns (F, s, grad) as scalars and a (d, N) array, or arrays."""
    v = np.asarray(v, dtype=np.complex128)
    single = v.ndim == 2
    if single:
        v = v[None]
    count, d, N = v.shape
    p = PRECISIONS[precision] if isinstance(precision, str) else precision
    b = np.ascontiguousarray(np.transpose(v, (0, 2, 1))).view(np.float64).reshape(-1).copy()
    F = np.zeros(count)
    s = np.zeros(count)
    g = np.zeros_like(b) if grad else None
    _check(lib().trstmi_lse_frames(N, d, count, b.ctypes.data_as(_dp), delta, p,
                                   F.ctypes.data_as(_dp), s.ctypes.data_as(_dp),
                                   g.ctypes.data_as(_dp) if grad else None), "trstmi_lse_frames")
    G = None
    if grad:
        G = g.view(np.complex128).reshape(count, N, d).transpose(0, 2, 1).copy()
    if single:
        return float(F[0]), float(s[0]), (G[0] if grad else None)
    return F, s, G


def lse_scratch_bytes(N: int, d: int, count: int, precision="fp32") -> int:
    p = PRECISIONS[precision] if isinstance(precision, str) else precision
    out = ctypes.c_size_t()
    _check(lib().trstmi_lse_scratch_bytes(N, d, count, p, ctypes.byref(out)),
           "trstmi_lse_scratch_bytes")
    return out.value


def lse_device(N: int, d: int, count: int, v_ptr: int, delta: float, precision, scratch_ptr: int,
               scratch_bytes: int, out_ptr: int, grad_ptr: int = 0, stream: int = 0) -> None:
    """Allocation-free smooth maximum on device buffers (raw pointers); only
    enqueues on `stream`."""
    p = PRECISIONS[precision] if isinstance(precision, str) else precision
    _check(lib().trstmi_lse_frames_device(N, d, count, v_ptr, delta, p, scratch_ptr,
                                          scratch_bytes, out_ptr, grad_ptr or None,
                                          stream or None), "trstmi_lse_frames_device")


def measure_peaks(stream: int = 0) -> dict:
    """TFLOP/s of FFMA, DFMA and the bf16 / tf32 tensor cores on the current
    device (trstmi_measure_peaks)."""
    p = Peaks()
    _check(lib().trstmi_measure_peaks(ctypes.byref(p), ctypes.c_void_p(stream)),
           "trstmi_measure_peaks")
    return {k: getattr(p, k) for k, _ in p._fields_}


def mu2_frame(phi: np.ndarray, precision="fp64") -> float:
    d, N = phi.shape
    p = PRECISIONS[precision] if isinstance(precision, str) else precision
    b = _flat(phi)
    out = ctypes.c_double()
    _check(lib().trstmi_mu2_frame(N, d, b.ctypes.data_as(_dp), p, ctypes.byref(out)),
           "trstmi_mu2_frame")
    return out.value
