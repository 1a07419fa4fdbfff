"""ctypes loader for the TRSTMI CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and
its binding) never imports or calls it.  See ``trstmi_oracle.c`` for what the
oracle computes and the passages of arXiv 2207.06374 each part follows.

Frames are numpy complex128 arrays of shape (d, N) here; the C side stores
them column-major with interleaved (re, im), which is the memory layout of
``np.asfortranarray(phi)`` viewed as float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trstmi_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) into _build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC",
                               "-shared", "-ffp-contract=off", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class OracleOpts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("T", ctypes.c_int),
                ("delta0", ctypes.c_double), ("gamma_inc", ctypes.c_double),
                ("gamma_dec", ctypes.c_double), ("delta_min", ctypes.c_double),
                ("delta_max", ctypes.c_double), ("target_mu", ctypes.c_double)]


class TraceRow(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint32), ("cstar", ctypes.c_uint32),
                ("mu2_best", ctypes.c_double), ("mu2_cur", ctypes.c_double),
                ("delta_used", ctypes.c_double), ("delta_next", ctypes.c_double),
                ("accepted", ctypes.c_int32), ("pad", ctypes.c_int32)]


TRACE_DTYPE = np.dtype([("t", "<u4"), ("cstar", "<u4"), ("mu2_best", "<f8"),
                        ("mu2_cur", "<f8"), ("delta_used", "<f8"),
                        ("delta_next", "<f8"), ("accepted", "<i4"), ("pad", "<i4")])
assert TRACE_DTYPE.itemsize == ctypes.sizeof(TraceRow)

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
HV_FN = ctypes.CFUNCTYPE(None, _dp, _dp, ctypes.c_void_p)


class TrOpts(ctypes.Structure):
    _fields_ = [("n_delta", ctypes.c_int), ("delta", ctypes.c_double * 16),
                ("max_outer", ctypes.c_int), ("max_cg", ctypes.c_int),
                ("radius0", ctypes.c_double), ("radius_max", ctypes.c_double),
                ("eta", ctypes.c_double), ("gtol", ctypes.c_double),
                ("fd_step", ctypes.c_double), ("hessian", ctypes.c_int),
                ("pad", ctypes.c_int)]


TR_DTYPE = np.dtype([("stage", "<i4"), ("iter", "<i4"), ("F", "<f8"), ("s", "<f8"),
                     ("gnorm", "<f8"), ("radius", "<f8"), ("rho", "<f8"),
                     ("step_norm", "<f8"), ("pred", "<f8"), ("cg_iters", "<i4"),
                     ("cg_status", "<i4"), ("accepted", "<i4"), ("pad", "<i4")])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.oracle_gauss_entry.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, _dp, _dp]
            L.oracle_mu2.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
            L.oracle_mu2.restype = ctypes.c_double
            L.oracle_gram_abs2.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int]
            L.oracle_gram_abs2.restype = ctypes.c_double
            L.oracle_welch.argtypes = [ctypes.c_int, ctypes.c_int]
            L.oracle_welch.restype = ctypes.c_double
            L.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _dp]
            L.oracle_candidate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _dp,
                                           ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, _dp]
            L.oracle_score.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _dp,
                                       ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int, _dp, ctypes.c_int]
            L.oracle_score_f32.argtypes = L.oracle_score.argtypes
            L.oracle_search.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.POINTER(OracleOpts), _dp, _dp, _dp,
                                        ctypes.c_uint32, ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_void_p, ctypes.c_int]
            L.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.POINTER(OracleOpts), _dp, _dp, _dp,
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_int]
            L.oracle_replay.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.POINTER(OracleOpts), _dp, _dp, _dp,
                                        ctypes.c_uint32, ctypes.c_int, _u32p, ctypes.c_void_p]
            L.oracle_lse.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp, _dp,
                                     _dp]
            for f in ("oracle_orthoplex", "oracle_levenshtein"):
                getattr(L, f).argtypes = [ctypes.c_int, ctypes.c_int]
                getattr(L, f).restype = ctypes.c_double
            L.oracle_gram_extremes.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_gram_extremes.restype = None
            L.oracle_distinct_distances.argtypes = [ctypes.c_int, ctypes.c_int, _dp,
                                                    ctypes.c_double]
            L.oracle_distinct_distances.restype = ctypes.c_int
            L.oracle_cg_steihaug.argtypes = [ctypes.c_int, _dp, HV_FN, ctypes.c_void_p,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             _dp, _dp, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]
            L.oracle_lse_hv.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                        ctypes.c_double, _dp, _dp]
            L.oracle_lse_hv_exact.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                              _dp, _dp]
            L.oracle_lse_hv_exact.restype = ctypes.c_int
            L.oracle_tr_solve.argtypes = [ctypes.c_int, ctypes.c_int, _dp,
                                          ctypes.POINTER(TrOpts), ctypes.c_void_p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]
            for f in ("oracle_init", "oracle_candidate", "oracle_score", "oracle_score_f32",
                      "oracle_search",
                      "oracle_run", "oracle_replay", "oracle_lse", "oracle_cg_steihaug",
                      "oracle_lse_hv", "oracle_tr_solve"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _flat(phi: np.ndarray) -> np.ndarray:
    """(d, N) complex -> contiguous float64 buffer, column-major interleaved."""
    a = np.asarray(phi, dtype=np.complex128)
    return np.ascontiguousarray(a.T).view(np.float64).reshape(-1).copy()


def _unflat(buf: np.ndarray, d: int, N: int) -> np.ndarray:
    return buf.view(np.complex128).reshape(N, d).T.copy()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check(st: int, what: str):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def gauss_entry(seed, d, i, j, c, t, tag):
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_gauss_entry(seed, d, i, j, c, t, tag, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def mu2(phi: np.ndarray) -> float:
    d, N = phi.shape
    b = _flat(phi)
    return float(lib().oracle_mu2(N, d, _ptr(b)))


def mu(phi: np.ndarray) -> float:
    return float(np.sqrt(mu2(phi)))


def welch(N: int, d: int) -> float:
    return float(lib().oracle_welch(N, d))


def init(N: int, d: int, seed: int) -> np.ndarray:
    b = np.zeros(2 * d * N)
    _check(lib().oracle_init(N, d, seed, _ptr(b)), "init")
    return _unflat(b, d, N)


def candidate(phi: np.ndarray, seed: int, delta: float, t: int, c: int) -> np.ndarray:
    d, N = phi.shape
    b = _flat(phi)
    o = np.zeros_like(b)
    _check(lib().oracle_candidate(N, d, seed, _ptr(b), delta, t, c, _ptr(o)), "candidate")
    return _unflat(o, d, N)


def score(phi: np.ndarray, seed: int, delta: float, t: int, c0: int, K: int,
          nthreads: int = 1) -> np.ndarray:
    """mu^2 of candidates c0..c0+K-1 of iteration t (float64 array of K)."""
    d, N = phi.shape
    b = _flat(phi)
    out = np.zeros(K)
    _check(lib().oracle_score(N, d, seed, _ptr(b), delta, t, c0, K, _ptr(out), nthreads),
           "score")
    return out


def score_f32(phi: np.ndarray, seed: int, delta: float, t: int, c0: int, K: int,
              nthreads: int = 1) -> np.ndarray:
    """mu^2 of K candidates by the binary32 plain-loop variant (a timing
    baseline; equal to score() within binary32 rounding)."""
    d, N = phi.shape
    b = _flat(phi)
    out = np.zeros(K)
    _check(lib().oracle_score_f32(N, d, seed, _ptr(b), delta, t, c0, K, _ptr(out), nthreads),
           "score_f32")
    return out


def make_opts(K=256, T=100, delta0=0.1, gamma_inc=2.0, gamma_dec=0.25,
              delta_min=1e-9, delta_max=1.0, target_mu=0.0) -> OracleOpts:
    return OracleOpts(K, T, delta0, gamma_inc, gamma_dec, delta_min, delta_max, target_mu)


def run(N: int, d: int, seed: int, opts: OracleOpts, nthreads: int = 1):
    """Whole search from the seeded init.  Returns (phi, mu2, delta, trace)."""
    b = np.zeros(2 * d * N)
    m2, dl = ctypes.c_double(), ctypes.c_double()
    it = ctypes.c_int()
    tr = np.zeros(max(opts.T, 1), dtype=TRACE_DTYPE)
    _check(lib().oracle_run(N, d, seed, ctypes.byref(opts), _ptr(b), ctypes.byref(m2),
                            ctypes.byref(dl), ctypes.byref(it), tr.ctypes.data, nthreads),
           "run")
    return _unflat(b, d, N), m2.value, dl.value, tr[: it.value]


def search(phi: np.ndarray, seed: int, opts: OracleOpts, delta: float, mu2_cur: float,
           t0: int, nthreads: int = 1):
    """Continue a search from a given state.  Returns (phi, mu2, delta, trace)."""
    d, N = phi.shape
    b = _flat(phi)
    m2, dl = ctypes.c_double(mu2_cur), ctypes.c_double(delta)
    it = ctypes.c_int()
    tr = np.zeros(max(opts.T, 1), dtype=TRACE_DTYPE)
    _check(lib().oracle_search(N, d, seed, ctypes.byref(opts), _ptr(b), ctypes.byref(dl),
                               ctypes.byref(m2), t0, ctypes.byref(it), tr.ctypes.data,
                               nthreads), "search")
    return _unflat(b, d, N), m2.value, dl.value, tr[: it.value]


def replay(phi: np.ndarray, seed: int, opts: OracleOpts, delta: float, mu2_cur: float,
           t0: int, cstar_seq):
    """Re-run the accept/radius rule on a given candidate choice per iteration."""
    d, N = phi.shape
    b = _flat(phi)
    cs = np.ascontiguousarray(np.asarray(cstar_seq, dtype=np.uint32))
    m2, dl = ctypes.c_double(mu2_cur), ctypes.c_double(delta)
    tr = np.zeros(max(len(cs), 1), dtype=TRACE_DTYPE)
    _check(lib().oracle_replay(N, d, seed, ctypes.byref(opts), _ptr(b), ctypes.byref(dl),
                               ctypes.byref(m2), t0, len(cs),
                               cs.ctypes.data_as(_u32p), tr.ctypes.data), "replay")
    return _unflat(b, d, N), m2.value, dl.value, tr[: len(cs)]


def lse(v: np.ndarray, delta: float, grad: bool = True):
    """Smooth maximum F_{s,delta} of |G_jk|^2 (j < k) of the column-normalised
    frame of V (d, N), its s = max |G_jk|^2, and the real gradient in V as a
    complex (d, N) array (dF/dRe V + i dF/dIm V), or None."""
    d, N = v.shape
    b = _flat(v)
    Fv, sv = ctypes.c_double(), ctypes.c_double()
    g = np.zeros_like(b) if grad else None
    _check(lib().oracle_lse(N, d, _ptr(b), delta, ctypes.byref(Fv), ctypes.byref(sv),
                            _ptr(g) if grad else None), "lse")
    return Fv.value, sv.value, (_unflat(g, d, N) if grad else None)


def orthoplex(N: int, d: int) -> float:
    return float(lib().oracle_orthoplex(N, d))


def levenshtein(N: int, d: int) -> float:
    return float(lib().oracle_levenshtein(N, d))


def gram_extremes(phi: np.ndarray):
    """(max, min) of |G_jk|^2 over j < k."""
    d, N = phi.shape
    b = _flat(phi)
    mx, mn = ctypes.c_double(), ctypes.c_double()
    lib().oracle_gram_extremes(N, d, _ptr(b), ctypes.byref(mx), ctypes.byref(mn))
    return mx.value, mn.value


def distinct_distances(phi: np.ndarray, tol: float) -> int:
    d, N = phi.shape
    b = _flat(phi)
    r = int(lib().oracle_distinct_distances(N, d, _ptr(b), tol))
    if r < 0:
        raise ValueError("oracle distinct_distances: bad arguments")
    return r


def cg_steihaug(g, hv, radius: float, eps: float, maxit: int):
    """CG-Steihaug on m(p) = g.p + p.Bp/2, |p| <= radius; hv(v) -> B v (numpy).
    Returns (p, m(p), iterations, status)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
    n = g.size

    def _cb(vp, op, _ctx):
        v = np.ctypeslib.as_array(vp, shape=(n,))
        o = np.ctypeslib.as_array(op, shape=(n,))
        o[:] = hv(v.copy())

    cb = HV_FN(_cb)
    p = np.zeros(n)
    m, it, st = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _check(lib().oracle_cg_steihaug(n, _ptr(g), cb, None, radius, eps, maxit, _ptr(p),
                                    ctypes.byref(m), ctypes.byref(it), ctypes.byref(st)),
           "cg_steihaug")
    return p, m.value, it.value, st.value


def lse_hv(v: np.ndarray, delta: float, h: float, u: np.ndarray) -> np.ndarray:
    """Hessian of F_{s,delta} at V applied to U by a central difference of the
    exact gradient (complex (d, N) arrays, real inner product)."""
    d, N = v.shape
    b, ub = _flat(v), _flat(u)
    o = np.zeros_like(b)
    _check(lib().oracle_lse_hv(N, d, _ptr(b), delta, h, _ptr(ub), _ptr(o)), "lse_hv")
    return _unflat(o, d, N)


def tr_opts(deltas=(0.1, 0.01, 0.001), max_outer=50, max_cg=50, radius0=0.1, radius_max=1.0,
            eta=1e-4, gtol=1e-9, fd_step=1e-6, hessian="exact") -> TrOpts:
    """hessian: "exact" (B_k, the Hessian of F: the paper's model) or
    "difference" (central differences of the gradient with step fd_step)."""
    o = TrOpts()
    o.hessian = {"exact": 0, "difference": 1}[hessian]
    o.n_delta = len(deltas)
    for i, x in enumerate(deltas):
        o.delta[i] = x
    o.max_outer, o.max_cg = max_outer, max_cg
    o.radius0, o.radius_max, o.eta, o.gtol, o.fd_step = radius0, radius_max, eta, gtol, fd_step
    return o


def tr_solve(v: np.ndarray, opts: TrOpts, cap: int = 4096):
    """The trust-region CG-Steihaug procedure over the smoothing stages.
    Returns (the final frame, unit columns; the per-iteration trace)."""
    d, N = v.shape
    b = _flat(v)
    tr = np.zeros(max(cap, 1), dtype=TR_DTYPE)
    n = ctypes.c_int()
    _check(lib().oracle_tr_solve(N, d, _ptr(b), ctypes.byref(opts), tr.ctypes.data, cap,
                                 ctypes.byref(n)), "tr_solve")
    return _unflat(b, d, N), tr[: min(n.value, cap)]


def lse_hv_exact(v: np.ndarray, delta: float, u: np.ndarray) -> np.ndarray:
    """The exact Hessian of F_{s,delta} at V applied to U (the chain rule
    through the gradient), complex (d, N) arrays."""
    d, N = v.shape
    b, ub = _flat(v), _flat(u)
    o = np.zeros_like(b)
    _check(lib().oracle_lse_hv_exact(N, d, _ptr(b), delta, _ptr(ub), _ptr(o)), "lse_hv_exact")
    return _unflat(o, d, N)
