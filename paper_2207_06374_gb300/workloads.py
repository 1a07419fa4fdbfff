"""Seeded synthetic workload descriptions (no search arithmetic here).

These only draw the shapes and seeds of the instances a workload runs; the
frames themselves are the library's seeded Philox draws.
"""
from __future__ import annotations

import numpy as np


def batched_instances(n: int = 512, seed: int = 7, d_lo: int = 2, d_hi: int = 16):
    """n instances with d ~ U{d_lo..d_hi} and N ~ U{d+1..d^2}; per-instance
    seeds seed*1_000_003 + i.  Returns (Ns, ds, seeds) lists."""
    rng = np.random.default_rng(seed)
    ds = rng.integers(d_lo, d_hi + 1, size=n)
    Ns = np.array([rng.integers(d + 1, d * d + 1) for d in ds])
    seeds = [seed * 1_000_003 + i for i in range(n)]
    return [int(x) for x in Ns], [int(x) for x in ds], seeds


def serving_requests(n: int = 10000, seed: int = 11, rate_hz: float = 200.0, d_lo: int = 4,
                     d_hi: int = 64, n_max: int = 4096):
    """Poisson arrival stream of search requests: inter-arrival ~ Exp(rate),
    d ~ U{d_lo..d_hi}, N log-uniform on [d+1, n_max] (rounded), a seed each.
    Returns a list of dicts with t_arrive (s), N, d, seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps)
    out = []
    for i in range(n):
        d = int(rng.integers(d_lo, d_hi + 1))
        lo, hi = np.log(d + 1), np.log(n_max)
        N = int(round(float(np.exp(rng.uniform(lo, hi)))))
        N = max(d + 1, min(N, n_max))
        out.append({"t_arrive": float(t[i]), "N": N, "d": d, "seed": seed * 7_000_001 + i})
    return out
