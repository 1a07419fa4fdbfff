"""Bounded device waits: a stalled tensor-core screen ends with a status.

The screen's roles hand work to each other through shared-memory barriers.
Every wait on one of them gives up after a time limit, flags
TRSTMI_ETIMEOUT and lets the CTA's other roles leave, so a launch whose
producer never delivers ends instead of hanging the GPU.  The test launches
the screen with its block producers withheld (a barrier that nothing
completes) and a short limit, checks the status, and then checks that the
context still computes correct results.
"""
import time

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")


@pytest.mark.parametrize("precision,d", [("bf16", 16), ("tf32", 16), ("bf16", 48)])
def test_stalled_screen_times_out_and_context_survives(precision, d):
    N, seed, K = 200, 11, 32
    with T.Search(N, d, seed, K=K, precision=precision) as s:
        phi0 = s.get_phi()
        t0 = time.perf_counter()
        rc = s.screen_wait_test(precision, wait_limit_ms=20.0)
        elapsed = time.perf_counter() - t0
        assert rc == T.TRSTMI_ETIMEOUT
        # the limit, plus the polling granularity and launch overhead
        assert elapsed < 1.5
        # the search state is untouched and the context still works: screen
        # scores of the same candidates and a binary64 score against the oracle
        assert np.array_equal(s.get_phi(), phi0)
        scr = s.score(1, 0, 8, 0.1, precision)
        ref = O.score(phi0, seed, 0.1, 1, 0, 8, nthreads=4)
        assert np.max(np.abs(np.sqrt(scr) - np.sqrt(ref))) < 4e-3
        got = s.score(1, 0, 8, 0.1, "fp64")
        assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_wait_test_rejects_bad_arguments():
    with T.Search(40, 8, 3, K=8) as s:
        assert s.screen_wait_test("fp32", 20.0) == T.TRSTMI_EINVAL
        assert s.screen_wait_test("bf16", 0.0) == T.TRSTMI_EINVAL
        assert s.screen_wait_test("bf16", 5000.0) == T.TRSTMI_EINVAL
    with T.Search(40, 65, 3, K=8) as s:   # d > 64: outside the screen's range
        assert s.screen_wait_test("bf16", 20.0) == T.TRSTMI_EUNSUPPORTED
