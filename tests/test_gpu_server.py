"""Serving loop: continuous batching of searches in shared launches.

Each request's result must be exactly the one the same search gives alone
(same options, seed, iteration budget and target): its iterations, final mu
and final frame are compared bit for bit with a standalone trstmi_create +
trstmi_step run.  Admission respects the device-memory budget, cancellation
and unknown tickets are reported, and bad arguments are rejected on the host.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")
W = pytest.importorskip("paper_2207_06374_gb300.workloads")


def _alone(N, d, seed, K, budget, target, precision="fp32"):
    with T.Search(N, d, seed, K=K, precision=precision, target_mu=target, trace_cap=0) as s:
        info = s.step(budget)
        return info, s.get_phi()


def test_results_equal_standalone_runs():
    K = 32
    reqs = [(4, 2, 11, 300, 0.5775), (9, 3, 12, 120, 0.0), (30, 5, 13, 80, 0.0),
            (200, 16, 14, 40, 0.0), (7, 3, 15, 200, 0.48), (64, 8, 16, 60, 0.0),
            (1000, 32, 17, 6, 0.0), (3, 2, 18, 50, 0.55)]
    with T.Server(hbm_budget=256 << 20, max_slots=5, iters_per_round=7, K=K,
                  precision="fp32") as srv:
        tickets = []
        for i, (N, d, seed, budget, target) in enumerate(reqs):
            tickets.append(srv.submit(N, d, seed, budget, target_mu=target, want_phi=True))
            if i % 3 == 2:
                time.sleep(0.01)          # later requests arrive while others run
        results = [srv.wait(t, with_phi=True) for t in tickets]
        stats = srv.stats()
    assert stats.completed == len(reqs) and stats.worker_status == 0
    assert stats.pairs_scored == sum(res.pairs_scored for _, res, _ in results)
    for (N, d, seed, budget, target), (st, res, phi) in zip(reqs, results):
        assert st == T.TRSTMI_OK
        info, phi_alone = _alone(N, d, seed, K, budget, target)
        assert res.iters == info.iters_done, (N, d)
        assert res.accepts == info.accepts, (N, d)
        assert res.mu == info.mu, (N, d)
        assert np.array_equal(phi, phi_alone), (N, d)
        assert res.t_submit_ns <= res.t_admit_ns <= res.t_done_ns
        if target > 0 and res.reached_target:
            assert res.mu <= target


@pytest.mark.parametrize("precision", ["bf16", "fp16", "tf32"])
def test_screen_mode_results_equal_standalone_runs(precision):
    """Precision form through the serving loop (screen, fp32 top-k re-score,
    fp64 certification as shared launches over the resident slots): each
    result equals the standalone run of the same request bit for bit."""
    K = 32
    reqs = [(4, 2, 21, 120, 0.5775), (40, 6, 22, 30, 0.0), (300, 24, 23, 10, 0.0),
            (50, 40, 24, 12, 0.0), (1024, 32, 25, 4, 0.0), (12, 4, 26, 40, 0.0),
            (600, 56, 27, 6, 0.0)]
    with T.Server(hbm_budget=256 << 20, max_slots=4, iters_per_round=5, K=K, topk=4,
                  precision=precision) as srv:
        tickets = [srv.submit(N, d, seed, budget, target_mu=target, want_phi=True)
                   for N, d, seed, budget, target in reqs]
        results = [srv.wait(t, with_phi=True) for t in tickets]
        stats = srv.stats()
    assert stats.completed == len(reqs) and stats.worker_status == 0
    for (N, d, seed, budget, target), (st, res, phi) in zip(reqs, results):
        assert st == T.TRSTMI_OK
        with T.Search(N, d, seed, K=K, topk=4, precision=precision, target_mu=target,
                      trace_cap=0) as s:
            info = s.step(budget)
            phi_alone = s.get_phi()
        assert res.iters == info.iters_done, (N, d)
        assert res.mu == info.mu, (N, d)
        assert np.array_equal(phi, phi_alone), (N, d)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16", "tf32"])
def test_served_requests_replay_in_the_oracle(precision):
    """Served requests against the oracle, not only against the CUDA path: a
    mix is served together; for each request the oracle replays in binary64
    the choices its search took (the standalone run of the same request, which
    the served result equals bit for bit, gives the choice sequence) and must
    reproduce the served frame and mu.  Precision form: every accept decision
    and the final frame to 1e-12 (decisions rest on certified binary64 mu).
    Binary32: the chosen candidates' mu to 1e-6 and the decisions wherever the
    improvement exceeds binary32 resolution."""
    K = 48
    reqs = [(9, 3, 41, 40, 0.5001), (30, 5, 42, 25, 0.0), (64, 8, 43, 15, 0.0),
            (150, 12, 44, 10, 0.0)]
    extra = [(600, 24, 45, 6, 0.0), (5, 2, 46, 60, 0.0)]   # served beside them only
    opts = dict(K=K, precision=precision, topk=4) if precision != "fp32" else \
        dict(K=K, precision=precision)
    with T.Server(hbm_budget=256 << 20, max_slots=4, iters_per_round=4, **opts) as srv:
        tickets = [srv.submit(N, d, seed, budget, target_mu=target, want_phi=True)
                   for N, d, seed, budget, target in reqs + extra]
        results = [srv.wait(t, with_phi=True) for t in tickets][: len(reqs)]
    import oracle as O
    from test_gpu_parity import check_precision_form_rows
    for (N, d, seed, budget, target), (st, res, phi) in zip(reqs, results):
        assert st == T.TRSTMI_OK
        with T.Search(N, d, seed, target_mu=target, trace_cap=4096, **opts) as s:
            phi0 = s.get_phi()
            info = s.step(budget)
            tr = s.trace()
            assert np.array_equal(s.get_phi(), phi)
        assert res.iters == info.iters_done == len(tr)
        oo = O.make_opts(K=K, T=res.iters, target_mu=target)
        m0 = O.mu2(phi0)
        rphi, rm2, _, rtr = O.replay(phi0, seed, oo, 0.1, m0, 0, tr["cstar"])
        if precision == "fp32":
            gaps = np.abs(np.sqrt(rtr["mu2_best"]) - np.sqrt(np.maximum(rtr["mu2_cur"], 0)))
            clear = gaps > 1e-5
            assert np.array_equal(tr["accepted"][clear], rtr["accepted"][clear])
            assert np.max(np.abs(np.sqrt(tr["mu2_best"]) - np.sqrt(rtr["mu2_best"]))) < 1e-6
            assert abs(res.mu - np.sqrt(O.mu2(phi.astype(np.complex64).astype(complex)))) < 1e-6
        else:
            check_precision_form_rows(tr, rtr, d, m0)
            assert np.array_equal(tr["accepted"], rtr["accepted"])
            assert np.abs(phi - rphi).max() < 1e-12
            assert abs(res.mu - np.sqrt(rm2)) < 1e-12


def test_fp32_results_with_large_requests_equal_standalone_runs():
    """Binary32 serving with requests large enough (N >= 384) for the loop's
    draw-once scratch: every result equals the standalone run."""
    K = 32
    reqs = [(1024, 16, 31, 12), (40, 6, 32, 30), (600, 40, 33, 10), (3000, 4, 34, 6)]
    with T.Server(hbm_budget=512 << 20, max_slots=4, iters_per_round=4, K=K,
                  precision="fp32") as srv:
        tickets = [srv.submit(N, d, seed, budget, want_phi=True) for N, d, seed, budget in reqs]
        results = [srv.wait(t, with_phi=True) for t in tickets]
        stats = srv.stats()
    # three kernels per admission, at least three per iteration of the longest request
    assert stats.kernel_launches >= 3 * len(reqs) + 3 * max(r[3] for r in reqs)
    for (N, d, seed, budget), (st, res, phi) in zip(reqs, results):
        assert st == T.TRSTMI_OK and res.iters == budget
        with T.Search(N, d, seed, K=K, precision="fp32", trace_cap=0) as s:
            s.step(budget)
            assert res.mu == s.step(0).mu, (N, d)
            assert np.array_equal(phi, s.get_phi()), (N, d)


def test_admission_respects_memory_budget():
    # each (N=1024, d=32) slot needs ~0.8 MiB; a 2 MiB budget holds two at a time
    with T.Server(hbm_budget=2 << 20, max_slots=8, iters_per_round=2, K=8,
                  precision="fp32") as srv:
        tickets = [srv.submit(1024, 32, 100 + i, 6) for i in range(5)]
        peak = 0
        while True:
            s = srv.stats()
            peak = max(peak, s.active_slots)
            assert s.hbm_in_use <= 2 << 20
            if s.completed == 5:
                break
            time.sleep(0.002)
        assert peak <= 2
        for t in tickets:
            st, res, _ = srv.poll(t)
            assert st == T.TRSTMI_OK and res.iters == 6
        # a request larger than the whole budget can never be admitted
        t = srv.submit(8192, 256, 1, 5)
        st, res, _ = srv.wait(t)
        assert st == T.TRSTMI_ENOMEM


def test_resident_work_cap_limits_admission():
    """max_resident_pairs: with room for two (N=512, K=8) searches at a time,
    at most two are resident; a request larger than the cap is still served
    once the server is empty."""
    K, N = 8, 512
    cap = 2 * K * N * (N - 1) // 2
    with T.Server(hbm_budget=256 << 20, max_slots=16, iters_per_round=2, K=K, precision="fp32",
                  max_resident_pairs=cap) as srv:
        tickets = [srv.submit(N, 16, 300 + i, 8) for i in range(5)]
        big = srv.submit(1024, 16, 400, 4)
        peak = 0
        while True:
            st = srv.stats()
            peak = max(peak, st.active_slots)
            if st.completed == 6:
                break
            time.sleep(0.001)
        assert 1 <= peak <= 2
        for t in tickets:
            assert srv.poll(t)[0] == T.TRSTMI_OK
        st, res, _ = srv.poll(big)
        assert st == T.TRSTMI_OK and res.iters == 4


def test_cancel_and_unknown_ticket():
    with T.Server(hbm_budget=64 << 20, max_slots=1, iters_per_round=5, K=8,
                  precision="fp32") as srv:
        long = srv.submit(512, 16, 1, 1_000_000)
        queued = srv.submit(16, 4, 2, 10)
        time.sleep(0.05)
        assert srv.cancel(queued) in (T.TRSTMI_PENDING, T.TRSTMI_ECANCELLED)
        assert srv.cancel(long) == T.TRSTMI_PENDING
        st, res, _ = srv.wait(long)
        assert st == T.TRSTMI_ECANCELLED and res.iters > 0
        st, _, _ = srv.wait(queued)
        assert st == T.TRSTMI_ECANCELLED
        st, _, _ = srv.poll(987654321)
        assert st == T.TRSTMI_ENOTFOUND


def test_deadlines_end_running_and_queued_requests():
    """A request past its deadline ends with TRSTMI_ETIMEOUT: while running at
    the next round boundary (with the iterations and mu it reached), while
    queued without starting; a request without a deadline is unaffected."""
    with T.Server(hbm_budget=64 << 20, max_slots=1, iters_per_round=5, K=8,
                  precision="fp32") as srv:
        long = srv.submit(512, 16, 1, 1_000_000, deadline_ms=300.0)
        queued = srv.submit(16, 4, 2, 10, deadline_ms=100.0)
        after = srv.submit(12, 3, 3, 20)
        st, res, _ = srv.wait(long)
        assert st == T.TRSTMI_ETIMEOUT
        assert 0 < res.iters < 1_000_000 and res.mu >= res.welch
        assert (res.t_done_ns - res.t_submit_ns) >= 300e6
        st, res, _ = srv.wait(queued)
        assert st == T.TRSTMI_ETIMEOUT and res.iters == 0
        st, res, _ = srv.wait(after)
        assert st == T.TRSTMI_OK and res.iters == 20
        s = srv.stats()
        assert s.timed_out == 2 and s.completed >= 1
        with pytest.raises(T.TrstmiError) as e:
            srv.submit(8, 2, 0, 10, deadline_ms=-1.0)
        assert e.value.status == T.TRSTMI_EINVAL


def test_bad_requests_rejected_on_host():
    with T.Server(hbm_budget=16 << 20, max_slots=2, K=8, precision="fp32") as srv:
        for bad in ((1, 3), (8, 0), (8, 300)):
            with pytest.raises(T.TrstmiError) as e:
                srv.submit(bad[0], bad[1], 0, 10)
            assert e.value.status == T.TRSTMI_EINVAL
    with pytest.raises(T.TrstmiError) as e:
        T.Server(precision="bf16", K=4, topk=8)
    assert e.value.status == T.TRSTMI_EINVAL


def test_serving_request_mix_runs():
    """A slice of the serving workload's request recipe (d ~ U[4,64], N
    log-uniform on [d+1, 4096], target 1.05 x Welch) through the loop."""
    reqs = W.serving_requests(40, seed=11)
    with T.Server(hbm_budget=1 << 30, max_slots=16, iters_per_round=10, K=8,
                  precision="fp32") as srv:
        tickets = [srv.submit(r["N"], r["d"], r["seed"], 30, target_rel_welch=1.05) for r in reqs]
        out = [srv.wait(t) for t in tickets]
    for r, (st, res, _) in zip(reqs, out):
        assert st == T.TRSTMI_OK
        assert 1 <= res.iters <= 30
        assert res.mu >= res.welch - 1e-6
