"""Batched searches: many uneven instances in shared launches.

Each instance of a batch must follow exactly the trajectory it follows
alone (same seed and options): the scores of its candidates are the same
bits whatever tile width the autotuner picks, so the argmin sequence, the
decisions and the final frame are identical.  In binary64 the batch also
matches the CPU oracle choice for choice.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2207_06374_gb300.trstmi")
W = pytest.importorskip("paper_2207_06374_gb300.workloads")

MIX = [(4, 2), (7, 3), (9, 3), (2, 5), (13, 4), (33, 6), (70, 8), (129, 13), (200, 16),
       (256, 16), (17, 16), (100, 10)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_instances_match_single_runs_bitwise(precision):
    Ns = [n for n, _ in MIX]
    ds = [d for _, d in MIX]
    seeds = [1000 + i for i in range(len(MIX))]
    K, iters = 64, 25
    with T.Batch(Ns, ds, seeds, K=K, precision=precision, trace_cap=64) as b:
        info = b.step(iters)
        assert info.iters_done == iters
        widths = b.tile_widths()
        assert all(w in (0, 16, 32, 64) for w in widths)   # 0: whole candidate
        mus, its = b.mu()
        assert np.all(its == iters)
        for i, (N, d) in enumerate(MIX):
            with T.Search(N, d, seeds[i], K=K, precision=precision, trace_cap=64) as s:
                s.step(iters)
                tr_single = s.trace()
                phi_single = s.get_phi()
                mu_single = s.step(0).mu
            tr = b.trace(i)
            assert np.array_equal(tr["cstar"], tr_single["cstar"]), (i, N, d)
            assert np.array_equal(tr["accepted"], tr_single["accepted"]), (i, N, d)
            assert np.array_equal(b.get_phi(i), phi_single), (i, N, d)
            assert mus[i] == mu_single


# large instances (N >= 384, scored in tiles): their candidate passes draw each
# candidate once into a scratch and run the double-buffered tile pass, one
# instance at a time, between the shared launches of the others
LARGE_MIX = [(400, 12), (1024, 24), (30, 5), (700, 48), (2000, 8), (129, 13)]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_large_instances_match_single_runs_bitwise(precision):
    Ns = [n for n, _ in LARGE_MIX]
    ds = [d for _, d in LARGE_MIX]
    seeds = [500 + i for i in range(len(LARGE_MIX))]
    K, iters = 64, 10
    with T.Batch(Ns, ds, seeds, K=K, precision=precision, topk=4, trace_cap=32) as b:
        b.step(iters)
        mus, its = b.mu()
        assert np.all(its == iters)
        for i, (N, d) in enumerate(LARGE_MIX):
            with T.Search(N, d, seeds[i], K=K, precision=precision, topk=4, trace_cap=32) as s:
                s.step(iters)
                tr_single = s.trace()
                assert np.array_equal(b.get_phi(i), s.get_phi()), (i, N, d)
                mu_single = s.step(0).mu
            tr = b.trace(i)
            for f in ("cstar", "accepted", "flags", "mu2_best", "mu2_screen"):
                assert np.array_equal(tr[f], tr_single[f]), (f, i, N, d)
            assert mus[i] == mu_single


def test_batch_fp64_matches_oracle():
    Ns, ds = [4, 7, 12, 30], [2, 3, 5, 4]
    seeds = [5, 6, 7, 8]
    K, iters = 96, 40
    with T.Batch(Ns, ds, seeds, K=K, precision="fp64") as b:
        b.step(iters)
        for i in range(4):
            _, _, _, otr = O.run(Ns[i], ds[i], seeds[i], O.make_opts(K=K, T=iters), nthreads=4)
            tr = b.trace(i)
            assert np.array_equal(tr["cstar"], otr["cstar"])
            assert np.array_equal(tr["accepted"], otr["accepted"])
            assert np.allclose(tr["mu2_cur"], otr["mu2_cur"], rtol=1e-12, atol=0)


def test_batched_workload_sample_matches_single_runs():
    """The batched workload's instance recipe (d ~ U[2,16], N ~ U[d+1, d^2],
    seed base 7): a 48-instance prefix, K=128, 8 iterations; six instances
    spread over the mix are re-run alone."""
    Ns, ds, seeds = W.batched_instances(48, seed=7)
    K, iters = 128, 8
    with T.Batch(Ns, ds, seeds, K=K, precision="fp32", trace_cap=16) as b:
        b.step(iters)
        for i in (0, 9, 17, 28, 39, 47):
            with T.Search(Ns[i], ds[i], seeds[i], K=K, precision="fp32", trace_cap=16) as s:
                s.step(iters)
                assert np.array_equal(b.get_phi(i), s.get_phi())
                assert np.array_equal(b.trace(i)["cstar"], s.trace()["cstar"])


def test_batch_target_stops_each_instance():
    # optima: 1/sqrt(3) for N=4 and 1/2 for N=3 in C^2, both below the target
    with T.Batch([4, 4, 3], [2, 2, 2], [1, 2, 3], K=128, target_mu=0.6) as b:
        info = b.step(3000)
        mus, its = b.mu()
        assert info.done == 1
        assert np.all(mus <= 0.6) and np.all(its < 3000)


def test_batch_rejects_bad_arguments():
    with pytest.raises(T.TrstmiError):
        T.Batch([1], [2], [0])
    with pytest.raises(T.TrstmiError) as e:
        T.Batch([4], [2], [0], precision="bf16", K=4, topk=8)
    assert e.value.status == T.TRSTMI_EINVAL


# shapes of the screen modes: inside the tensor-core screen's range (d <= 32;
# 32 < d <= 64 with bf16 / fp16 operands; N beyond 1536 (768 with two operand
# atoms) swept in bands) and outside it (d > 32 with tf32), which rank in
# binary32
SCREEN_MIX = [(4, 2), (9, 3), (40, 8), (129, 13), (200, 16), (17, 16), (300, 32), (1024, 32),
              (50, 40), (1600, 4), (700, 64), (120, 33), (800, 40)]


def screened_shape(precision, N, d):
    return d <= (32 if precision == "tf32" else 64) and 2 <= N <= 65536


@pytest.mark.parametrize("precision", ["bf16", "fp16", "tf32"])
def test_batch_screen_modes_match_single_runs_bitwise(precision):
    """Precision form in the batch: the shared screen launch over all
    (instance, candidate) items, shared top-k re-score and certification.
    With the default radius gate both regimes occur (screen while delta >=
    0.01, binary32 ranking below), and every instance's decisions, certified
    scores and final frame equal its standalone run."""
    Ns = [n for n, _ in SCREEN_MIX]
    ds = [d for _, d in SCREEN_MIX]
    seeds = [300 + i for i in range(len(SCREEN_MIX))]
    K, iters = 48, 14
    with T.Batch(Ns, ds, seeds, K=K, precision=precision, topk=6, trace_cap=64) as b:
        info = b.step(iters)
        assert info.iters_done == iters
        mus, its = b.mu()
        assert np.all(its == iters)
        screened = 0
        for i, (N, d) in enumerate(SCREEN_MIX):
            with T.Search(N, d, seeds[i], K=K, precision=precision, topk=6, trace_cap=64) as s:
                s.step(iters)
                tr_single = s.trace()
                phi_single = s.get_phi()
                mu_single = s.step(0).mu
            tr = b.trace(i)
            for f in ("cstar", "accepted", "flags", "mu2_best", "mu2_screen", "delta_used"):
                assert np.array_equal(tr[f], tr_single[f]), (f, i, N, d)
            assert np.array_equal(b.get_phi(i), phi_single), (i, N, d)
            assert mus[i] == mu_single
            if not screened_shape(precision, N, d):
                assert np.all(tr["flags"] & 1 == 0)
            screened += int(np.sum(tr["flags"] & 1))
        assert screened > 0


def test_batch_bf16_decisions_replay_in_fp64():
    """Independent check of the batched precision form: the oracle replays the
    chosen candidates of each instance in binary64 and reproduces every
    certified score, decision and the final frame."""
    Ns, ds, seeds = [6, 30, 300], [3, 5, 24], [41, 42, 43]
    K, iters = 64, 12
    with T.Batch(Ns, ds, seeds, K=K, precision="bf16", screen_min_delta=0.0, trace_cap=32) as b:
        phi0 = [b.get_phi(i) for i in range(3)]
        b.step(iters)
        for i in range(3):
            tr = b.trace(i)
            assert np.all(tr["flags"] & 1 == 1)
            rphi, rm2, _, rtr = O.replay(phi0[i], seeds[i], O.make_opts(K=K, T=iters), 0.1,
                                         O.mu2(phi0[i]), 0, tr["cstar"])
            cert = (tr["flags"] & 2) == 0
            assert np.allclose(tr["mu2_best"][cert], rtr["mu2_best"][cert], rtol=1e-12, atol=0)
            assert np.all(np.abs(tr["mu2_best"][~cert] - rtr["mu2_best"][~cert])
                          <= 2.0 * (2 * ds[i] + 18) * 2.0 ** -24)
            assert np.array_equal(tr["accepted"], rtr["accepted"])
            assert np.abs(b.get_phi(i) - rphi).max() < 1e-12


def test_batched_workload_full_size_sampled_against_oracle():
    """The bench's batched workload at full size (512 instances, d ~ U{2..16},
    N ~ U{d+1..d^2}, K = 512, fp32, autotuned widths): one iteration, then for
    a sample of instances the oracle scores all 512 candidates in binary64 and
    the batch's choice must be a valid argmin (its binary32 score within 1e-6
    of its binary64 mu, and no candidate better by more than 2e-6 in mu)."""
    Ns, ds, seeds = W.batched_instances(512, seed=7)
    K = 512
    with T.Batch(Ns, ds, seeds, K=K, precision="fp32", trace_cap=4) as b:
        phi0 = {i: b.get_phi(i) for i in range(0, 512, 37)}
        b.step(1)
        for i, phi in phi0.items():
            ref = np.sqrt(O.score(phi, seeds[i], 0.1, 1, 0, K, nthreads=8))
            row = b.trace(i)[0]
            c = int(row["cstar"])
            assert abs(np.sqrt(row["mu2_best"]) - ref[c]) < 1e-6, (i, Ns[i], ds[i])
            assert ref[c] <= ref.min() + 2e-6, (i, Ns[i], ds[i])
