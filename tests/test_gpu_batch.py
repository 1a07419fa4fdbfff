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
        assert all(w in (16, 32, 64) for w in widths)
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
        T.Batch([4], [2], [0], precision="bf16")
    assert e.value.status == T.TRSTMI_EUNSUPPORTED
