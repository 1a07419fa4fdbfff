"""The seeded workload recipes (CPU only): shapes, ranges, distributions and
reproducibility of the batched instances and the serving request stream."""
import numpy as np

from paper_2207_06374_gb300 import workloads as W


def test_batched_instances_follow_the_recipe():
    Ns, ds, seeds = W.batched_instances(512, seed=7)
    assert len(Ns) == len(ds) == len(seeds) == 512
    ds_a, Ns_a = np.array(ds), np.array(Ns)
    assert ds_a.min() >= 2 and ds_a.max() <= 16
    assert np.all(Ns_a >= ds_a + 1) and np.all(Ns_a <= ds_a * ds_a)
    assert set(np.unique(ds_a)) == set(range(2, 17))       # every d occurs at n = 512
    assert len(set(seeds)) == 512
    assert W.batched_instances(512, seed=7) == (Ns, ds, seeds)
    assert W.batched_instances(512, seed=8) != (Ns, ds, seeds)


def test_serving_stream_follows_the_recipe():
    n, rate = 10000, 200.0
    reqs = W.serving_requests(n, seed=11, rate_hz=rate)
    t = np.array([r["t_arrive"] for r in reqs])
    d = np.array([r["d"] for r in reqs])
    N = np.array([r["N"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps: mean 1/rate, standard deviation equal to the mean
    assert abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    assert d.min() == 4 and d.max() == 64
    assert np.all(N >= d + 1) and np.all(N <= 4096)
    # log-uniform N on [d+1, 4096]: the position of log N in that range is uniform
    u = (np.log(N) - np.log(d + 1)) / (np.log(4096) - np.log(d + 1))
    assert abs(np.median(u) - 0.5) < 0.03 and abs(np.mean(u < 0.25) - 0.25) < 0.03
    assert len({r["seed"] for r in reqs}) == n
    assert W.serving_requests(n, seed=11, rate_hz=rate) == reqs


def test_share_of_the_serving_stream_within_the_screen_shapes():
    """The tensor-core screen takes every shape of the serving recipe: d <= 32
    (bf16, fp16, tf32) and d <= 64 (bf16, fp16) at any N up to 65536, larger
    candidates swept in bands; the stream's d never exceeds 64 and its N never
    4096."""
    reqs = W.serving_requests(10000, seed=11)
    assert all(4 <= r["d"] <= 64 and r["d"] + 1 <= r["N"] <= 4096 for r in reqs)
    # the share that needs the band sweep (N beyond 1536, or 768 at d > 32)
    banded = np.mean([(r["d"] <= 32 and r["N"] > 1536) or (r["d"] > 32 and r["N"] > 768)
                      for r in reqs])
    assert 0.26 < banded < 0.30
