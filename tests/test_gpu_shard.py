"""Candidate sharding on the device: several shards of one search, emulated on
one GPU (each shard its own instance, the MAX all-reduce done by
torch.maximum over their score vectors), must reproduce the unsharded search
bit for bit in every precision mode; and the torch.distributed path of
``shard.ShardedSearch`` runs through NCCL with a single rank."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
T = pytest.importorskip("paper_2207_06374_gb300.trstmi")
from paper_2207_06374_gb300.shard import ShardedSearch, candidate_range, score_dtype  # noqa: E402


def _run_sharded(N, d, seed, K, iters, world, **opt):
    stream = torch.cuda.current_stream()
    shards = [T.Search(N, d, seed, K=K, trace_cap=64, stream=stream.cuda_stream, **opt)
              for _ in range(world)]
    nbytes = shards[0].shard_score_bytes()
    dt = score_dtype(torch, nbytes, K)
    bufs = [torch.zeros(K, dtype=dt, device="cuda") for _ in range(world)]
    for _ in range(iters):
        for r, (s, b) in enumerate(zip(shards, bufs)):
            lo, hi = candidate_range(K, r, world)
            s.shard_score(lo, hi, b.data_ptr())
        full = bufs[0].clone()
        for b in bufs[1:]:
            full = torch.maximum(full, b)
        for s in shards:
            s.shard_finish(full.data_ptr())
    out = [(s.trace(), s.get_phi(), s.step(0).mu) for s in shards]
    for s in shards:
        s.close()
    return out


@pytest.mark.parametrize("precision,N,d,K", [("fp64", 12, 3, 40), ("fp32", 70, 8, 50),
                                             ("bf16", 300, 24, 64), ("fp16", 40, 6, 33),
                                             ("tf32", 150, 10, 24)])
def test_sharded_search_equals_unsharded(precision, N, d, K):
    seed, iters = 17, 10
    with T.Search(N, d, seed, K=K, precision=precision, trace_cap=64) as s:
        s.step(iters)
        ref_tr, ref_phi, ref_mu = s.trace(), s.get_phi(), s.step(0).mu
    for world in (2, 3):
        for tr, phi, mu in _run_sharded(N, d, seed, K, iters, world, precision=precision):
            for f in ("cstar", "accepted", "mu2_best", "mu2_cur", "delta_used", "flags"):
                assert np.array_equal(tr[f], ref_tr[f]), (precision, world, f)
            assert np.array_equal(phi, ref_phi)
            assert mu == ref_mu


def test_shard_rejects_bad_ranges():
    with T.Search(8, 3, 1, K=16, precision="fp32") as s:
        buf = torch.zeros(16, dtype=torch.int32, device="cuda")
        for lo, hi in ((-1, 4), (5, 4), (0, 17)):
            with pytest.raises(T.TrstmiError) as e:
                s.shard_score(lo, hi, buf.data_ptr())
            assert e.value.status == T.TRSTMI_EINVAL


def test_sharded_search_through_nccl_single_rank():
    import torch.distributed as dist
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        N, d, seed, K, iters = 200, 16, 5, 96, 6
        with T.Search(N, d, seed, K=K, precision="bf16") as ref:
            ref.step(iters)
            ref_phi = ref.get_phi()
        with T.Search(N, d, seed, K=K, precision="bf16",
                      stream=torch.cuda.current_stream().cuda_stream) as s:
            sh = ShardedSearch(s, K, torch, dist, device="cuda")
            assert (sh.c_lo, sh.c_hi) == (0, K)
            info = sh.step(iters)
            assert info.iters_done == 1
            assert np.array_equal(s.get_phi(), ref_phi)
    finally:
        dist.destroy_process_group()
