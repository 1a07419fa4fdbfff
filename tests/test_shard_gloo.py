"""Candidate sharding, host side: two gloo ranks on CPU.

Each rank steps the same search through ``paper_2207_06374_gb300.shard``
(candidate ranges, MAX all-reduce of the score vector, identical decision on
every rank).  The scorer behind it is a host stand-in built on the oracle
(fp64 scores of the rank's candidates; the decision replayed by the oracle's
accept/radius rule), so the test checks the sharding logic itself: every
rank's trajectory must equal the unsharded oracle search, choice for choice.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2207_06374_gb300.shard import ShardedSearch, candidate_range

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

N, D, SEED, K, T = 9, 3, 21, 48, 12


class OracleShardSearch:
    """Host stand-in of trstmi.Search's sharding calls (binary64 scores)."""

    def __init__(self, N, d, seed, K):
        self.seed, self.K = seed, K
        self.phi = O.init(N, d, seed)
        self.mu2 = O.mu2(self.phi)
        self.delta = 0.1
        self.t = 0
        self.trace = []

    def shard_score_bytes(self):
        return self.K * 8

    def _view(self, ptr):
        return np.ctypeslib.as_array((ctypes.c_int64 * self.K).from_address(ptr))

    def shard_score(self, c_lo, c_hi, ptr):
        v = self._view(ptr)
        v[:] = 0
        if c_hi > c_lo:
            sc = O.score(self.phi, self.seed, self.delta, self.t + 1, c_lo, c_hi - c_lo)
            v[c_lo:c_hi] = np.asarray(sc, dtype=np.float64).view(np.int64)

    def shard_finish(self, ptr):
        scores = self._view(ptr).copy().view(np.float64)
        cstar = int(np.argmin(scores))            # lowest index on ties
        self.phi, self.mu2, self.delta, tr = O.replay(
            self.phi, self.seed, O.make_opts(K=self.K, T=1), self.delta, self.mu2, self.t, [cstar])
        self.t += 1
        self.trace.append((int(tr["cstar"][0]), int(tr["accepted"][0]), float(tr["mu2_cur"][0])))
        return None


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = OracleShardSearch(N, D, SEED, K)
        ShardedSearch(s, K, torch, dist, device="cpu").step(T)
        np.save(os.path.join(out_dir, f"phi{rank}.npy"), s.phi)
        np.save(os.path.join(out_dir, f"trace{rank}.npy"), np.array(s.trace))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_candidate_ranges_partition_every_candidate_once():
    for K_ in (1, 7, 48, 1024):
        for world in (1, 2, 3, 8):
            got = [candidate_range(K_, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == K_
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        candidate_range(8, 2, 2)


def test_two_gloo_ranks_follow_the_unsharded_search(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    _, _, _, otr = O.run(N, D, SEED, O.make_opts(K=K, T=T))
    ref_phi = None
    for r in range(world):
        tr = np.load(tmp_path / f"trace{r}.npy")
        phi = np.load(tmp_path / f"phi{r}.npy")
        assert np.array_equal(tr[:, 0].astype(np.int64), otr["cstar"].astype(np.int64))
        assert np.array_equal(tr[:, 1].astype(np.int64), otr["accepted"].astype(np.int64))
        assert np.array_equal(tr[:, 2], otr["mu2_cur"])
        if ref_phi is None:
            ref_phi = phi
        assert np.array_equal(phi, ref_phi)       # identical frames on every rank
