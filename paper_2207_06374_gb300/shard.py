"""Candidate sharding of one search over several processes (one GPU each).

The K candidates of an iteration are independent, and each is a pure function
of (seed, t, c, Phi) (arXiv 2207.06374, Sec. "Optimization procedure": the
Monte-Carlo sampling of the trust region), so rank r of G scores a contiguous
range of them and the ranks exchange only the K-entry score vector by an
element-wise MAX all-reduce (every entry is written by exactly one rank; the
others leave it at zero, and the entries are bit patterns of non-negative
floats, so the integer MAX of them is exact).  Every rank then takes the same
decision from the same vector and keeps an identical frame: the result is
bit-identical to the unsharded search.

The exchange goes through ``torch.distributed`` (NCCL between GPUs, gloo on
CPU); this module holds only the host logic, the device work is the library's
(``trstmi_shard_score`` / ``trstmi_shard_finish``).
"""
from __future__ import annotations


def candidate_range(K: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [c_lo, c_hi) of candidates 0..K-1 for rank of world:
    the first K % world ranks take one candidate more."""
    if world < 1 or not 0 <= rank < world or K < 0:
        raise ValueError("bad rank / world / K")
    base, extra = divmod(K, world)
    c_lo = rank * base + min(rank, extra)
    return c_lo, c_lo + base + (1 if rank < extra else 0)


def score_dtype(torch, score_bytes: int, K: int):
    """Integer dtype holding one score bit pattern (int32 or int64)."""
    per = score_bytes // K
    if per == 4:
        return torch.int32
    if per == 8:
        return torch.int64
    raise ValueError(f"unexpected score size {per}")


class ShardedSearch:
    """Steps one search whose candidates are split over the ranks of ``group``.

    ``search`` offers ``shard_score_bytes()``, ``shard_score(c_lo, c_hi, ptr)``
    and ``shard_finish(ptr)`` (``trstmi.Search`` does); every rank must have
    created it with the same N, d, seed and options.  ``device`` is where the
    score vector lives (the search's GPU, or "cpu" for a host-side stand-in).
    """

    def __init__(self, search, K: int, torch, dist, group=None, device="cuda"):
        self.search, self.K, self.torch, self.dist, self.group = search, K, torch, dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.c_lo, self.c_hi = candidate_range(K, self.rank, self.world)
        nbytes = search.shard_score_bytes()
        self.scores = torch.zeros(K, dtype=score_dtype(torch, nbytes, K), device=device)

    def step(self, iters: int = 1):
        """Runs iters iterations; returns the last iteration's step info."""
        info = None
        on_gpu = self.scores.is_cuda
        for _ in range(iters):
            self.search.shard_score(self.c_lo, self.c_hi, self.scores.data_ptr())
            self.dist.all_reduce(self.scores, op=self.dist.ReduceOp.MAX, group=self.group)
            if on_gpu:
                # the library reads the vector on its own stream
                self.torch.cuda.current_stream().synchronize()
            info = self.search.shard_finish(self.scores.data_ptr())
        return info
