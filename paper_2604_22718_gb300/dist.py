"""Multi-process layout of the sampler: chains are independent, so N ranks
(one per GPU) each run a contiguous block of the global chain index range --
the Metropolis stream of a chain depends only on its global index (chain0 +
local index), so a sharded run reproduces the unsharded one chain by chain.
The only exchange is the final FP64 merge of trace moments."""
from __future__ import annotations

import numpy as np


def shard(total_chains: int, rank: int, world: int) -> tuple[int, int]:
    """(chain0, count) of this rank's contiguous block; blocks differ by at most one."""
    if world < 1 or not (0 <= rank < world) or total_chains < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(total_chains, world)
    count = base + (1 if rank < extra else 0)
    chain0 = rank * base + min(rank, extra)
    return chain0, count


def local_moments(trace: np.ndarray, center: float = 0.0) -> np.ndarray:
    """[n, sum (x - center), sum (x - center)^2] of a local trace (FP64)."""
    d = np.asarray(trace, dtype=np.float64) - center
    return np.array([float(d.size), float(d.sum()), float((d * d).sum())])


def merge_moments(trace: np.ndarray, group=None) -> dict:
    """Global mean and variance (1/n) of all ranks' traces, in two passes of
    FP64 sums across the process group (torch.distributed, any backend): the
    first gives n and the mean, the second the squared deviations from that
    mean, so the variance never comes from the difference of two large sums
    (sum x^2 / n - mean^2 loses every digit the mean has in common with the
    spread).  The residual sum of deviations corrects the mean's rounding."""
    import torch
    import torch.distributed as dist
    live = dist.is_available() and dist.is_initialized()

    def allsum(v):
        t = torch.from_numpy(v)
        if live:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.numpy()

    n, s1, _ = allsum(local_moments(trace))
    mean = s1 / n
    _, d1, d2 = allsum(local_moments(trace, mean))
    return {"n": float(n), "mean": float(mean + d1 / n), "var": float((d2 - d1 * d1 / n) / n)}
