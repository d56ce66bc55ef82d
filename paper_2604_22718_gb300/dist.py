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


def local_moments(trace: np.ndarray) -> np.ndarray:
    """[n, sum x, sum x^2] of a local trace (FP64)."""
    x = np.asarray(trace, dtype=np.float64)
    return np.array([float(x.size), float(x.sum()), float((x * x).sum())])


def merge_moments(trace: np.ndarray, group=None) -> dict:
    """Global mean and variance (1/n) of all ranks' traces by an FP64 sum of
    local moments across the process group (torch.distributed, any backend)."""
    m = local_moments(trace)
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(m)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    n, s1, s2 = (float(v) for v in t)
    mean = s1 / n
    return {"n": n, "mean": mean, "var": s2 / n - mean * mean}
