"""Sharding the ensemble over several GPUs (host logic).

Trajectories are independent and trajectory e belongs to sub-ensemble
e mod N_R whichever process draws it, so the ensemble shards by disjoint
trajectory ranges with no exchange while sampling.  The one exchange is a sum
of every rank's sub-ensemble sums and counts (gbs_get_accumulators) before
the inversion (Eq. total_counts with the sub-ensemble errors of Appendix A),
after which any rank inverts the combined sums (gbs_set_accumulators,
gbs_binned_counts).  torch.distributed's gloo backend carries the sum in
host memory: it is a few tens of MB once per run, so no device collective
is needed.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def rank_range(rank: int, world: int, per_rank: int, first: int = 0) -> Tuple[int, int]:
    """(first trajectory, count) of rank `rank` of `world` when every rank
    draws `per_rank` consecutive trajectories after `first`."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("rank must be in [0, world) and per_rank >= 0")
    return first + rank * per_rank, per_rank


def combine_accumulators(acc: np.ndarray, counts: np.ndarray,
                         group=None) -> Tuple[np.ndarray, np.ndarray]:
    """All-reduce (sum) of the sub-ensemble sums acc[2][N_R][K1] (complex128)
    and counts[N_R] (int64) over a gloo process group (host tensors); returns
    the sums, equal on every rank."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(acc, dtype=np.complex128)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    ta = torch.from_numpy(a.view(np.float64).copy())
    tc = torch.from_numpy(c.copy())
    dist.all_reduce(ta, group=group)
    dist.all_reduce(tc, group=group)
    out = ta.cpu().numpy().view(np.complex128).reshape(a.shape)
    return out, tc.cpu().numpy()
