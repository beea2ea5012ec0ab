"""Sharding of histories over ranks (one process per GPU).

Histories are independent and each one draws from its own counter-based Philox
stream keyed by its history id, so any partition of the id range reproduces the
single-process result exactly: integer tallies and spectra add, the FEPE and
its sigma follow from the summed counts.  Rank r of W transports ids
[offset + r * n, offset + (r + 1) * n) -- weak scaling, no exchange while
transporting; the tallies are summed once at the end.
"""
from __future__ import annotations

import math

import numpy as np

COUNT_KEYS = ("n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_segments", "n_interactions")


def history_offset(rank: int, n_per_rank: int, base: int = 0) -> int:
    """First history id of `rank` when every rank runs n_per_rank histories."""
    if rank < 0 or n_per_rank < 0:
        raise ValueError("rank and n_per_rank must be non-negative")
    return base + rank * n_per_rank


def split_range(n_total: int, world: int, rank: int):
    """Contiguous share of n_total histories for `rank` (strong scaling): (offset, count)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    q, r = divmod(n_total, world)
    start = rank * q + min(rank, r)
    return start, q + (1 if rank < r else 0)


def reduce_tallies(counts: dict, spectrum: np.ndarray, group=None):
    """Sum integer tallies and the spectrum over all ranks (torch.distributed,
    any backend); returns (counts, spectrum, fepe, sigma) identical on every rank."""
    import torch
    import torch.distributed as dist
    keys = [k for k in COUNT_KEYS if k in counts]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    c = torch.tensor([int(counts[k]) for k in keys], dtype=torch.int64, device=dev)
    s = torch.as_tensor(np.asarray(spectrum, dtype=np.int64), device=dev)
    dist.all_reduce(c, group=group)
    dist.all_reduce(s, group=group)
    out = dict(zip(keys, (int(v) for v in c.cpu().tolist())))
    n = out.get("n_hist", 0)
    fepe = out["n_fep"] / n if n else 0.0
    sigma = math.sqrt(fepe * (1 - fepe) / n) if n else 0.0
    return out, s.cpu().numpy(), fepe, sigma
