"""Multi-GPU sharding of the frequency grid (one process per GPU).

The periodogram's frequencies are independent (Eq. 1-2 are evaluated per
frequency), so N ranks split a grid into contiguous blocks with no exchange of
data: rank r evaluates its block and the results are concatenated in rank
order.  Two layouts:

* weak scaling  -- every rank takes N_f frequencies of one grid N times as
  long: rank r starts at f_0 + r N_f df (what the benchmark runs);
* strong scaling -- a fixed grid of N_f frequencies is cut into near-equal
  contiguous blocks.

Only host arithmetic lives here; the timing reduction across ranks (the
maximum of the per-rank times) uses torch.distributed.
"""
from __future__ import annotations


def weak_block(f0: float, df: float, nf: int, rank: int, world: int):
    """(f0_r, df, nf) of rank r when each rank adds nf frequencies."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return f0 + rank * nf * df, df, nf


def strong_block(f0: float, df: float, nf: int, rank: int, world: int):
    """(f0_r, df, nf_r, k_r) of rank r when world ranks share one grid of nf
    frequencies; k_r is the block's first index in the full grid."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(nf, world)
    k = rank * base + min(rank, extra)
    n = base + (1 if rank < extra else 0)
    return f0 + k * df, df, n, k


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest `value` over all ranks (the job's time is its slowest rank)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
