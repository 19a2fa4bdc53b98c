"""Multi-GPU Monte-Carlo sharding (host side): frames are independent and the channel is
counter-based (Philox counter = frame id), so rank r simulates its own disjoint range of
frame ids and the only exchange is a sum of the integer counters (and a max of the timed
duration).  No collective touches the data path.
"""
from __future__ import annotations

COUNTERS = ("frames", "frame_errors", "bit_errors", "iters_sum", "undetected")
RANK_STRIDE = 1 << 40  # frame ids per rank: rank r owns [r * 2^40 + 2^36, (r + 1) * 2^40)
RANK_OFFSET = 1 << 36


def first_frame(rank: int, step: int, frames_per_step: int) -> int:
    """First frame id of `step` (>= -2^36 / frames_per_step, warm-up steps negative) on `rank`."""
    f = rank * RANK_STRIDE + RANK_OFFSET + step * frames_per_step
    if not (rank * RANK_STRIDE <= f and f + frames_per_step <= (rank + 1) * RANK_STRIDE):
        raise ValueError("step outside the rank's frame-id range")
    return f


def merge_counts(results, dist=None, device=None) -> dict:
    """Sum the counters of this rank's results (dicts with COUNTERS keys) over all ranks."""
    import torch

    local = [sum(int(r[k]) for r in results) for k in COUNTERS]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor(local, dtype=torch.int64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        local = [int(x) for x in t.tolist()]
    return dict(zip(COUNTERS, local))


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value of x over all ranks (the job's duration is the slowest rank's)."""
    import torch

    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(x)
