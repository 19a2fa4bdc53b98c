"""Multi-GPU sharding (host side).

Monte-Carlo simulation: frames are independent and the channel is counter-based (Philox
counter = frame id), so rank r simulates its own disjoint range of frame ids and the only
exchange is a sum of the integer counters (and a max of the timed duration).  No
collective touches the data path.

Data-parallel training of the learned min-sum: each rank draws its own frames and runs the
forward and backward kernels on them; the loss is a mean over frames, so the gradient over
all ranks' frames is the frame-weighted mean of the ranks' gradients -- one all-reduce of
the [T][J*L][2] gradient (with the frame count appended) per step.
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


def average_gradient(grad, frames: int, dist=None):
    """Gradient over the frames of every rank, from this rank's gradient of a per-frame mean loss on
    `frames` frames: sum_r frames_r * grad_r / sum_r frames_r (one all-reduce of grad and the count).
    Returns a new tensor on grad's device; without a process group of more than one rank, grad itself."""
    import torch

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return grad
    flat = torch.cat([(grad.detach().to(torch.float64) * frames).reshape(-1),
                      torch.tensor([float(frames)], dtype=torch.float64, device=grad.device)])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    return (flat[:-1] / flat[-1]).reshape(grad.shape).to(grad.dtype)
