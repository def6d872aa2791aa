"""Replica combination across ranks.

Restarts are independent, so several GPUs each solve their own restart set of
the same instance and exchange nothing while stepping.  The only collective is
the final choice of the best answer: the lowest energy over ranks, ties to the
lowest rank, then the lowest restart index (the single-GPU tie rule).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def combine_best(E: float, r: int, group=None) -> tuple[float, int, int]:
    """All-gather each rank's (E, r) and return (E, rank, r) of the best one.

    Works with any backend (gloo on CPU, nccl on GPU); the tensors live on
    the backend's device."""
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    mine = torch.tensor([float(E), float(r)], dtype=torch.float64, device=dev)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    best = None
    for rank, t in enumerate(parts):
        cand = (float(t[0]), rank, int(t[1]))
        if best is None or cand[0] < best[0]:
            best = cand
    return best
