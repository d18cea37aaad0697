"""Replica bookkeeping for runs on several GPUs of one node.

Grid cells are independent, so N GPUs run N replicas of the solve, each on
its own cells, with no exchange on the data path.  This module holds the only
cross-rank steps: which cells a rank owns and the whole-job throughput
(cells of all ranks over the slowest rank's time)."""
from __future__ import annotations


def cell_seed(base_seed: int, rank: int) -> int:
    """Seed of the cells rank `rank` owns (rank 0 keeps the base seed)."""
    return base_seed + 1000 * rank


def aggregate(local_cells: float, local_seconds: float, dist=None):
    """(total cells, max seconds, whole-job cells/s) over all ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_cells, local_seconds, local_cells / local_seconds
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    c = torch.tensor([float(local_cells)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return c.item(), t.item(), c.item() / t.item()
