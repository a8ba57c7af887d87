"""Host-side placement of independent boxes on ranks (one GPU per rank).

The batched form's boxes are independent problems, so a multi-GPU run needs
no data-path collective: each rank advances its own boxes.  Boxes are placed
by longest-processing-time-first on their cell counts (each box to the
currently least-loaded rank), which keeps the ranks' work within one box of
each other.  Only the timing (max over ranks) and, optionally, the per-box
diagnostics are gathered.
"""
from __future__ import annotations


def lpt_assign(costs, world):
    """Return a list of box-index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value, group=None):
    """Maximum of a host float over all ranks of the default process group
    (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
