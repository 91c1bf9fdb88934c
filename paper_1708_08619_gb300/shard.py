"""Host-side sharding of independent correlation problems across ranks.

The correlation of one trajectory never needs data from another, so a batch
of instances (trajectories, atom subclasses, flux series) is split across
ranks with no exchange on the data path: each rank runs tcorr_batch on its
own share.  The only collective is the harness's max-over-ranks of the step
time.  Work per instance is the number of (atom, origin, lag) updates,
N * sum_tau n_o(tau); shares are balanced greedily (largest instance first,
to the least-loaded rank), which keeps the heaviest rank within one instance
of the average.
"""
from __future__ import annotations


def instance_work(T: int, N: int, tau_max: int, stride: int = 1) -> int:
    """Updates of one instance: N * sum_{tau=0..tau_max} (floor((T-1-tau)/s) + 1)."""
    total = 0
    for tau in range(tau_max + 1):
        total += (T - 1 - tau) // stride + 1
    return N * total


def partition(works, world: int):
    """Greedy largest-first assignment; returns one list of indices per rank."""
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    loads = [0] * world
    shares = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        shares[r].append(i)
        loads[r] += works[i]
    return [sorted(s) for s in shares]


def my_share(shapes, rank: int, world: int):
    """Indices of the instances that `rank` runs; shapes = [(T, N, tau_max, stride), ...]."""
    works = [instance_work(*s) for s in shapes]
    return partition(works, world)[rank]


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over all ranks (the harness's step time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
