"""Host-side sharding of correlation problems across ranks.

The correlation of one trajectory never needs data from another, so a batch
of instances (trajectories, atom subclasses, flux series) is split across
ranks with no exchange on the data path: each rank runs tcorr_batch on its
own share.  The only collective is the harness's max-over-ranks of the step
time.  Work per instance is the number of (atom, origin, lag) updates,
N * sum_tau n_o(tau); shares are balanced greedily (largest instance first,
to the least-loaded rank), which keeps the heaviest rank within one instance
of the average.

One large trajectory can instead be split by atoms (``atom_range``): each rank
correlates its atom slice and ``combine_atom_shards`` weights the per-lag
averages by atom count in one all-reduce (the paper's Conclusion suggests
dividing a species' data over devices by atoms).
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


def atom_range(N: int, rank: int, world: int):
    """Contiguous atoms [a0, a1) of `rank` when one trajectory is split by atoms
    (sizes differ by at most one)."""
    base, extra = divmod(N, world)
    a0 = rank * base + min(rank, extra)
    return a0, a0 + base + (1 if rank < extra else 0)


def combine_atom_shards(result, n_local: float, group=None):
    """Whole-trajectory average from per-rank results over disjoint atom slices.

    Every per-lag MSD / autocorrelation value is an average over atoms and
    origins; the origin count n_o(tau) is the same on every rank (same T and
    stride), so the average over all atoms is sum_r N_r result_r / sum_r N_r:
    one FP64 all-reduce of tau_max + 2 values.  For weighted averages n_local
    is the rank's weight sum W_r instead of its atom count.  Works on any
    backend (NCCL with CUDA tensors, gloo with CPU tensors); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return result
    buf = torch.empty(result.numel() + 1, dtype=torch.float64, device=result.device)
    buf[:-1] = result.to(torch.float64) * float(n_local)
    buf[-1] = float(n_local)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[:-1] / buf[-1]


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
