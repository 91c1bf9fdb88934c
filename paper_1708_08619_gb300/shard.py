"""Host-side sharding of correlation problems across ranks.

The correlation of one trajectory never needs data from another, so a batch
of instances (trajectories, atom subclasses, flux series) is split across
ranks with no exchange on the data path: each rank runs tcorr_batch on its
own share.  The only collective is the harness's max-over-ranks of the step
time.  Work per instance is the number of (atom, origin, lag) updates,
N * sum_tau n_o(tau); shares are balanced greedily (largest instance first,
to the least-loaded rank), which keeps the heaviest rank within one instance
of the average.

One large trajectory can instead be split by atoms (``atom_range``; the
paper's Conclusion suggests dividing a species' data over devices by atoms):
each rank correlates its atom slice with the library, writes one record (its
per-lag averages and its atom count or weight sum), the records are gathered
in rank order (``gather_shard_records``, the one exchange: an all-gather of
tau_max + 2 doubles per rank), and the library's tcorr_combine_shards forms
the average over all atoms with fixed-order FP64 sums, so every rank holds the
same bits.  This module does no arithmetic of the method itself.
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


def shard_record(result, weight=None, n_atoms: int | None = None):
    """One rank's record: its per-lag averages followed by its weight, as a new
    float64 tensor of n + 1 values on the result's device.  The weight is the
    slice's atom count (n_atoms) or a one-element float64 tensor holding its
    weight sum (from tcorr_weight_total); it is copied, not computed here."""
    import torch
    n = result.numel()
    rec = torch.empty(n + 1, dtype=torch.float64, device=result.device)
    rec[:n].copy_(result.reshape(-1))
    if weight is not None:
        rec[n:].copy_(weight.reshape(-1)[:1])
    else:
        rec[n] = float(n_atoms)
    return rec


def gather_shard_records(rec, group=None):
    """All ranks' records as rows of a [world][n + 1] float64 tensor in rank
    order, on rec's device (all-gather; with gloo the exchange goes through host
    memory).  Without a process group: the one record as a [1][n + 1] tensor."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return rec.reshape(1, -1)
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    comm_dev = rec.device if backend == "nccl" else torch.device("cpu")
    mine = rec.to(comm_dev)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return torch.stack(parts).to(rec.device)


def combine_atom_shards(result, weight=None, n_atoms: int | None = None, group=None, stream=None):
    """Whole-trajectory average from per-rank results over disjoint atom slices
    (CUDA tensors): gather the ranks' records and combine them with
    tcorr_combine_shards.  Pass n_atoms (the slice's atom count) for plain
    averages, or weight (a one-element float64 CUDA tensor with the slice's
    weight sum, from tcorr_weight_total) for weighted ones.  Identity without a
    process group."""
    import torch.distributed as dist
    from . import tcorr
    if not (dist.is_available() and dist.is_initialized()):
        return result
    rows = gather_shard_records(shard_record(result, weight, n_atoms), group)
    return tcorr.tcorr_combine_shards(rows, result.numel(), stream=stream)


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
