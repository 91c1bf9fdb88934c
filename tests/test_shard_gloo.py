"""Multi-rank host logic on CPU with two gloo ranks: instance sharding and the
max-over-ranks timing used by the benchmark harness."""
import os
import socket

import numpy as np
import pytest

from paper_1708_08619_gb300 import shard

torch = pytest.importorskip("torch")


def test_instance_work_matches_definition():
    T, N, tm, s = 37, 5, 20, 3
    want = N * sum(len(range(0, T - tau, s)) for tau in range(tm + 1))
    assert shard.instance_work(T, N, tm, s) == want


def test_partition_is_complete_disjoint_and_balanced():
    rng = np.random.default_rng(5)
    works = [int(w) for w in rng.integers(1, 10 ** 6, size=257)]
    for world in (1, 2, 3, 8):
        shares = shard.partition(works, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(works)))
        loads = [sum(works[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(works)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shapes, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.my_share(shapes, rank, world)
    t = shard.max_over_ranks(10.0 + rank)
    # gather every rank's share on every rank to check coverage
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    dist.destroy_process_group()
    q.put((rank, mine, t, gathered))


def test_two_gloo_ranks_share_a_batch_and_agree_on_the_step_time():
    import torch.multiprocessing as mp
    rng = np.random.default_rng(7)
    shapes = [(int(rng.integers(100, 2000)), int(rng.integers(1, 500)), 0, 1) for _ in range(40)]
    shapes = [(T, N, T // 4, 1) for T, N, _, _ in shapes]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, shapes, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    for rank, mine, t, gathered in results:
        assert t == 11.0                      # max over ranks of 10 + rank
        flat = sorted(i for s in gathered for i in s)
        assert flat == list(range(len(shapes)))
        assert gathered[rank] == mine


def test_atom_ranges_cover_the_atoms_once():
    for N in (1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            rs = [shard.atom_range(N, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == N
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


def _atom_worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_1708_08619_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = synth.random_walk_positions(120, 37, 0.02, 2.0, seed=91)
    a0, a1 = shard.atom_range(37, rank, world)
    # each rank's share: the oracle stands in for the device library on CPU; the
    # records are gathered through gloo (the combine itself runs in the library)
    part = torch.from_numpy(oracle.msd(np.ascontiguousarray(x[:, a0:a1]), 60, 2))
    rows = shard.gather_shard_records(shard.shard_record(part, n_atoms=a1 - a0))
    dist.destroy_process_group()
    q.put((rank, rows.numpy()))


def _run_two(target):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(results, key=lambda r: r[0])


def test_two_gloo_ranks_gather_atom_shard_records():
    """Both ranks receive both records, in rank order, each holding that rank's
    per-lag averages and its atom count; their count-weighted mean is the
    oracle's average over all atoms."""
    import oracle
    from paper_1708_08619_gb300 import synth
    results = _run_two(_atom_worker)
    x = synth.random_walk_positions(120, 37, 0.02, 2.0, seed=91)
    want = oracle.msd(x, 60, 2)
    for _, rows in results:
        assert rows.shape == (2, 62)
        for r in range(2):
            a0, a1 = shard.atom_range(37, r, 2)
            assert rows[r, 61] == a1 - a0
            assert np.array_equal(rows[r, :61], oracle.msd(np.ascontiguousarray(x[:, a0:a1]), 60, 2))
        w = rows[:, 61]
        np.testing.assert_allclose((w[:, None] * rows[:, :61]).sum(axis=0) / w.sum(), want, rtol=1e-12, atol=0)
    assert np.array_equal(results[0][1], results[1][1])


def _weighted_atom_worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_1708_08619_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = synth.ou_velocities(150, 41, 0.1, 1.0, seed=93)
    w = np.random.default_rng(94).uniform(0.5, 16.0, size=41).astype(np.float32)
    a0, a1 = shard.atom_range(41, rank, world)
    # a weighted share carries its weight sum in place of its atom count
    part = torch.from_numpy(oracle.acf_weighted(np.ascontiguousarray(v[:, a0:a1]), w[a0:a1], 70, 1))
    wsum = torch.tensor([float(w[a0:a1].astype(np.float64).sum())], dtype=torch.float64)
    rows = shard.gather_shard_records(shard.shard_record(part, weight=wsum))
    dist.destroy_process_group()
    q.put((rank, rows.numpy()))


def test_two_gloo_ranks_gather_weighted_atom_shard_records():
    import oracle
    from paper_1708_08619_gb300 import synth
    results = _run_two(_weighted_atom_worker)
    v = synth.ou_velocities(150, 41, 0.1, 1.0, seed=93)
    w = np.random.default_rng(94).uniform(0.5, 16.0, size=41).astype(np.float32)
    want = oracle.acf_weighted(v, w, 70, 1)
    for _, rows in results:
        wr = rows[:, 71]
        np.testing.assert_allclose((wr[:, None] * rows[:, :71]).sum(axis=0) / wr.sum(), want, rtol=1e-12,
                                   atol=1e-15)
