"""Atom-sharded correlation through the library on one GPU: two gloo ranks
(processes) share cuda:0, each runs tcorr_msd / tcorr_acf (and the weighted
calls) on its own atom slice, the ranks gather their records and combine them
with tcorr_combine_shards; the result is checked against the oracle on all
atoms.  The ranks' kernels are independent (no rank waits on another on the
GPU); the exchange goes through gloo on the host."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1708_08619_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TN, NA, TM, S = 900, 301, 400, 2


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _inputs():
    x = synth.random_walk_positions(TN, NA, 0.02, 3.0, seed=311)
    v = synth.ou_velocities(TN, NA, 0.1, 1.0, seed=312)
    w = np.random.default_rng(313).uniform(0.5, 16.0, size=NA).astype(np.float32)
    return x, v, w


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_1708_08619_gb300 import build, shard, tcorr
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    build.build()
    tcorr.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, v, w = _inputs()
    a0, a1 = shard.atom_range(NA, rank, world)
    xs = torch.from_numpy(np.ascontiguousarray(x[:, a0:a1])).cuda()
    vs = torch.from_numpy(np.ascontiguousarray(v[:, a0:a1])).cuda()
    ws = torch.from_numpy(np.ascontiguousarray(w[a0:a1])).cuda()
    out = {}
    for method in ("plain", "fp16x3"):
        m = tcorr.tcorr_msd(xs, TM, S, method)
        c = tcorr.tcorr_acf(vs, TM, S, method)
        out[("msd", method)] = shard.combine_atom_shards(m, n_atoms=a1 - a0).cpu().numpy()
        out[("acf", method)] = shard.combine_atom_shards(c, n_atoms=a1 - a0).cpu().numpy()
    W = tcorr.tcorr_weight_total(ws)
    mw = tcorr.tcorr_msd_weighted(xs, ws, TM, S, "fp16x3")
    out[("msd_w", "fp16x3")] = shard.combine_atom_shards(mw, weight=W).cpu().numpy()
    torch.cuda.synchronize()
    status = tcorr.tcorr_status_poll()
    dist.destroy_process_group()
    q.put((rank, out, status))


def test_two_ranks_share_cuda0_and_combine_atom_shards():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted([q.get(timeout=600) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    x, v, w = _inputs()
    rm = oracle.msd(x, TM, S)
    rc = oracle.acf(v, TM, S)
    rmw = oracle.msd_weighted(x, w, TM, S)
    for rank, out, status in results:
        assert status == 0
        parity.check_plain_msd(out[("msd", "plain")], rm, what=f"rank {rank} plain msd")
        parity.check_acf(out[("acf", "plain")], rc, parity.PLAIN_TOL, what=f"rank {rank} plain acf")
        parity.check_tc_msd(out[("msd", "fp16x3")], rm, what=f"rank {rank} fp16x3 msd")
        parity.check_acf(out[("acf", "fp16x3")], rc, parity.TC_TOL, what=f"rank {rank} fp16x3 acf")
        parity.check_tc_msd(out[("msd_w", "fp16x3")], rmw, what=f"rank {rank} weighted msd")
    # the combine sums the gathered rows in a fixed order: both ranks hold the same bits
    for key in results[0][1]:
        assert np.array_equal(results[0][1][key], results[1][1][key]), key


def test_combine_shards_matches_the_weighted_mean():
    """tcorr_combine_shards on one process: three made-up records (values and
    weights) against the weighted mean formed here in FP64."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_08619_gb300 import build, tcorr
    build.build()
    tcorr.load()
    rng = np.random.default_rng(314)
    n = 1001
    rows = np.zeros((3, n + 7))            # padded rows (ld = n + 7)
    rows[:, :n] = rng.normal(size=(3, n))
    rows[:, n] = [17.0, 3.0, 250.0]
    d = torch.from_numpy(rows).cuda()
    got = tcorr.tcorr_combine_shards(d, n).cpu().numpy()
    w = rows[:, n]
    want = (w[0] * rows[0, :n] + w[1] * rows[1, :n] + w[2] * rows[2, :n]) / (w[0] + w[1] + w[2])
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=1e-15)
    wt = torch.from_numpy(rng.uniform(0, 2, size=5000).astype(np.float32)).cuda()
    W = tcorr.tcorr_weight_total(wt).cpu().numpy()[0]
    assert abs(W / wt.double().sum().item() - 1) < 1e-14
