"""Batched path (tcorr_batch): one set of batched launches for many uneven
instances, captured in a CUDA graph and replayed (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1708_08619_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    tcorr.load()
    return tcorr


def uneven_instances(rng, count, Nmax=2048, Tmax=3000):
    """Mixed MSD (random walk) / ACF (OU) instances of uneven N, T, tau_max = T/4."""
    items = []
    for i in range(count):
        N = int(round(np.exp(rng.uniform(np.log(8), np.log(Nmax)))))
        Tn = int(rng.integers(60, Tmax))
        tm = Tn // 4
        s = int(rng.choice([1, 1, 1, 2, 3]))
        kind = i % 2
        if kind == 0:
            x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=synth.BASE_SEED + i)
        else:
            x = synth.ou_velocities(Tn, N, float(rng.uniform(0.01, 0.5)), 1.0, seed=synth.BASE_SEED + i)
        items.append((kind, x, tm, s))
    return items


def run_batch(T, items, method, stream=None, ws=None):
    dev = [(k, torch.from_numpy(x).cuda(), tm, s,
            torch.full((tm + 1,), np.nan, dtype=torch.float64, device="cuda")) for k, x, tm, s in items]
    inst = T.make_instances(dev)
    T.tcorr_batch(inst, method, stream=stream, ws=ws)
    torch.cuda.synchronize()
    return dev, inst


@pytest.mark.parametrize("method", ["plain", "fp16x3", "bf16x4", "tf32x3"])
def test_batch_equals_single_calls(T, method):
    rng = np.random.default_rng(77)
    items = uneven_instances(rng, 9, Nmax=600, Tmax=1500)
    dev, _ = run_batch(T, items, method)
    for kind, x, tm, s, out in dev:
        f = T.tcorr_msd if kind == 0 else T.tcorr_acf
        single = f(x, tm, s, method).cpu().numpy()
        assert np.array_equal(out.cpu().numpy(), single), (method, kind, x.shape, tm, s)
    assert T.tcorr_status_poll() == 0


def test_graph_replay_sees_new_data(T):
    rng = np.random.default_rng(78)
    items = uneven_instances(rng, 6, Nmax=400, Tmax=1200)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        dev0 = [(k, torch.from_numpy(x).cuda(), tm, s, torch.empty(tm + 1, dtype=torch.float64, device="cuda"))
                for k, x, tm, s in items]
        need = T.tcorr_batch_workspace_size(T.make_instances(dev0), "fp16x3")
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        dev, inst = run_batch(T, items, "fp16x3", stream=st, ws=ws)
        first = [o.cpu().numpy().copy() for *_, o in dev]
        # overwrite every input in place (same pointers), replay the cached graph
        for kind, x, tm, s, out in dev:
            x.mul_(2.0)
        T.tcorr_batch(inst, "fp16x3", stream=st, ws=ws)
        st.synchronize()
    for (kind, x, tm, s, out), f0 in zip(dev, first):
        # doubling the input multiplies both MSD and ACF by exactly 4 up to rounding
        np.testing.assert_allclose(out.cpu().numpy(), 4.0 * f0, rtol=2e-6, atol=1e-12)


@pytest.mark.slow
def test_uneven_batch_vs_oracle(T):
    """Shape of the batching workload, scaled down: 24 instances, N log-uniform in
    [64, 4096], T uniform in [500, 5000], tau_max = T/4, half MSD / half VACF."""
    rng = np.random.default_rng(synth.BASE_SEED)
    items = []
    for i in range(24):
        N = int(round(np.exp(rng.uniform(np.log(64), np.log(4096)))))
        Tn = int(rng.integers(500, 5001))
        tm = Tn // 4
        if i % 2 == 0:
            x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=synth.BASE_SEED + i)
        else:
            x = synth.ou_velocities(Tn, N, float(rng.uniform(0.01, 0.5)), 1.0, seed=synth.BASE_SEED + i)
        items.append((i % 2, x, tm, 1))
    for method in ("fp16x3", "plain"):
        dev, _ = run_batch(T, items, method)
        for (kind, xh, tm, s), (_, _, _, _, out) in zip(items, dev):
            lags = np.unique(np.array([0, 1, 2, tm // 3, tm // 2, tm]))
            got = out.cpu().numpy()[lags]
            ref = (oracle.msd if kind == 0 else oracle.acf)(xh, stride=s, lags=lags)
            if method == "plain":
                if kind == 0:
                    assert got[0] == 0.0
                    assert np.max(np.abs(got[1:] - ref[1:]) / ref[1:]) <= parity.PLAIN_TOL
                else:
                    assert np.max(np.abs(got - ref)) / abs(ref[0]) <= parity.PLAIN_TOL
            else:
                scale = ref[-1] if kind == 0 else ref[0]
                assert np.max(np.abs(got - ref)) / abs(scale) <= parity.TC_TOL, (method, kind, xh.shape)


def test_batch_with_a_big_instance(T):
    """A batch where one instance has enough work items for a launch of its own
    (N=6000, T=8000, tau_max=2000) next to small ones: bit-identical to single calls."""
    rng = np.random.default_rng(79)
    items = uneven_instances(rng, 4, Nmax=300, Tmax=800)
    items.insert(1, (0, synth.random_walk_positions(8000, 6000, 0.005, 5.0, seed=80), 2000, 1))
    dev, _ = run_batch(T, items, "fp16x3")
    for kind, x, tm, s, out in dev:
        f = T.tcorr_msd if kind == 0 else T.tcorr_acf
        assert np.array_equal(out.cpu().numpy(), f(x, tm, s, "fp16x3").cpu().numpy()), x.shape


@pytest.fixture(scope="module")
def full_batch(T):
    """The batching workload at full size, drawn on the device, with the oracle's
    values at lags 0, 1, tau_max/3, four lags in tau_max-192 .. tau_max-1 and
    tau_max for every instance."""
    if torch.cuda.get_device_properties(0).total_memory < 150e9:
        pytest.skip("needs a large-memory GPU")
    shapes = synth.batch_workload_shapes(256)
    data = []
    for i, shp in enumerate(shapes):
        kind, Tn, N, tm, s, _ = shp
        x = synth.batch_instance_device(i, shp)
        tail = np.linspace(max(0, tm - 192), tm - 1, 4).astype(np.int64)
        lags = np.unique(np.concatenate([[0, 1, tm // 3, tm], tail]))
        xh = x.cpu().numpy()
        ref = (oracle.msd if kind == 0 else oracle.acf)(xh, stride=s, lags=lags)
        del xh
        data.append((kind, x, tm, s, lags, ref))
    yield data
    del data
    torch.cuda.empty_cache()


@pytest.mark.slow
@pytest.mark.parametrize("method", ["fp16x3", "plain"])
def test_full_batching_workload_vs_oracle(T, full_batch, method):
    """The batching workload at full size: 256 uneven instances (N log-uniform
    in [64, 16384], T uniform in [500, 20000], tau_max = T/4; even: MSD of a
    random walk, odd: VACF of OU velocities) in one tcorr_batch call, every
    instance against the oracle at its sampled lags."""
    items = [(kind, x, tm, s, torch.full((tm + 1,), np.nan, dtype=torch.float64, device="cuda"))
             for kind, x, tm, s, _, _ in full_batch]
    inst = T.make_instances(items)
    T.tcorr_batch(inst, method)
    torch.cuda.synchronize()
    assert T.tcorr_status_poll() == 0
    worst = 0.0
    for (kind, x, tm, s, out), (_, _, _, _, lags, ref) in zip(items, full_batch):
        got = out.cpu().numpy()[lags]
        what = f"{method} instance kind {kind} T={x.shape[0]} N={x.shape[1]}"
        if method == "plain":
            if kind == 0:
                err = parity.check_plain_msd(got, ref, what=what)
            else:
                err = parity.check_acf(got, ref, parity.PLAIN_TOL, what=what)
        else:
            if kind == 0:
                assert got[0] == 0.0, what
                err = parity.check_tc_msd(got, ref, what=what)
            else:
                err = parity.check_acf(got, ref, parity.TC_TOL, what=what)
        worst = max(worst, err)
    print(f"{method}: worst error over 256 instances {worst:.2e}")
