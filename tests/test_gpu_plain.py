"""Plain FP32 path, Green-Kubo and Einstein kernels vs the FP64 oracle (GPU)."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_small_config_msd_vacf(T):
    """N=512, T=1000, tau_max=500, stride 1: random-walk MSD and OU VACF."""
    x = synth.random_walk_positions(1000, 512, 0.01, 3.0, seed=synth.BASE_SEED)
    v = synth.ou_velocities(1000, 512, 0.1, 1.0, seed=synth.BASE_SEED + 1)
    m = T.tcorr_msd(dev(x), 500, 1, "plain").cpu().numpy()
    c = T.tcorr_acf(dev(v), 500, 1, "plain").cpu().numpy()
    parity.check_plain_msd(m, oracle.msd(x, 500, 1))
    parity.check_acf(c, oracle.acf(v, 500, 1), parity.PLAIN_TOL)


SHAPES = [  # (T, N, tau_max, stride)
    (1, 1, 0, 1), (2, 1, 1, 1), (5, 3, 4, 2), (129, 7, 128, 1), (300, 37, 299, 1),
    (300, 37, 100, 3), (1000, 5, 400, 7), (257, 130, 256, 200), (50, 11, 0, 1),
    (64, 1, 63, 64), (400, 43, 399, 1), (700, 6, 650, 129), (131, 300, 130, 1),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "T%d_N%d_tm%d_s%d" % s)
def test_edge_shapes(T, shape):
    Tn, N, tm, s = shape
    rng = np.random.default_rng(hash(shape) & 0xffff)
    x = (rng.normal(size=(Tn, N, 3)).cumsum(axis=0) * 0.1 + rng.uniform(0, 3, size=(1, N, 3)))
    x = x.astype(np.float32)
    a = rng.normal(size=(Tn, N, 3)).astype(np.float32)
    m = T.tcorr_msd(dev(x), tm, s, "plain").cpu().numpy()
    c = T.tcorr_acf(dev(a), tm, s, "plain").cpu().numpy()
    parity.check_plain_msd(m, oracle.msd(x, tm, s), what=f"msd {shape}")
    # white-noise correlations are ~0 beyond lag 0: scale by C(0)
    parity.check_acf(c, oracle.acf(a, tm, s), parity.PLAIN_TOL, what=f"acf {shape}")


@pytest.mark.parametrize("Tn,N", [(500, 64), (300, 1000)])
def test_constant_velocity_closed_form(T, Tn, N):
    """Ballistic motion: MSD = <|v|^2> tau^2, and the autocorrelation of the
    constant velocities is <|v|^2> at every lag.  Every origin gives the same
    pair sum here, so rounding cannot average out over origins; the short FP32
    runs of the plain kernel keep it within the 1e-6 bar all the same (K = 192
    is one segment, K = 3000 spans twelve)."""
    x, v = synth.constant_velocity(Tn, N, seed=5)
    m = T.tcorr_msd(dev(x), Tn - 1, 1, "plain").cpu().numpy()
    v2 = (v ** 2).sum(axis=1).mean()
    want = v2 * np.arange(Tn, dtype=np.float64) ** 2
    parity.check_plain_msd(m, want, what="ballistic msd")
    a = np.ascontiguousarray(np.broadcast_to(v.astype(np.float32)[None], (Tn, N, 3)))
    c = T.tcorr_acf(dev(a), Tn - 1, 1, "plain").cpu().numpy()
    parity.check_acf(c, np.full(Tn, v2), parity.PLAIN_TOL, what="constant-velocity acf")


def test_deterministic_and_workspace_independent(T):
    x = synth.random_walk_positions(600, 200, 0.02, 3.0, seed=7)
    xd = dev(x)
    need = T.tcorr_workspace_size(600, 200, 300, 2, "plain")
    ws = torch.full((need + 4096,), 0x7f, dtype=torch.uint8, device="cuda")
    a = T.tcorr_msd(xd, 300, 2, "plain").cpu().numpy()
    b = T.tcorr_msd(xd, 300, 2, "plain", ws=ws).cpu().numpy()
    c = T.tcorr_acf(xd, 300, 2, "plain").cpu().numpy()
    d = T.tcorr_acf(xd, 300, 2, "plain", ws=ws).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(c, d)
    assert T.tcorr_status_poll() == 0


def test_gk_integrate_and_einstein(T):
    rng = np.random.default_rng(9)
    # block spans of 2048 increments; up to 32 blocks one launch, more three
    for n in (1, 2, 3, 1000, 2048, 2049, 2050, 4098, 5001, 20001, 65537, 65538, 300001):
        cvals = rng.normal(size=n)
        got = T.gk_integrate(dev(cvals), 0.25, 3.5).cpu().numpy()
        want = oracle.gk_integrate(cvals, 0.25, 3.5)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max(initial=1.0))
    msd = np.cumsum(np.abs(rng.normal(size=2001)))
    got = T.einstein_slope(dev(msd), 0.5, 3).cpu().numpy()
    want = oracle.einstein(msd, 0.5, 3)
    assert abs(got[0] / want[0] - 1) < 1e-12 and abs(got[1] / want[1] - 1) < 1e-14
    got2 = T.einstein_slope(dev(msd), 0.5, 2, 17, 1900).cpu().numpy()
    want2 = oracle.einstein(msd, 0.5, 2, 17, 1900)
    assert abs(got2[0] / want2[0] - 1) < 1e-12


def test_gk_integrate_batch(T):
    rng = np.random.default_rng(10)
    # single-launch and three-pass sizes; padded rows; a grid taller than 65535 series
    for n, count, pad in ((1, 3, 0), (20001, 65, 0), (5001, 7, 13), (65538, 3, 5), (3, 70000, 1)):
        c = rng.normal(size=(count, n + pad))
        cd = dev(c)[:, :n]
        got = T.gk_integrate_batch(cd, 0.25, 3.5).cpu().numpy()
        for j in {0, count // 2, count - 1}:
            want = oracle.gk_integrate(c[j, :n], 0.25, 3.5)
            assert np.allclose(got[j], want, rtol=1e-12, atol=1e-12 * np.abs(want).max(initial=1.0)), (n, j)
            single = T.gk_integrate(cd[j].contiguous(), 0.25, 3.5).cpu().numpy()
            assert np.array_equal(got[j], single), (n, j)      # same arithmetic as one call
    # a padded output
    c = rng.normal(size=(4, 3000))
    out = torch.full((4, 3010), 7.0, dtype=torch.float64, device="cuda")
    T.gk_integrate_batch(dev(c), 1.0, 1.0, out=out[:, :3000])
    o = out.cpu().numpy()
    assert np.all(o[:, 3000:] == 7.0)
    assert np.allclose(o[2, :3000], oracle.gk_integrate(c[2], 1.0, 1.0), rtol=1e-12, atol=1e-9)
    assert T.tcorr_status_poll() == 0


def test_batch_matches_single_calls(T):
    rng = np.random.default_rng(21)
    items, refs = [], []
    for i in range(5):
        Tn = int(rng.integers(50, 400))
        N = int(rng.integers(1, 60))
        tm = int(rng.integers(0, Tn))
        s = int(rng.integers(1, 4))
        x = dev(rng.normal(size=(Tn, N, 3)).astype(np.float32))
        kind = i % 2
        out = torch.empty(tm + 1, dtype=torch.float64, device="cuda")
        items.append((kind, x, tm, s, out))
        f = T.tcorr_msd if kind == 0 else T.tcorr_acf
        refs.append(f(x, tm, s, "plain").cpu().numpy())
    inst = T.make_instances(items)
    T.tcorr_batch(inst, "plain")
    torch.cuda.synchronize()
    for (kind, x, tm, s, out), ref in zip(items, refs):
        assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.slow
def test_water_scale_sampled_lags(T):
    """N=32768 (3-site molecules), T=10000, tau_max=2000: sampled lags vs oracle."""
    Tn, N, tm = 10000, 32768, 2000
    x = synth.random_walk_positions_device(Tn, N, 0.005, 5.0, seed=synth.BASE_SEED,
                                           sites_per_molecule=3)
    v = synth.ou_velocities_device(Tn, N, 0.05, 1.0, seed=synth.BASE_SEED + 1)
    m = T.tcorr_msd(x, tm, 1, "plain").cpu().numpy()
    c = T.tcorr_acf(v, tm, 1, "plain").cpu().numpy()
    lags = np.unique(np.concatenate([np.linspace(0, tm, 48).astype(np.int64),
                                     [1, 2, 3, 10, 127, 128, 129, 255, 256],
                                     np.linspace(tm - 191, tm, 16).astype(np.int64)]))
    xh, vh = x.cpu().numpy(), v.cpu().numpy()
    del x, v
    rm = oracle.msd(xh, stride=1, lags=lags)
    rc = oracle.acf(vh, stride=1, lags=lags)
    assert m[0] == 0.0
    assert np.max(np.abs(m[lags[1:]] - rm[1:]) / rm[1:]) <= parity.PLAIN_TOL
    assert np.max(np.abs(c[lags] - rc)) / abs(rc[0]) <= parity.PLAIN_TOL


def test_profile_hooks_time_the_dominant_kernel(T):
    x = dev(synth.random_walk_positions(800, 300, 0.01, 3.0, seed=12))
    T.tcorr_profile_enable(True)
    T.tcorr_profile_read(0)
    T.tcorr_profile_read(1)
    for _ in range(3):
        T.tcorr_msd(x, 300, 1, "plain")
    T.tcorr_acf(x, 300, 1, "plain")
    ms0, n0 = T.tcorr_profile_read(0)
    ms1, n1 = T.tcorr_profile_read(1)
    T.tcorr_profile_enable(False)
    T.tcorr_msd(x, 300, 1, "plain")
    assert n0 == 3 and n1 == 1 and ms0 > 0 and ms1 > 0
    assert T.tcorr_profile_read(0) == (0.0, 0)


def test_device_timeout_sets_status_word_and_context_survives(T):
    assert T.tcorr_status_poll() == 0
    T.tcorr_selftest_timeout()
    assert T.tcorr_status_poll() == 6          # TCORR_ETIMEOUT, reported once
    assert T.tcorr_status_poll() == 0          # and cleared
    x = dev(synth.random_walk_positions(300, 20, 0.01, 3.0, seed=13))
    m = T.tcorr_msd(x, 100, 1, "fp16x3").cpu().numpy()   # the context is still usable
    assert m[0] == 0.0 and np.all(np.isfinite(m))
