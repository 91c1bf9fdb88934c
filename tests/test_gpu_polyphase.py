"""Polyphase recast for small K (flux autocorrelation, few-atom MSD) on the GPU."""
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


@pytest.mark.parametrize("method", ["fp16x3", "tf32x3", "bf16x4"])
def test_flux_acf(T, method):
    """(Pxy, Pxz, Pyz) as [T][1][3], AR(1) phi = 0.999, T = 20000, tau_max = 2000."""
    a = synth.ar1_flux(20000, 0.999, seed=synth.BASE_SEED + 5)
    c = T.tcorr_acf(dev(a), 2000, 1, method).cpu().numpy()
    parity.check_acf(c, oracle.acf(a, 2000, 1), parity.TC_TOL, what=f"flux {method}")
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("shape", [(5000, 5, 1000), (3000, 8, 2999), (1200, 1, 383), (777, 2, 500)])
def test_small_n_msd_and_acf(T, shape):
    Tn, N, tm = shape
    x = synth.random_walk_positions(Tn, N, 0.02, 3.0, seed=Tn + N)
    v = synth.ou_velocities(Tn, N, 0.05, 1.0, seed=Tn + N + 1)
    m = T.tcorr_msd(dev(x), tm, 1, "fp16x3").cpu().numpy()
    c = T.tcorr_acf(dev(v), tm, 1, "fp16x3").cpu().numpy()
    assert m[0] == 0.0
    parity.check_tc_msd(m, oracle.msd(x, tm, 1), what=f"poly msd {shape}")
    parity.check_acf(c, oracle.acf(v, tm, 1), parity.TC_TOL, what=f"poly acf {shape}")


def test_polyphase_agrees_with_band_method(T, monkeypatch):
    a = synth.ar1_flux(6000, 0.99, seed=9)
    ad = dev(a)
    poly = T.tcorr_acf(ad, 1500, 1, "fp16x3").cpu().numpy()
    monkeypatch.setenv("TCORR_NO_POLYPHASE", "1")
    band = T.tcorr_acf(ad, 1500, 1, "fp16x3").cpu().numpy()
    assert np.max(np.abs(poly - band)) / abs(band[0]) < 2e-6


@pytest.mark.slow
def test_long_flux_sampled_lags(T):
    """T = 2,000,000 steps, tau_max = 20,000 (the viscosity workload), sampled lags."""
    a = synth.ar1_flux(2000000, 0.999, seed=synth.BASE_SEED + 6)
    c = T.tcorr_acf(dev(a), 20000, 1, "fp16x3").cpu().numpy()
    lags = np.array([0, 1, 2, 383, 384, 385, 1000, 7777, 19999, 20000])
    rc = oracle.acf(a, stride=1, lags=lags)
    assert np.max(np.abs(c[lags] - rc)) / abs(rc[0]) <= parity.TC_TOL
    cp = T.tcorr_acf(dev(a), 20000, 1, "plain").cpu().numpy()
    assert np.max(np.abs(cp[lags] - rc)) / abs(rc[0]) <= parity.PLAIN_TOL


def test_batch_of_flux_series(T):
    series = [synth.ar1_flux(int(n), 0.999, seed=100 + i) for i, n in enumerate([5000, 12000, 800, 20000])]
    outs = []
    items = []
    for i, a in enumerate(series):
        tm = min(2000, a.shape[0] - 1)
        o = torch.empty(tm + 1, dtype=torch.float64, device="cuda")
        items.append((1, dev(a), tm, 1, o))
    inst = T.make_instances(items)
    T.tcorr_batch(inst, "fp16x3")
    torch.cuda.synchronize()
    for kind, x, tm, s, o in items:
        single = T.tcorr_acf(x, tm, s, "fp16x3").cpu().numpy()
        assert np.array_equal(o.cpu().numpy(), single)


@pytest.mark.slow
def test_full_flux_workload_vs_oracle(T):
    """The Green-Kubo flux workload at full size: one T = 2,000,000 series and a
    batch of 64 series of T = 200,000, tau_max = 20,000, FP16x3 (polyphase),
    every series against the oracle at 30 lags (the polyphase block edges
    383/384/767/768, spread lags and the last ones); the batched running
    integrals of all 65 series against the oracle's integral of the device
    correlations."""
    tm = 20000
    lags = np.unique(np.concatenate([[0, 1, 2, 383, 384, 767, 768, tm - 1, tm],
                                     np.linspace(0, tm, 21).astype(np.int64)]))
    longh = synth.ar1_flux(2000000, 0.999, seed=synth.BASE_SEED + 6)
    shorth = [synth.ar1_flux(200000, 0.999, seed=synth.BASE_SEED + 1000 + i) for i in range(64)]
    outs = torch.full((65, tm + 1), np.nan, dtype=torch.float64, device="cuda")
    T.tcorr_acf(dev(longh), tm, 1, "fp16x3", out=outs[0])
    xs = [dev(a) for a in shorth]
    inst = T.make_instances([(1, x, tm, 1, outs[1 + i]) for i, x in enumerate(xs)])
    T.tcorr_batch(inst, "fp16x3")
    gk = T.gk_integrate_batch(outs, 1.0, 1.0 / 3.0)
    torch.cuda.synchronize()
    assert T.tcorr_status_poll() == 0
    got = outs.cpu().numpy()
    g = gk.cpu().numpy()
    worst = 0.0
    for j, a in enumerate([longh] + shorth):
        ref = oracle.acf(a, stride=1, lags=lags)
        worst = max(worst, parity.check_acf(got[j][lags], ref, parity.TC_TOL, what=f"flux series {j}"))
        # the device integral is that of the device correlation (to FP64 rounding)
        want = oracle.gk_integrate(got[j], 1.0, 1.0 / 3.0)
        assert np.allclose(g[j], want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), j
    print(f"flux workload: worst error {worst:.2e} of C(0) over 65 series")
