"""FFT route (method "fft"): MSD, autocorrelation and cross-correlation
through the correlation theorem, against the oracle (GPU)."""
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


@pytest.mark.parametrize("Tn,N,tm,s", [
    (1000, 64, 999, 1),     # tau_max = T - 1: the case the route is for (FP32 transforms missed 1e-5 here)
    (1000, 64, 300, 1),
    (777, 40, 776, 3),      # strided origins: masked origin-side transform
    (640, 7, 200, 2),
    (300, 1, 299, 1),       # one atom (K = 3)
    (97, 5, 0, 1),          # lag 0 only
    (12000, 3, 5000, 1),    # L = 5 2^12: column pass of length 8, rows of 2560 (radix-5 stage)
    (7000, 4, 5000, 2),     # L = 3 2^12: column pass of length 4, rows of 3072 (radix-3), masked
    (40000, 1, 39999, 1),   # L = 5 2^14: column pass of length 32
])
def test_fft_msd_acf_match_oracle(T, Tn, N, tm, s):
    x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=synth.BASE_SEED + Tn + N)
    v = synth.ou_velocities(Tn, N, 0.05, 1.0, seed=synth.BASE_SEED + 2 * Tn + N)
    lags = np.arange(tm + 1)
    m = T.tcorr_msd(torch.from_numpy(x).cuda(), tm, s, "fft").cpu().numpy()
    c = T.tcorr_acf(torch.from_numpy(v).cuda(), tm, s, "fft").cpu().numpy()
    m_ref = oracle.msd(x, stride=s, lags=lags)
    c_ref = oracle.acf(v, stride=s, lags=lags)
    assert m[0] == 0.0
    if tm > 0:
        assert np.max(np.abs(m - m_ref)) / m_ref[-1] <= parity.TC_TOL, np.max(np.abs(m - m_ref)) / m_ref[-1]
    assert np.max(np.abs(c - c_ref)) / abs(c_ref[0]) <= parity.TC_TOL
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("s", [1, 2])
def test_fft_xcf_matches_oracle(T, s):
    u = synth.ou_velocities(1300, 24, 0.05, 1.0, seed=51)
    a = (u[:1200] + synth.ou_velocities(1200, 24, 0.5, 0.5, seed=52)).astype(np.float32)
    b = np.ascontiguousarray(u[100:1300])
    got = T.tcorr_xcf(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 1199, s, "fft").cpu().numpy()
    ref = oracle.xcf(a, b, 1199, s)
    scale = np.sqrt(oracle.acf(a, lags=np.array([0]))[0] * oracle.acf(b, lags=np.array([0]))[0])
    assert np.max(np.abs(got - ref)) / scale <= parity.TC_TOL


def test_fft_many_column_chunks(T):
    """K larger than one chunk of columns (2 x 2^23 / L columns per chunk)."""
    Tn, N, tm = 4000, 6000, 3999            # L = 8192 -> 2048 columns per chunk, K = 18000: 9 chunks
    v = synth.ou_velocities(Tn, N, 0.1, 1.0, seed=53)
    c = T.tcorr_acf(torch.from_numpy(v).cuda(), tm, 1, "fft").cpu().numpy()
    lags = np.array([0, 1, 2, 100, 1000, 3000, 3999])
    ref = oracle.acf(v, stride=1, lags=lags)
    assert np.max(np.abs(c[lags] - ref)) / abs(ref[0]) <= parity.TC_TOL


def test_fft_not_in_batch(T):
    x = torch.from_numpy(synth.ou_velocities(200, 4, 0.1, 1.0, seed=54)).cuda()
    out = torch.empty(51, dtype=torch.float64, device="cuda")
    inst = T.make_instances([(1, x, 50, 1, out)])
    with pytest.raises(T.TcorrError):
        T.tcorr_batch(inst, "fft")


@pytest.mark.slow
def test_fft_long_series_last_lags(T):
    """T = 100000 frames with tau_max = T - 1 (padded length 2^18: 64 x 4096).
    The last lags have n_o = 1, 2, ... origins, so the transform's rounding
    error, spread evenly over all lags, is divided by a single origin there;
    the double-float transforms keep it far below 1e-5 of C(0)."""
    Tn, N = 100000, 2
    v = synth.ou_velocities(Tn, N, 0.01, 1.0, seed=71)
    x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=72)
    lags = np.unique(np.concatenate([np.linspace(0, Tn - 1, 40).astype(np.int64), np.arange(Tn - 20, Tn)]))
    c = T.tcorr_acf(torch.from_numpy(v).cuda(), Tn - 1, 1, "fft").cpu().numpy()
    m = T.tcorr_msd(torch.from_numpy(x).cuda(), Tn - 1, 1, "fft").cpu().numpy()
    rc = oracle.acf(v, stride=1, lags=lags)
    rm = oracle.msd(x, stride=1, lags=lags)
    err_c = np.max(np.abs(c[lags] - rc)) / abs(rc[0])
    err_m = np.max(np.abs(m[lags] - rm)) / rm[-1]
    print(f"fft T={Tn}, tau_max=T-1: acf err {err_c:.2e} of C(0), msd err {err_m:.2e} of MSD(tau_max)")
    assert err_c <= parity.TC_TOL and err_m <= parity.TC_TOL
    assert T.tcorr_status_poll() == 0
