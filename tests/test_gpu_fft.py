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
    """K larger than one chunk of columns (chunks of 2^27 / L columns)."""
    Tn, N, tm = 4000, 6000, 3999            # L = 8192 -> 16384 columns per chunk, K = 18000
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
