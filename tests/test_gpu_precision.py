"""Precision workload at full size (GPU, slow): N=100000 atoms, T=20000 frames,
tau_max=10000, start positions uniform in [0, 100) nm plus a random walk of
sigma 0.005 nm per axis per frame (large offsets stress the cancellation in
S(t0) + S(t0+tau) - 2G), OU velocities (gamma 0.05) for the correlation.
Every split tensor-core method is checked at sampled lags against the FP64
oracle: |d| / MSD_ref(tau_max) and |d| / C_ref(0) <= 1e-5."""
import numpy as np
import pytest

import oracle
from paper_1708_08619_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TN, NA, TM = 20000, 100000, 10000
LAGS = np.array([0, 1, 2, 5, 64, 127, 128, 191, 192, 1000, 5000, 9999, 10000])


@pytest.fixture(scope="module")
def T():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < 100e9:
        pytest.skip("needs a large-memory GPU")
    build.build()
    tcorr.load()
    return tcorr


@pytest.fixture(scope="module")
def data(T):
    x = synth.random_walk_positions_device(TN, NA, 0.005, 100.0, seed=synth.BASE_SEED + 3)
    xh = x.cpu().numpy()
    rm = oracle.msd(xh, stride=1, lags=LAGS)
    del xh
    v = synth.ou_velocities_device(TN, NA, 0.05, 1.0, seed=synth.BASE_SEED + 4)
    vh = v.cpu().numpy()
    rc = oracle.acf(vh, stride=1, lags=LAGS)
    del vh
    return x, v, rm, rc


@pytest.mark.parametrize("method", ["fp16x3", "tf32x3", "bf16x4", "bf16x3"])
def test_precision_workload(T, data, method):
    x, v, rm, rc = data
    ws = torch.empty(T.tcorr_workspace_size(TN, NA, TM, 1, method), dtype=torch.uint8, device="cuda")
    m = T.tcorr_msd(x, TM, 1, method, ws=ws).cpu().numpy()
    c = T.tcorr_acf(v, TM, 1, method, ws=ws).cpu().numpy()
    del ws
    assert m[0] == 0.0
    err_m = np.max(np.abs(m[LAGS] - rm)) / rm[-1]
    err_c = np.max(np.abs(c[LAGS] - rc)) / abs(rc[0])
    print(f"{method}: msd err {err_m:.2e}, acf err {err_c:.2e}")
    assert err_m <= parity.TC_TOL and err_c <= parity.TC_TOL
    assert T.tcorr_status_poll() == 0
