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
# 32 evenly spaced lags, tile edges of the first band columns, and the last column
# tile of every band row (lags TM-191 .. TM) at lag stride 3 plus its last 8 lags
LAGS = np.unique(np.concatenate([
    np.linspace(0, TM, 32).astype(np.int64), [1, 2, 5, 64, 127, 128, 191, 192, 383, 384],
    np.arange(TM - 191, TM + 1, 3), np.arange(TM - 7, TM + 1)]))


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
    v = synth.ou_velocities_device(TN, NA, 0.05, 1.0, seed=synth.BASE_SEED + 4)
    xh = x.cpu().numpy()
    vh = v.cpu().numpy()
    rm = oracle.msd(xh, stride=1, lags=LAGS)
    rc = oracle.acf(vh, stride=1, lags=LAGS)
    yield x, v, xh, vh, rm, rc
    del x, v
    torch.cuda.empty_cache()


@pytest.mark.parametrize("method", ["fp16x3", "tf32x3", "bf16x4", "bf16x3"])
def test_precision_workload(T, data, method):
    x, v, _, _, rm, rc = data
    ws = torch.empty(T.tcorr_workspace_size(TN, NA, TM, 1, method), dtype=torch.uint8, device="cuda")
    m = T.tcorr_msd(x, TM, 1, method, ws=ws).cpu().numpy()
    c = T.tcorr_acf(v, TM, 1, method, ws=ws).cpu().numpy()
    del ws
    assert m[0] == 0.0
    err_m = np.max(np.abs(m[LAGS] - rm)) / rm[-1]
    err_c = np.max(np.abs(c[LAGS] - rc)) / abs(rc[0])
    print(f"{method}: msd err {err_m:.2e}, acf err {err_c:.2e} at {len(LAGS)} lags")
    assert err_m <= parity.TC_TOL and err_c <= parity.TC_TOL
    assert T.tcorr_status_poll() == 0


def test_precision_workload_origin_stride_3(T, data):
    """The same arrays with every third frame as an origin (three residues of
    the band tiling), FP16x3, at the same lags."""
    x, v, xh, vh, _, _ = data
    rm = oracle.msd(xh, stride=3, lags=LAGS)
    rc = oracle.acf(vh, stride=3, lags=LAGS)
    ws = torch.empty(T.tcorr_workspace_size(TN, NA, TM, 3, "fp16x3"), dtype=torch.uint8, device="cuda")
    m = T.tcorr_msd(x, TM, 3, "fp16x3", ws=ws).cpu().numpy()
    c = T.tcorr_acf(v, TM, 3, "fp16x3", ws=ws).cpu().numpy()
    del ws
    assert m[0] == 0.0
    parity.check_tc_msd(m[LAGS], rm, what="precision msd, stride 3")
    parity.check_acf(c[LAGS], rc, parity.TC_TOL, what="precision acf, stride 3")
    assert T.tcorr_status_poll() == 0
