"""Band contraction on CTA pairs (cta_group::2, TCORR_PAIR=1) vs the FP64 oracle (GPU).

The pair kernel computes two row tiles per M = 256 product with the frame
tile's rows split between the two CTAs; odd row tiles see their lags shifted
by one row tile in the window layout, which the lag reduction undoes.  Same
tolerances as the single-CTA tensor-core path: 1e-5 of MSD_ref(tau_max) and
of C_ref(0) at every lag.
"""
import os

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
    old = os.environ.get("TCORR_PAIR")
    os.environ["TCORR_PAIR"] = "1"      # read by the library at every call
    yield tcorr
    if old is None:
        del os.environ["TCORR_PAIR"]
    else:
        os.environ["TCORR_PAIR"] = old


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [  # (T, N, tau_max, stride): odd and even row-tile counts, narrow last columns, strides
    (1, 1, 0, 1), (5, 3, 4, 2), (129, 7, 128, 1), (300, 37, 299, 1), (300, 37, 100, 3),
    (1000, 5, 400, 7), (257, 130, 256, 200), (400, 43, 399, 1), (700, 6, 650, 129),
    (600, 700, 500, 1), (900, 40, 300, 2), (1300, 9, 1299, 1),
]


@pytest.mark.parametrize("method", ["fp16x3", "tf32x3", "bf16x4"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "T%d_N%d_tm%d_s%d" % s)
def test_pair_edge_shapes(T, shape, method):
    Tn, N, tm, s = shape
    rng = np.random.default_rng(sum(shape) * 7919 + 11)
    x = (rng.normal(size=(Tn, N, 3)).cumsum(axis=0) * 0.1 + rng.uniform(0, 3, size=(1, N, 3))).astype(np.float32)
    a = rng.normal(size=(Tn, N, 3)).astype(np.float32)
    m = T.tcorr_msd(dev(x), tm, s, method).cpu().numpy()
    c = T.tcorr_acf(dev(a), tm, s, method).cpu().numpy()
    rm = oracle.msd(x, tm, s)
    assert m[0] == 0.0
    if tm > 0:
        parity.check_tc_msd(m, rm, what=f"pair {method} msd {shape}", tau_max_ref=np.max(rm))
    parity.check_acf(c, oracle.acf(a, tm, s), parity.TC_TOL, what=f"pair {method} acf {shape}")
    assert T.tcorr_status_poll() == 0


def test_pair_mid_size_sampled_lags(T):
    """Several K-groups and supertiles: T = 3000, N = 6000, tau_max = 1500, lags at tile edges."""
    Tn, N, tm = 3000, 6000, 1500
    x = synth.random_walk_positions(Tn, N, 0.01, 50.0, seed=synth.BASE_SEED + 71)
    v = synth.ou_velocities(Tn, N, 0.05, 1.0, seed=synth.BASE_SEED + 72)
    lags = sorted({0, 1, 2, 63, 64, 127, 128, 129, 191, 192, 255, 256, 383, 384, 700, 1023,
                   1308, 1309, 1310, 1400, 1499, 1500})
    m = T.tcorr_msd(dev(x), tm, 1, "fp16x3").cpu().numpy()
    c = T.tcorr_acf(dev(v), tm, 1, "fp16x3").cpu().numpy()
    rm = oracle.msd(x, tm, 1, lags=lags)
    rc = oracle.acf(v, tm, 1, lags=lags)
    err_m = np.max(np.abs(m[lags] - rm)) / rm[-1]
    err_c = np.max(np.abs(c[lags] - rc)) / abs(rc[0])
    assert err_m <= parity.TC_TOL, f"pair msd: {err_m:.3e}"
    assert err_c <= parity.TC_TOL, f"pair acf: {err_c:.3e}"


def test_pair_matches_single_cta_path(T):
    """Same inputs through both tilings: the sums differ only in FP32 window rounding."""
    x = synth.random_walk_positions(2000, 3000, 0.01, 30.0, seed=synth.BASE_SEED + 73)
    d = dev(x)
    pair = T.tcorr_msd(d, 1000, 1, "fp16x3").cpu().numpy()
    os.environ["TCORR_PAIR"] = "0"
    try:
        single = T.tcorr_msd(d, 1000, 1, "fp16x3").cpu().numpy()
    finally:
        os.environ["TCORR_PAIR"] = "1"
    assert np.max(np.abs(pair - single)) / single[-1] <= 1e-6
