"""Tensor-core banded Gram path (tcgen05) vs the FP64 oracle (GPU).

Tolerance (split forms): 1e-5 of MSD_ref(tau_max) for the MSD and of C_ref(0)
for correlations, at every lag.
"""
import numpy as np
import pytest

import oracle
from paper_1708_08619_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ACCURATE = ["fp16x3", "tf32x3", "bf16x4"]


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


@pytest.fixture(scope="module")
def small():
    x = synth.random_walk_positions(1000, 512, 0.01, 3.0, seed=synth.BASE_SEED)
    v = synth.ou_velocities(1000, 512, 0.1, 1.0, seed=synth.BASE_SEED + 1)
    return x, v, oracle.msd(x, 500, 1), oracle.acf(v, 500, 1)


@pytest.mark.parametrize("method", ACCURATE)
def test_small_config(T, small, method):
    x, v, rm, rc = small
    m = T.tcorr_msd(dev(x), 500, 1, method).cpu().numpy()
    c = T.tcorr_acf(dev(v), 500, 1, method).cpu().numpy()
    assert m[0] == 0.0
    parity.check_tc_msd(m, rm, what=f"{method} msd")
    parity.check_acf(c, rc, parity.TC_TOL, what=f"{method} acf")
    assert T.tcorr_status_poll() == 0


def test_bf16x3_within_its_bound(T, small):
    """BF16 x3 drops lo.lo: its MSD error is bounded by a few bf16 ulps^2 of |x|."""
    x, v, rm, rc = small
    m = T.tcorr_msd(dev(x), 500, 1, "bf16x3").cpu().numpy()
    c = T.tcorr_acf(dev(v), 500, 1, "bf16x3").cpu().numpy()
    assert np.max(np.abs(m - rm)) / rm[-1] < 1e-4
    parity.check_acf(c, rc, 1e-4, what="bf16x3 acf")


SHAPES = [  # (T, N, tau_max, stride)
    (1, 1, 0, 1), (2, 1, 1, 1), (5, 3, 4, 2), (129, 7, 128, 1), (300, 37, 299, 1),
    (300, 37, 100, 3), (1000, 5, 400, 7), (257, 130, 256, 200), (50, 11, 0, 1),
    (64, 1, 63, 64), (400, 43, 399, 1), (700, 6, 650, 129), (131, 300, 130, 1),
    (600, 700, 500, 1), (900, 40, 300, 2),
]


@pytest.mark.parametrize("method", ACCURATE)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "T%d_N%d_tm%d_s%d" % s)
def test_edge_shapes(T, shape, method):
    Tn, N, tm, s = shape
    rng = np.random.default_rng(hash(shape) & 0xffff)
    x = (rng.normal(size=(Tn, N, 3)).cumsum(axis=0) * 0.1 + rng.uniform(0, 3, size=(1, N, 3)))
    x = x.astype(np.float32)
    a = rng.normal(size=(Tn, N, 3)).astype(np.float32)
    m = T.tcorr_msd(dev(x), tm, s, method).cpu().numpy()
    c = T.tcorr_acf(dev(a), tm, s, method).cpu().numpy()
    rm = oracle.msd(x, tm, s)
    assert m[0] == 0.0
    if tm > 0:
        parity.check_tc_msd(m, rm, what=f"{method} msd {shape}", tau_max_ref=np.max(rm))
    parity.check_acf(c, oracle.acf(a, tm, s), parity.TC_TOL, what=f"{method} acf {shape}")


def test_constant_velocity(T):
    x, v = synth.constant_velocity(500, 64, seed=5)
    v2 = (v ** 2).sum(axis=1).mean()
    want = v2 * np.arange(500, dtype=np.float64) ** 2
    for method in ACCURATE:
        m = T.tcorr_msd(dev(x), 499, 1, method).cpu().numpy()
        assert np.max(np.abs(m - want)) / want[-1] < parity.TC_TOL, method


def test_deterministic(T):
    x = synth.random_walk_positions(900, 300, 0.02, 3.0, seed=7)
    xd = dev(x)
    for method in ACCURATE:
        a = T.tcorr_msd(xd, 600, 2, method).cpu().numpy()
        b = T.tcorr_msd(xd, 600, 2, method).cpu().numpy()
        assert np.array_equal(a, b), method
    assert T.tcorr_status_poll() == 0


@pytest.fixture(scope="module")
def water(T):
    Tn, N = 10000, 32768
    x = synth.random_walk_positions_device(Tn, N, 0.005, 5.0, seed=synth.BASE_SEED,
                                           sites_per_molecule=3)
    v = synth.ou_velocities_device(Tn, N, 0.05, 1.0, seed=synth.BASE_SEED + 1)
    yield x, v, x.cpu().numpy(), v.cpu().numpy()
    del x, v
    torch.cuda.empty_cache()


# 48 evenly spaced lags, the first tile edges, and every lag of the last column
# tile of the band rows (tau_max - 191 .. tau_max)
WATER_TM = 2000
WATER_LAGS = np.unique(np.concatenate([
    np.linspace(0, WATER_TM, 48).astype(np.int64), [1, 2, 3, 10, 127, 128, 129, 191, 192, 255, 256],
    np.arange(WATER_TM - 191, WATER_TM + 1)]))


@pytest.mark.slow
@pytest.mark.parametrize("stride", [1, 3])
def test_water_scale_sampled_lags(T, water, stride):
    """N=32768 (3-site molecules), T=10000, tau_max=2000, FP16x3: 48 spread lags
    and the whole last column tile vs the oracle, origin stride 1 and 3."""
    x, v, xh, vh = water
    tm = WATER_TM
    m = T.tcorr_msd(x, tm, stride, "fp16x3").cpu().numpy()
    c = T.tcorr_acf(v, tm, stride, "fp16x3").cpu().numpy()
    lags = WATER_LAGS
    rm = oracle.msd(xh, stride=stride, lags=lags)
    rc = oracle.acf(vh, stride=stride, lags=lags)
    assert m[0] == 0.0
    parity.check_tc_msd(m[lags], rm, what=f"water msd, stride {stride}")
    parity.check_acf(c[lags], rc, parity.TC_TOL, what=f"water acf, stride {stride}")


