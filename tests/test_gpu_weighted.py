"""Weighted atom averages (tcorr_msd_weighted / tcorr_acf_weighted) against the
FP64 oracle and against the unweighted calls (GPU)."""
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


def check(kind, got, want, method):
    if method == "plain":
        if kind == 0:
            assert got[0] == 0.0
            assert np.max(np.abs(got[1:] - want[1:]) / want[1:]) <= parity.PLAIN_TOL
        else:
            parity.check_acf(got, want, parity.PLAIN_TOL, what="weighted plain acf")
    elif kind == 0:
        parity.check_tc_msd(got, want, what=f"weighted {method} msd", tau_max_ref=want[-1])
    else:
        parity.check_acf(got, want, parity.TC_TOL, what=f"weighted {method} acf")


@pytest.mark.parametrize("method", ["plain", "fp16x3", "tf32x3", "fft", "auto"])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("Tn,N,tm,s", [(1500, 200, 600, 1), (900, 37, 400, 3), (3000, 4, 1200, 1)])
def test_weighted_matches_oracle(T, method, kind, Tn, N, tm, s):
    """Mass-like weights (uniform in [0.5, 16]); N = 4 with tau_max >= 383 takes the polyphase
    form for the tensor-core autocorrelation."""
    rng = np.random.default_rng(Tn + N + kind)
    x = (synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=Tn + N) if kind == 0
         else synth.ou_velocities(Tn, N, 0.1, 1.0, seed=Tn + N))
    w = rng.uniform(0.5, 16.0, size=N).astype(np.float32)
    f = T.tcorr_msd_weighted if kind == 0 else T.tcorr_acf_weighted
    got = f(dev(x), dev(w), tm, s, method).cpu().numpy()
    want = (oracle.msd_weighted if kind == 0 else oracle.acf_weighted)(x, w, tm, s)
    check(kind, got, want, method)


@pytest.mark.parametrize("method", ["plain", "fp16x3", "fft"])
def test_unit_weights_give_the_plain_average(T, method):
    """With w = 1 the autocorrelation's copy is the signal itself, so every method returns the
    unweighted result bit for bit; so does the tensor-core MSD, whose split forms the same
    x - x_m as the copy.  The plain and FFT MSD subtract frames their own way, so there the
    copy's rounding of x - x_m shows (within the method's tolerance)."""
    x = synth.random_walk_positions(800, 64, 0.01, 3.0, seed=81)
    v = synth.ou_velocities(800, 64, 0.1, 1.0, seed=82)
    ones = torch.ones(64, dtype=torch.float32, device="cuda")
    vd, xd = dev(v), dev(x)
    assert np.array_equal(T.tcorr_acf_weighted(vd, ones, 300, 1, method).cpu().numpy(),
                          T.tcorr_acf(vd, 300, 1, method).cpu().numpy())
    mw = T.tcorr_msd_weighted(xd, ones, 300, 1, method).cpu().numpy()
    m = T.tcorr_msd(xd, 300, 1, method).cpu().numpy()
    if method == "fp16x3":
        assert np.array_equal(mw, m)
    else:
        check(0, mw, oracle.msd(x, 300, 1), method)


def test_selection_and_repetition(T):
    """0/1 weights equal the unweighted call on the selected atoms; integer weights equal the
    unweighted call on a trajectory holding atom i w_i times."""
    rng = np.random.default_rng(83)
    Tn, N, tm = 1200, 50, 500
    x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=84)
    sel = (np.arange(N) % 4 == 1).astype(np.float32)
    got = T.tcorr_msd_weighted(dev(x), dev(sel), tm, 1, "fp16x3").cpu().numpy()
    want = T.tcorr_msd(dev(x[:, sel > 0, :]), tm, 1, "fp16x3").cpu().numpy()
    parity.check_tc_msd(got, want, what="selection", tau_max_ref=want[-1])
    wi = rng.integers(1, 4, size=N).astype(np.float32)
    got = T.tcorr_msd_weighted(dev(x), dev(wi), tm, 1, "plain").cpu().numpy()
    want = T.tcorr_msd(dev(np.repeat(x, wi.astype(np.int64), axis=1)), tm, 1, "plain").cpu().numpy()
    assert np.max(np.abs(got[1:] - want[1:]) / want[1:]) <= parity.PLAIN_TOL
    assert T.tcorr_status_poll() == 0
