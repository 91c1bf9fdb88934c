"""Cross-correlation <A(t0).B(t0+tau)> (tcorr_xcf): parity with the oracle on
both methods, and X(A, A) equal to the autocorrelation (GPU)."""
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


def pair(Tn, N, seed, lag=7):
    """Two correlated signals from one OU field u: A(t) = u(t) + noise and
    B(t) = u(t + lag), so X_AB(tau) ~ C_u(tau + lag) and X_BA(tau) ~ C_u(tau - lag)."""
    b = synth.ou_velocities(Tn + lag, N, 0.05, 1.0, seed=seed)
    noise = synth.ou_velocities(Tn, N, 0.5, 0.5, seed=seed + 1)
    a = (b[:Tn] + noise).astype(np.float32)
    return a, np.ascontiguousarray(b[lag:lag + Tn])


def scale_of(a, b):
    """Cauchy-Schwarz bound on |X(tau)|: sqrt(C_AA(0) C_BB(0))."""
    return float(np.sqrt(oracle.acf(a, lags=np.array([0]))[0] * oracle.acf(b, lags=np.array([0]))[0]))


@pytest.mark.parametrize("method", ["plain", "fp16x3", "tf32x3", "bf16x4"])
@pytest.mark.parametrize("Tn,N,tm,s", [(1200, 64, 400, 1), (900, 40, 899, 2), (700, 1, 300, 3), (513, 11, 0, 1)])
def test_xcf_matches_oracle(T, method, Tn, N, tm, s):
    a, b = pair(Tn, N, synth.BASE_SEED + Tn + N)
    got = T.tcorr_xcf(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), tm, s, method).cpu().numpy()
    ref = oracle.xcf(a, b, tm, s)
    tol = parity.PLAIN_TOL if method == "plain" else parity.TC_TOL
    assert np.max(np.abs(got - ref)) / scale_of(a, b) <= tol, (method, Tn, N, tm, s)
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("method", ["plain", "fp16x3"])
def test_xcf_of_a_signal_with_itself_is_its_acf(T, method):
    """N = 40 keeps the autocorrelation on the band form, so both calls run the
    same arithmetic on the same operands."""
    x = torch.from_numpy(synth.ou_velocities(800, 40, 0.1, 1.0, seed=41)).cuda()
    assert np.array_equal(T.tcorr_xcf(x, x, 300, 1, method).cpu().numpy(),
                          T.tcorr_acf(x, 300, 1, method).cpu().numpy())


def test_xcf_order_of_the_signals_matters(T):
    a, b = pair(1000, 16, 42, lag=25)
    ab = T.tcorr_xcf(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 100, 1, "fp16x3").cpu().numpy()
    ba = T.tcorr_xcf(torch.from_numpy(b).cuda(), torch.from_numpy(a).cuda(), 100, 1, "fp16x3").cpu().numpy()
    # X_AB decays from tau = 0; X_BA peaks where B's advance is undone, tau = 25
    assert int(np.argmax(ab)) == 0 and abs(int(np.argmax(ba)) - 25) <= 3
    ref_ba = oracle.xcf(b, a, 100)
    assert np.max(np.abs(ba - ref_ba)) / scale_of(a, b) <= parity.TC_TOL


@pytest.mark.parametrize("method", ["fp16x3", "tf32x3"])
@pytest.mark.parametrize("N,Tn,tm", [(1, 6000, 1500), (8, 3000, 700)])
def test_xcf_small_k_polyphase(T, method, N, Tn, tm):
    """K = 3N <= 24, stride 1, tau_max >= 383: the polyphase form, with the
    unshifted copy of A on the origin side and 8 shifted copies of B."""
    a, b = pair(Tn, N, synth.BASE_SEED + 7 * N, lag=40)
    got = T.tcorr_xcf(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), tm, 1, method).cpu().numpy()
    ref = oracle.xcf(a, b, tm, 1)
    assert np.max(np.abs(got - ref)) / scale_of(a, b) <= parity.TC_TOL
    x = torch.from_numpy(a).cuda()
    # X(A, A) on the polyphase form equals the polyphase autocorrelation bit for bit
    assert np.array_equal(T.tcorr_xcf(x, x, tm, 1, method).cpu().numpy(), T.tcorr_acf(x, tm, 1, method).cpu().numpy())
