"""Collective signal (tcorr_collective) and the collective quantities built on
it -- the Einstein-Helfand MSD of summed charged positions, the charge-current
autocorrelation and the velocity cross-correlation of two species -- against
the FP64 oracle (GPU)."""
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


def check_collective(got, x, w, ref):
    """Each entry within one FP32 rounding of the FP64 sum, plus the compensated
    sums' own errors (about 2^-44 of sum_i |w_i x_i| for the frame and, with a
    reference, for the reference frame, whose totals are subtracted)."""
    want = oracle.collective(x, w, ref)
    ww = np.ones(x.shape[1]) if w is None else w.astype(np.float64)
    mag = np.abs(ww[None, :, None] * x.astype(np.float64)).sum(axis=1)
    if ref >= 0:
        mag = mag + mag[ref][None]
    err = np.abs(got.reshape(-1, 3).astype(np.float64) - want)
    assert np.all(err <= 6e-8 * np.abs(want) + 1e-12 * mag + 1e-30), float(np.max(err / (np.abs(want) + 1e-300)))


@pytest.mark.parametrize("Tn,N,ref,weights", [
    (50, 1, -1, "unit"), (300, 1000, -1, "charges"), (300, 1000, 0, "charges"), (300, 1000, 150, "random"),
    (7, 70001, 3, "charges"), (2000, 33, 1999, "unit"),
])
def test_collective_matches_oracle(T, Tn, N, ref, weights):
    rng = np.random.default_rng(Tn + N)
    x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=Tn * 7 + N)
    w = None
    if weights == "charges":
        w = np.where(rng.random(N) < 0.5, 0.8, -0.8).astype(np.float32)
    elif weights == "random":
        w = rng.normal(size=N).astype(np.float32)
    got = T.tcorr_collective(dev(x), dev(w) if w is not None else None, ref).cpu().numpy()
    assert got.shape == (Tn, 1, 3)
    check_collective(got, x, w, ref)
    if ref >= 0:
        assert np.all(got[ref] == 0.0)          # the reference frame's own totals cancel exactly


def test_collective_deterministic(T):
    x = dev(synth.ou_velocities(400, 5000, 0.1, 1.0, seed=3))
    w = dev(np.random.default_rng(4).normal(size=5000).astype(np.float32))
    a = T.tcorr_collective(x, w).cpu().numpy()
    b = T.tcorr_collective(x, w).cpu().numpy()
    assert np.array_equal(a, b)
    assert T.tcorr_status_poll() == 0


def charges(N, seed):
    rng = np.random.default_rng(seed)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).astype(np.float32)
    return q[rng.permutation(N)]


@pytest.mark.parametrize("method", ["plain", "fp16x3", "fft", "auto"])
def test_einstein_helfand_msd(T, method):
    """MSD of sum_i q_i r_i (referenced to the middle frame), all origins."""
    Tn, N, tm = 2000, 512, 600
    x = synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=51)
    q = charges(N, 52)
    J = T.tcorr_collective(dev(x), dev(q), Tn // 2)
    got = T.tcorr_msd(J, tm, 1, method).cpu().numpy()
    Jref = oracle.collective(x, q, Tn // 2).astype(np.float32)[:, None, :]
    want = oracle.msd(Jref, tm, 1)
    if method == "plain":
        assert got[0] == 0.0 and np.max(np.abs(got[1:] - want[1:]) / want[1:]) <= parity.PLAIN_TOL
    else:
        parity.check_tc_msd(got, want, what=f"Einstein-Helfand {method}", tau_max_ref=want[-1])


@pytest.mark.parametrize("method", ["plain", "fp16x3", "auto"])
def test_charge_current_autocorrelation(T, method):
    """Autocorrelation of J(t) = sum_i q_i v_i; tau_max >= 383 takes the polyphase form on the
    tensor cores (K = 3)."""
    Tn, N, tm = 6000, 256, 800
    v = synth.ou_velocities(Tn, N, 0.05, 1.0, seed=53)
    q = charges(N, 54)
    J = T.tcorr_collective(dev(v), dev(q))
    got = T.tcorr_acf(J, tm, 1, method).cpu().numpy()
    want = oracle.acf(oracle.collective(v, q).astype(np.float32)[:, None, :], tm, 1)
    tol = parity.PLAIN_TOL if method == "plain" else parity.TC_TOL
    parity.check_acf(got, want, tol, what=f"charge current {method}")


@pytest.mark.parametrize("method", ["plain", "fp16x3", "fft"])
def test_species_velocity_cross_correlation(T, method):
    """<J_A(t0) . J_B(t0 + tau)> with J_S the summed velocities of species S (0/1 weights)."""
    Tn, N, tm = 3000, 300, 700
    v = synth.ou_velocities(Tn, N, 0.1, 1.0, seed=55)
    wa = (np.arange(N) % 3 == 0).astype(np.float32)
    wb = (np.arange(N) % 3 != 0).astype(np.float32)
    vd = dev(v)
    ja, jb = T.tcorr_collective(vd, dev(wa)), T.tcorr_collective(vd, dev(wb))
    got = T.tcorr_xcf(ja, jb, tm, 1, method).cpu().numpy()
    ra = oracle.collective(v, wa).astype(np.float32)[:, None, :]
    rb = oracle.collective(v, wb).astype(np.float32)[:, None, :]
    want = oracle.xcf(ra, rb, tm, 1)
    scale = np.sqrt(oracle.acf(ra, 0, 1)[0] * oracle.acf(rb, 0, 1)[0])
    tol = parity.PLAIN_TOL if method == "plain" else parity.TC_TOL
    assert np.max(np.abs(got - want)) / scale <= tol
