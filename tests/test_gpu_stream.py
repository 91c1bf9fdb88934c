"""Streamed (out-of-core) path: a host-resident trajectory processed in time
windows with a tau_max halo (tcorr_msd_stream / tcorr_acf_stream) gives the
whole-trajectory result (GPU)."""
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


def host(x, pinned):
    t = torch.from_numpy(x)
    return t.pin_memory() if pinned else t


def streamed(T, kind, xh, tm, s, method, chunk, pinned=True):
    f = T.tcorr_msd_stream if kind == 0 else T.tcorr_acf_stream
    out = f(host(xh, pinned), tm, s, method, chunk_frames=chunk)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def incore(T, kind, xh, tm, s, method):
    f = T.tcorr_msd if kind == 0 else T.tcorr_acf
    return f(torch.from_numpy(xh).cuda(), tm, s, method).cpu().numpy()


def traj(kind, Tn, N, seed):
    if kind == 0:
        return synth.random_walk_positions(Tn, N, 0.01, 3.0, seed=seed)
    return synth.ou_velocities(Tn, N, 0.1, 1.0, seed=seed)


def check_vs_oracle(kind, got, ref, method):
    if method == "plain":
        if kind == 0:
            assert got[0] == 0.0
            if len(got) > 1:
                assert np.max(np.abs(got[1:] - ref[1:]) / ref[1:]) <= parity.PLAIN_TOL
        else:
            assert np.max(np.abs(got - ref)) / abs(ref[0]) <= parity.PLAIN_TOL
    elif kind == 0 and len(got) == 1:
        assert got[0] == 0.0
    else:
        scale = ref[-1] if kind == 0 else ref[0]
        assert np.max(np.abs(got - ref)) / abs(scale) <= parity.TC_TOL


@pytest.mark.parametrize("method", ["plain", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("Tn,N,tm,s,chunk", [
    (1000, 96, 300, 1, 256),      # four windows, aligned to row tiles
    (1000, 96, 300, 1, 200),      # windows not aligned to 128-origin tiles
    (777, 40, 500, 3, 100),       # stride 3: chunk rounded up to 102; halo longer than a chunk
    (400, 33, 399, 1, 64),        # tau_max = T - 1
    (600, 17, 0, 2, 50),          # lag 0 only
])
def test_stream_matches_oracle(T, method, kind, Tn, N, tm, s, chunk):
    xh = traj(kind, Tn, N, synth.BASE_SEED + Tn + N + s)
    got = streamed(T, kind, xh, tm, s, method, chunk)
    lags = np.arange(tm + 1)
    ref = (oracle.msd if kind == 0 else oracle.acf)(xh, stride=s, lags=lags)
    check_vs_oracle(kind, got, ref, method)


@pytest.mark.parametrize("method", ["plain", "fp16x3"])
def test_stream_equals_incore_when_windows_align(T, method):
    """Windows of whole row tiles.  Plain: the streamed sums regroup the
    in-core ones, so they agree far below the parity tolerance.  Tensor core:
    each window references its own first frame (smaller magnitudes than frame
    0 of the whole run), so the streamed error against the oracle is no larger
    than the in-core one."""
    xh = traj(0, 2048, 256, 11)
    a = streamed(T, 0, xh, 400, 1, method, 512)
    b = incore(T, 0, xh, 400, 1, method)
    assert a[0] == 0.0 and b[0] == 0.0
    if method == "plain":
        assert np.max(np.abs(a[1:] - b[1:]) / b[1:]) <= 1e-9
    else:
        lags = np.array([1, 2, 50, 128, 129, 255, 256, 399, 400])
        ref = oracle.msd(xh, stride=1, lags=lags)
        ea = np.max(np.abs(a[lags] - ref)) / ref[-1]
        eb = np.max(np.abs(b[lags] - ref)) / ref[-1]
        assert ea <= parity.TC_TOL and ea <= 1.5 * eb + 1e-7, (ea, eb)


def test_one_window_and_one_frame_windows(T):
    xh = traj(1, 300, 8, 12)
    whole = streamed(T, 1, xh, 120, 1, "plain", 10 ** 6)          # one window = the in-core call
    ones = streamed(T, 1, xh, 120, 1, "plain", 1)                 # 300 windows of one origin
    ref = oracle.acf(xh, stride=1, lags=np.arange(121))
    check_vs_oracle(1, whole, ref, "plain")
    check_vs_oracle(1, ones, ref, "plain")


def test_pageable_host_memory(T):
    xh = traj(0, 900, 50, 13)
    a = streamed(T, 0, xh, 250, 1, "fp16x3", 256, pinned=False)
    b = streamed(T, 0, xh, 250, 1, "fp16x3", 256, pinned=True)
    assert np.array_equal(a, b)


def test_stream_repeated_calls_share_a_workspace(T):
    """Two calls in a row on one stream with one workspace: the second call's
    copies wait for the first call's kernels."""
    x1, x2 = traj(1, 1500, 64, 14), traj(1, 1500, 64, 15)
    need = T.tcorr_stream_workspace_size(1500, 64, 400, 1, "fp16x3", 300)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    o1 = T.tcorr_acf_stream(host(x1, True), 400, 1, "fp16x3", chunk_frames=300, ws=ws)
    o2 = T.tcorr_acf_stream(host(x2, True), 400, 1, "fp16x3", chunk_frames=300, ws=ws)
    torch.cuda.synchronize()
    for x, o in ((x1, o1), (x2, o2)):
        ref = oracle.acf(x, stride=1, lags=np.arange(401))
        check_vs_oracle(1, o.cpu().numpy(), ref, "fp16x3")
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("method", ["plain", "fp16x3"])
def test_stream_small_last_window_large_k(T, method):
    """N = 8192 (K = 24576), T = 5000, tau_max = 1000, 2048-origin windows: the
    last window holds 512 origins, and its plan splits K into more groups
    than a full window's, so it needs more workspace than the largest window
    (the workspace is the largest over every window shape)."""
    Tn, N, tm = 5000, 8192, 1000
    xh = traj(0, Tn, N, 61)
    got = streamed(T, 0, xh, tm, 1, method, 2048)
    lags = np.array([0, 1, 2, 127, 128, 500, 999, 1000])
    ref = oracle.msd(xh, stride=1, lags=lags)
    check_vs_oracle(0, got[lags], ref, method)


def test_stream_concurrent_with_incore_call_on_another_stream(T):
    """An in-core MSD on one stream while a streamed VACF (more windows than
    window buffers, so buffers are reused) runs on another, the streamed
    call's copies held until the positions' copy has landed: both results
    match the oracle, and the streamed one equals the same call run alone."""
    Tn, N, tm, chunk = 2600, 96, 300, 256
    xh, vh = traj(0, Tn, N, 71), traj(1, Tn, N, 72)
    alone = streamed(T, 1, vh, tm, 1, "fp16x3", chunk)
    xhp, vhp = host(xh, True), host(vh, True)
    xd = torch.empty((Tn, N, 3), dtype=torch.float32, device="cuda")
    sa, sb, sc = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    landed = torch.cuda.Event()
    with torch.cuda.stream(sc):
        xd.copy_(xhp, non_blocking=True)
        landed.record(sc)
    sa.wait_event(landed)
    sb.wait_event(landed)
    m = T.tcorr_msd(xd, tm, 1, "fp16x3", stream=sa)
    c = T.tcorr_acf_stream(vhp, tm, 1, "fp16x3", chunk_frames=chunk, stream=sb)
    # the bindings allocated both workspaces on the current stream and dropped them; fresh
    # allocations there, filled at once, must not get that memory while sa / sb still use it
    junk = [torch.full((T.tcorr_workspace_size(Tn, N, tm, 1, "fp16x3"),), 255, dtype=torch.uint8, device="cuda"),
            torch.full((T.tcorr_stream_workspace_size(Tn, N, tm, 1, "fp16x3", chunk),), 255, dtype=torch.uint8,
                       device="cuda")]
    torch.cuda.synchronize()
    del junk
    lags = np.arange(tm + 1)
    check_vs_oracle(0, m.cpu().numpy(), oracle.msd(xh, stride=1, lags=lags), "fp16x3")
    cc = c.cpu().numpy()
    check_vs_oracle(1, cc, oracle.acf(vh, stride=1, lags=lags), "fp16x3")
    assert np.array_equal(cc, alone)
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("method", ["plain", "fp16x3"])
def test_chunked_host_trajectory_equals_one_array(T, method):
    """A trajectory held as separately pinned frame chunks (boundaries inside windows,
    inside halos, one-frame chunks) streams to the same bits as the one-array call,
    and the chunked calls refuse an empty chunk list before any work."""
    rng = np.random.default_rng(91)
    Tn, N, tm, s, window = 1500, 37, 400, 1, 256
    x = (rng.normal(size=(Tn, N, 3)).cumsum(axis=0) * 0.1).astype(np.float32)
    a = rng.normal(size=(Tn, N, 3)).astype(np.float32)
    cuts = [0, 1, 2, 255, 700, 701, 1234, 1499, Tn]
    for kind, arr in ((0, x), (1, a)):
        whole = streamed(T, kind, arr, tm, s, method, window)
        chunks = [torch.from_numpy(np.ascontiguousarray(arr[c0:c1])).pin_memory()
                  for c0, c1 in zip(cuts[:-1], cuts[1:])]
        f = T.tcorr_msd_stream_chunks if kind == 0 else T.tcorr_acf_stream_chunks
        for _ in range(2):
            got = f(chunks, tm, s, method, window_frames=window)
            torch.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy(), whole), (kind, method)
    with pytest.raises(ValueError):
        T.tcorr_msd_stream_chunks([], tm, s, method)
    assert T.tcorr_status_poll() == 0
