"""The debug build (libtcorr_debug.so, TCORR_DEBUG_BOUNDS) on the GPU.

Its kernels check the global-memory indices of the plain path, the lag
reduction and the band kernel's window stores against their buffers' extents
and report a bad index as TCORR_EBOUNDS in the status word, skipping the
access, instead of faulting.  Checked here: on valid calls it gives the release
library's results bit for bit with a clean status word; with
TCORR_DEBUG_SHRINK=1 (every partial-sum buffer declared one window shorter
than it really is, the real buffer intact) the checks fire, the status word
reads TCORR_EBOUNDS, and the context stays usable."""
import ctypes

import numpy as np
import pytest

from paper_1708_08619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TCORR_EBOUNDS = 8


@pytest.fixture(scope="module")
def libs():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rel = tcorr.load(build.build())
    dbg = tcorr.load(build.build(debug=True))
    return rel, dbg


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _run(lib, kind, x, tau_max, stride, method):
    T, N = x.shape[0], x.shape[1]
    need = lib.tcorr_workspace_size(T, N, tau_max, stride, method)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    out = torch.full((tau_max + 1,), float("nan"), dtype=torch.float64, device="cuda")
    f = lib.tcorr_msd if kind == 0 else lib.tcorr_acf
    rc = f(x.data_ptr(), T, N, tau_max, stride, method, out.data_ptr(), ws.data_ptr(), need, _stream())
    assert rc == 0, rc
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [(600, 40, 300, 1), (500, 17, 499, 3), (900, 100, 200, 2)]


@pytest.mark.parametrize("method", [0, 4])          # plain, FP16x3 band kernel
def test_debug_build_matches_release_and_stays_clean(libs, method):
    rel, dbg = libs
    for T, N, tm, s in CASES:
        x = torch.from_numpy(synth.random_walk_positions(T, N, 0.02, 3.0, seed=T + N)).cuda()
        for kind in (0, 1):
            a = _run(rel, kind, x, tm, s, method)
            b = _run(dbg, kind, x, tm, s, method)
            assert np.array_equal(a, b), (method, kind, T, N, tm, s)
    assert dbg.tcorr_status_poll(_stream()) == 0
    assert rel.tcorr_status_poll(_stream()) == 0


@pytest.mark.parametrize("method", [0, 4])
def test_shrunk_extents_are_reported_not_faulted(libs, method, monkeypatch):
    rel, dbg = libs
    x = torch.from_numpy(synth.random_walk_positions(600, 40, 0.02, 3.0, seed=9)).cuda()
    assert dbg.tcorr_status_poll(_stream()) == 0
    monkeypatch.setenv("TCORR_DEBUG_SHRINK", "1")
    _run(dbg, 0, x, 300, 1, method)
    assert dbg.tcorr_status_poll(_stream()) == TCORR_EBOUNDS
    assert dbg.tcorr_status_poll(_stream()) == 0             # reported once, then cleared
    monkeypatch.delenv("TCORR_DEBUG_SHRINK")
    # the context is still usable and the results are right again
    assert np.array_equal(_run(dbg, 0, x, 300, 1, method), _run(rel, 0, x, 300, 1, method))
    assert dbg.tcorr_status_poll(_stream()) == 0
