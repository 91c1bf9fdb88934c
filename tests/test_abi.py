"""The C ABI: the library builds, loads, exports every declared symbol, and
rejects bad arguments on the host before any CUDA work (CPU only).

The calls below pass made-up device addresses that are never mapped; they are
safe only because validation rejects every one of them on the host.  So that a
regression in validation can never launch a kernel on such an address, the
checks that use the library run in a child process in which no CUDA device is
visible (CUDA_VISIBLE_DEVICES empty before CUDA starts): a launch that slipped
through would fail there with a CUDA error instead of touching a GPU.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_1708_08619_gb300 import build as tbuild
from paper_1708_08619_gb300 import tcorr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = os.environ.get("TCORR_ABI_CHILD") == "1"


def test_library_checks_in_a_process_without_cuda_devices():
    if CHILD:
        pytest.skip("this is the child process")
    tbuild.build()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", TCORR_ABI_CHILD="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.abspath(__file__), "-q", "-x",
                        "-p", "no:cacheprovider"], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def lib():
    if not CHILD:
        pytest.skip("runs in the child process with no CUDA device visible")
    path = tbuild.build()
    return tcorr.load(path)


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{)]*\)\s*;", text):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("tcorr_msd", "tcorr_acf", "tcorr_batch", "gk_integrate", "einstein_slope",
                 "tcorr_workspace_size", "tcorr_status_poll"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version_and_strerror(lib):
    assert lib.tcorr_version() >= 100
    for code in range(9):
        assert lib.tcorr_strerror(code).startswith(b"TCORR_")


FAKE_X = 0x10000        # never dereferenced: every call below fails validation first
FAKE_OUT = 0x20000
FAKE_WS = 0x30000


def call_msd(lib, x=FAKE_X, T=100, N=10, tau_max=50, s=1, method=0, out=FAKE_OUT,
             ws=FAKE_WS, ws_bytes=0):
    return lib.tcorr_msd(x, T, N, tau_max, s, method, out, ws, ws_bytes, None)


@pytest.mark.parametrize("kw", [
    dict(x=None), dict(out=None), dict(T=0), dict(N=0), dict(tau_max=-1), dict(tau_max=100),
    dict(s=0), dict(method=99), dict(method=-1),
])
def test_invalid_arguments(lib, kw):
    assert call_msd(lib, **kw) == 1   # TCORR_EINVAL


def test_misaligned(lib):
    assert call_msd(lib, x=FAKE_X + 2) == 2
    assert call_msd(lib, out=FAKE_OUT + 4) == 2
    assert call_msd(lib, ws=FAKE_WS + 8) == 2


def test_workspace_too_small(lib):
    need = lib.tcorr_workspace_size(100, 10, 50, 1, 0)
    assert need > 0
    assert call_msd(lib, ws_bytes=need - 1) == 4
    assert lib.tcorr_acf(FAKE_X, 100, 10, 50, 1, 0, FAKE_OUT, None, need, None) == 4


def test_workspace_size_rejects_invalid(lib):
    assert lib.tcorr_workspace_size(0, 10, 0, 1, 0) == 0
    assert lib.tcorr_workspace_size(10, 10, 10, 1, 0) == 0
    assert lib.tcorr_workspace_size(10, 10, 9, 0, 0) == 0
    assert lib.tcorr_workspace_size(10, 10, 9, 1, 42) == 0


def test_workspace_grows_with_the_band(lib):
    a = lib.tcorr_workspace_size(10000, 1000, 100, 1, 0)
    b = lib.tcorr_workspace_size(10000, 1000, 5000, 1, 0)
    assert b > a > 0


def test_gk_and_einstein_validation(lib):
    assert lib.gk_integrate(None, 10, 1.0, 1.0, FAKE_OUT, None) == 1
    assert lib.gk_integrate(FAKE_X, 0, 1.0, 1.0, FAKE_OUT, None) == 1
    assert lib.gk_integrate(FAKE_X + 4, 10, 1.0, 1.0, FAKE_OUT, None) == 2
    assert lib.gk_integrate(FAKE_X, 10, 1.0, 1.0, FAKE_X + 8, None) == 1   # overlap
    gb = lib.gk_integrate_batch
    assert gb(FAKE_X, 10, 0, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 0          # nothing to do
    assert gb(None, 10, 2, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 1
    assert gb(FAKE_X, 0, 2, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 1
    assert gb(FAKE_X, 10, -1, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 1
    assert gb(FAKE_X, 10, 2, 9, 1.0, 1.0, FAKE_OUT, 10, None) == 1           # ldc < n
    assert gb(FAKE_X, 10, 2, 10, 1.0, 1.0, FAKE_OUT, 9, None) == 1           # ldr < n
    assert gb(FAKE_X + 4, 10, 2, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 2
    assert gb(FAKE_X, 10, 3, 10, 1.0, 1.0, FAKE_X + 8 * 25, 10, None) == 1   # spans overlap
    assert gb(FAKE_X, 10, 1 << 60, 10, 1.0, 1.0, FAKE_OUT, 10, None) == 1    # span overflows
    for f in (lib.tcorr_msd_weighted, lib.tcorr_acf_weighted):
        assert f(FAKE_X, None, 100, 10, 50, 1, 0, FAKE_OUT, FAKE_WS, 0, None) == 1          # no weights
        assert f(None, FAKE_X, 100, 10, 50, 1, 0, FAKE_OUT, FAKE_WS, 0, None) == 1
        assert f(FAKE_X, FAKE_X, 100, 10, 100, 1, 0, FAKE_OUT, FAKE_WS, 0, None) == 1       # tau_max >= T
        assert f(FAKE_X, FAKE_X + 2, 100, 10, 50, 1, 0, FAKE_OUT, FAKE_WS, 0, None) == 2    # weights misaligned
        assert f(FAKE_X, FAKE_X, 100, 10, 50, 1, 0, FAKE_OUT, FAKE_WS, 0, None) == 4        # workspace too small
    need = lib.tcorr_weighted_workspace_size(100, 10, 50, 1, 0)
    assert need >= 100 * 10 * 3 * 4 + lib.tcorr_workspace_size(100, 10, 50, 1, 0)
    assert lib.tcorr_weighted_workspace_size(100, 10, 100, 1, 0) == 0
    col = lib.tcorr_collective
    assert col(None, None, 10, 4, -1, FAKE_OUT, None) == 1
    assert col(FAKE_X, None, 10, 4, -1, None, None) == 1
    assert col(FAKE_X, None, 0, 4, -1, FAKE_OUT, None) == 1                # T < 1
    assert col(FAKE_X, None, 10, 0, -1, FAKE_OUT, None) == 1               # N < 1
    assert col(FAKE_X, None, 10, 4, -2, FAKE_OUT, None) == 1               # ref < -1
    assert col(FAKE_X, None, 10, 4, 10, FAKE_OUT, None) == 1               # ref >= T
    assert col(FAKE_X + 2, None, 10, 4, -1, FAKE_OUT, None) == 2
    assert col(FAKE_X, FAKE_OUT + 2, 10, 4, -1, FAKE_OUT + 0x1000, None) == 2
    assert col(FAKE_X, None, 10, 4, -1, FAKE_X + 64, None) == 1            # output inside x
    assert col(FAKE_X, FAKE_OUT, 10, 4, -1, FAKE_OUT + 8, None) == 1       # output over the weights
    D = FAKE_OUT
    assert lib.einstein_slope(FAKE_X, 10, 1.0, 3, 5, 5, D, None) == 1     # hi <= lo
    assert lib.einstein_slope(FAKE_X, 10, 1.0, 3, 2, 10, D, None) == 1    # hi >= n
    assert lib.einstein_slope(FAKE_X, 10, 0.0, 3, 2, 9, D, None) == 1     # dt <= 0
    assert lib.einstein_slope(FAKE_X, 10, 1.0, 0, 2, 9, D, None) == 1     # dim < 1


def test_shard_combine_validation(lib):
    comb = lib.tcorr_combine_shards
    assert comb(None, 10, 2, 11, FAKE_OUT, None) == 1
    assert comb(FAKE_X, 10, 2, 11, None, None) == 1
    assert comb(FAKE_X, 0, 2, 11, FAKE_OUT, None) == 1          # n < 1
    assert comb(FAKE_X, 10, 0, 11, FAKE_OUT, None) == 1         # no rows
    assert comb(FAKE_X, 10, 2, 10, FAKE_OUT, None) == 1         # no room for the weight
    assert comb(FAKE_X + 4, 10, 2, 11, FAKE_OUT, None) == 2
    assert comb(FAKE_X, 10, 2, 11, FAKE_OUT + 4, None) == 2
    assert comb(FAKE_X, 10, 2, 11, FAKE_X + 8 * 12, None) == 1  # output over the rows
    tot = lib.tcorr_weight_total
    assert tot(None, 10, FAKE_OUT, None) == 1
    assert tot(FAKE_X, 0, FAKE_OUT, None) == 1
    assert tot(FAKE_X, 10, None, None) == 1
    assert tot(FAKE_X + 2, 10, FAKE_OUT, None) == 2
    assert tot(FAKE_X, 10, FAKE_OUT + 4, None) == 2


def test_batch_validation(lib):
    inst = (tcorr.TcorrInstance * 2)()
    inst[0] = tcorr.TcorrInstance(0, FAKE_X, 100, 10, 50, 1, FAKE_OUT)
    inst[1] = tcorr.TcorrInstance(2, FAKE_X, 100, 10, 50, 1, FAKE_OUT)   # bad kind
    assert lib.tcorr_batch(inst, 2, 0, FAKE_WS, 1 << 30, None) == 1
    inst[1] = tcorr.TcorrInstance(1, FAKE_X, 100, 10, 100, 1, FAKE_OUT)  # tau_max > T-1
    assert lib.tcorr_batch(inst, 2, 0, FAKE_WS, 1 << 30, None) == 1
    inst[1] = tcorr.TcorrInstance(1, FAKE_X, 100, 10, 99, 1, FAKE_OUT)
    need = lib.tcorr_batch_workspace_size(inst, 2, 0)
    assert need >= lib.tcorr_workspace_size(100, 10, 99, 1, 0)
    assert lib.tcorr_batch(inst, 2, 0, FAKE_WS, need - 1, None) == 4
    assert lib.tcorr_batch(inst, 0, 0, FAKE_WS, need, None) == 1


@pytest.mark.parametrize("bad,code", [
    (dict(kind=-1), 1), (dict(kind=2), 1), (dict(d_x=None), 1), (dict(d_out=None), 1), (dict(T=0), 1),
    (dict(N=-1), 1), (dict(stride=0), 1), (dict(tau_max=-1), 1), (dict(tau_max=100), 1),
    (dict(T=(1 << 40) + 1, tau_max=5), 1), (dict(N=1 << 41), 1), (dict(d_x=FAKE_X + 2), 2),
    (dict(d_out=FAKE_OUT + 4), 2)])
def test_batch_rejects_a_corrupted_descriptor(lib, bad, code):
    """One corrupted entry among valid ones: the whole call is refused on the
    host, before anything is enqueued (the pointers are never dereferenced)."""
    good = dict(kind=0, d_x=FAKE_X, T=100, N=10, tau_max=50, stride=1, d_out=FAKE_OUT)
    inst = (tcorr.TcorrInstance * 3)()
    inst[0] = tcorr.TcorrInstance(**good)
    inst[1] = tcorr.TcorrInstance(**dict(good, **bad))
    inst[2] = tcorr.TcorrInstance(**dict(good, kind=1))
    for method in (0, 4):
        assert lib.tcorr_batch(inst, 3, method, FAKE_WS, 1 << 40, None) == code, (bad, method)


def test_injected_host_allocation_failure_returns_enomem(lib, monkeypatch):
    """TCORR_FAULT_INJECT=host_alloc fails the batch plan's host allocation:
    tcorr_batch returns TCORR_ENOMEM (nothing is enqueued: the pointers here are
    never dereferenced) and the workspace query returns 0."""
    inst = (tcorr.TcorrInstance * 2)()
    inst[0] = tcorr.TcorrInstance(0, FAKE_X, 100, 10, 50, 1, FAKE_OUT)
    inst[1] = tcorr.TcorrInstance(1, FAKE_X, 300, 4, 99, 2, FAKE_OUT + 0x1000)
    need = {m: lib.tcorr_batch_workspace_size(inst, 2, m) for m in (0, 4)}
    assert all(v > 0 for v in need.values())
    monkeypatch.setenv("TCORR_FAULT_INJECT", "host_alloc")
    for m in (0, 4):
        assert lib.tcorr_batch_workspace_size(inst, 2, m) == 0
        assert lib.tcorr_batch(inst, 2, m, FAKE_WS, need[m], None) == 3    # TCORR_ENOMEM
    monkeypatch.delenv("TCORR_FAULT_INJECT")
    assert lib.tcorr_batch_workspace_size(inst, 2, 0) == need[0]


def test_binding_refuses_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    x = torch.zeros((10, 2, 3), dtype=torch.float32)
    with pytest.raises(TypeError):
        tcorr.tcorr_msd(x, 5)


def test_bindings_of_the_added_calls_refuse_bad_tensors(lib):
    """The bindings check their tensors before calling the library (no device needed)."""
    torch = pytest.importorskip("torch")
    x = torch.zeros((10, 2, 3), dtype=torch.float32)
    w = torch.ones(2, dtype=torch.float32)
    c = torch.zeros((3, 10), dtype=torch.float64)
    for call in (lambda: tcorr.tcorr_collective(x),                         # CPU trajectory
                 lambda: tcorr.tcorr_msd_weighted(x, w, 5),
                 lambda: tcorr.tcorr_acf_weighted(x, w, 5),
                 lambda: tcorr.tcorr_xcf(x, x, 5),
                 lambda: tcorr.gk_integrate_batch(c, 1.0),                  # CPU series
                 lambda: tcorr.gk_integrate_batch(c[0], 1.0),               # not 2-D
                 lambda: tcorr.tcorr_msd_stream(x.double(), 5)):            # not float32
        with pytest.raises(TypeError):
            call()


def call_msd_stream(lib, x=FAKE_X, T=100, N=10, tau_max=50, s=1, method=0, chunk=0, out=FAKE_OUT,
                    ws=FAKE_WS, ws_bytes=0):
    return lib.tcorr_msd_stream(x, T, N, tau_max, s, method, chunk, out, ws, ws_bytes, None)


@pytest.mark.parametrize("kw", [
    dict(x=None), dict(out=None), dict(T=0), dict(N=0), dict(tau_max=-1), dict(tau_max=100),
    dict(s=0), dict(method=99), dict(chunk=-1),
])
def test_stream_invalid_arguments(lib, kw):
    assert call_msd_stream(lib, **kw) == 1   # TCORR_EINVAL


def test_stream_misaligned_and_workspace(lib):
    assert call_msd_stream(lib, x=FAKE_X + 2) == 2
    assert call_msd_stream(lib, out=FAKE_OUT + 4) == 2
    assert call_msd_stream(lib, ws=FAKE_WS + 8) == 2
    need = lib.tcorr_stream_workspace_size(100, 10, 50, 1, 0, 32)
    assert need > 0
    assert call_msd_stream(lib, chunk=32, ws_bytes=need - 1) == 4


def test_stream_workspace_holds_three_windows(lib):
    T, N, tm = 5000, 64, 300
    small = lib.tcorr_stream_workspace_size(T, N, tm, 1, 0, 512)
    big = lib.tcorr_stream_workspace_size(T, N, tm, 1, 0, 2048)
    assert 3 * (512 + tm) * N * 3 * 4 <= small < big
    # a chunk covering the whole trajectory is one window (one buffer) of T frames
    whole = lib.tcorr_stream_workspace_size(T, N, tm, 1, 0, 10 ** 9)
    assert T * N * 3 * 4 <= whole < 2 * T * N * 3 * 4 + lib.tcorr_workspace_size(T, N, tm, 1, 0)
    assert lib.tcorr_stream_workspace_size(T, N, tm, 1, 0, -1) == 0


def call_msd_stream_chunks(lib, ptrs=(FAKE_X, FAKE_X + 0x10000), frames=(60, 40), n=None, N=10, tau_max=50, s=1,
                           method=0, window=0, out=FAKE_OUT, ws=FAKE_WS, ws_bytes=0, null=None):
    n = len(ptrs) if n is None else n
    P = (ctypes.c_void_p * max(1, len(ptrs)))(*ptrs)
    F = (ctypes.c_int64 * max(1, len(frames)))(*frames)
    pa = None if null == "ptrs" else ctypes.cast(P, ctypes.c_void_p)
    fa = None if null == "frames" else ctypes.cast(F, ctypes.c_void_p)
    return lib.tcorr_msd_stream_chunks(pa, fa, n, N, tau_max, s, method, window, out, ws, ws_bytes, None)


@pytest.mark.parametrize("kw", [
    dict(null="ptrs"), dict(null="frames"), dict(n=0), dict(frames=(60, 0)), dict(ptrs=(FAKE_X, None)),
    dict(out=None), dict(tau_max=100), dict(N=0), dict(s=0), dict(method=99), dict(window=-1),
])
def test_stream_chunks_invalid_arguments(lib, kw):
    assert call_msd_stream_chunks(lib, **kw) == 1   # TCORR_EINVAL


def test_stream_chunks_misaligned_and_workspace(lib):
    assert call_msd_stream_chunks(lib, ptrs=(FAKE_X, FAKE_X + 0x10002)) == 2
    assert call_msd_stream_chunks(lib, out=FAKE_OUT + 4) == 2
    need = lib.tcorr_stream_workspace_size(100, 10, 50, 1, 0, 32)      # T = the chunks' total
    assert need > 0
    assert call_msd_stream_chunks(lib, window=32, ws_bytes=need - 1) == 4


def call_xcf(lib, a=FAKE_X, b=FAKE_X + 0x1000, T=100, N=10, tau_max=50, s=1, method=0, out=FAKE_OUT,
             ws=FAKE_WS, ws_bytes=0):
    return lib.tcorr_xcf(a, b, T, N, tau_max, s, method, out, ws, ws_bytes, None)


@pytest.mark.parametrize("kw", [
    dict(a=None), dict(b=None), dict(out=None), dict(T=0), dict(N=0), dict(tau_max=100), dict(s=0),
    dict(method=99),
])
def test_xcf_invalid_arguments(lib, kw):
    assert call_xcf(lib, **kw) == 1


def test_xcf_misaligned_and_workspace(lib):
    assert call_xcf(lib, a=FAKE_X + 2) == 2
    assert call_xcf(lib, b=FAKE_X + 0x1000 + 1) == 2
    assert call_xcf(lib, out=FAKE_OUT + 4) == 2
    need = lib.tcorr_xcf_workspace_size(100, 10, 50, 1, 0)
    assert need > 0
    assert call_xcf(lib, ws_bytes=need - 1) == 4


def test_fft_method_is_known(lib):
    """Method 6 (FFT route) passes argument validation; its workspace size is
    host arithmetic (the route's own transforms, no plan on a device), and a
    padded length beyond the route's 2^23 gives 0."""
    assert tcorr.METHODS["fft"] == 6
    need = lib.tcorr_workspace_size(1000, 64, 999, 1, 6)
    assert need >= 32 * 2048 * 16                   # 32 complex rows of the padded length
    assert lib.tcorr_workspace_size(5000000, 1, 4000000, 1, 6) == 0
    assert lib.tcorr_workspace_size(4000000, 1, 4000000 - 1, 1, 6) > 0
    assert call_msd(lib, T=5000000, N=1, tau_max=4000000, method=6) == 7   # TCORR_EUNSUPPORTED
