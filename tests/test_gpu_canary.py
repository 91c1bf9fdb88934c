"""Canary words around the caller's buffers (GPU): every call writes only
inside the workspace size it asked for and the tau_max + 1 outputs, and never
writes its inputs.  Each buffer is allocated with a guard region filled with a
known byte pattern; after the call (and a device synchronise) the guards, and
the inputs, must be unchanged, for every method and path."""
import numpy as np
import pytest

from paper_1708_08619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 1 << 16          # bytes of canary after each buffer
PAT = 0xA5


@pytest.fixture(scope="module")
def T():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    tcorr.load()
    return tcorr


def guarded_ws(nbytes):
    buf = torch.full((nbytes + GUARD,), PAT, dtype=torch.uint8, device="cuda")
    return buf, buf[:nbytes] if nbytes else None


def guarded_out(n):
    buf = torch.full((n + GUARD // 8,), 12345.5, dtype=torch.float64, device="cuda")
    return buf, buf[:n]


def check_guards(ws_buf, nbytes, out_buf, n, what):
    torch.cuda.synchronize()
    assert bool((ws_buf[nbytes:] == PAT).all()), f"{what}: workspace written past its {nbytes} bytes"
    assert bool((out_buf[n:] == 12345.5).all()), f"{what}: output written past its {n} values"
    assert bool(torch.isfinite(out_buf[:n]).all()), f"{what}: output not written"


SHAPES = [(700, 50, 400, 1), (900, 33, 500, 3), (5000, 1, 1200, 1), (300, 200, 299, 7)]


@pytest.mark.parametrize("method", ["plain", "fp16x3", "tf32x3", "bf16x4", "bf16x3", "fft"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "T%d_N%d_tm%d_s%d" % s)
def test_correlation_calls_stay_inside_their_buffers(T, method, shape):
    Tn, N, tm, s = shape
    x = torch.from_numpy(synth.random_walk_positions(Tn, N, 0.02, 3.0, seed=Tn + N)).cuda()
    x0 = x.clone()
    for name, f, wsize in (("msd", T.tcorr_msd, T.tcorr_workspace_size),
                           ("acf", T.tcorr_acf, T.tcorr_workspace_size)):
        need = wsize(Tn, N, tm, s, method)
        ws_buf, ws = guarded_ws(need)
        out_buf, out = guarded_out(tm + 1)
        f(x, tm, s, method, out=out, ws=ws)
        check_guards(ws_buf, need, out_buf, tm + 1, f"{name} {method} {shape}")
    y = torch.from_numpy(synth.ou_velocities(Tn, N, 0.1, 1.0, seed=Tn + N + 1)).cuda()
    need = T.tcorr_xcf_workspace_size(Tn, N, tm, s, method)
    ws_buf, ws = guarded_ws(need)
    out_buf, out = guarded_out(tm + 1)
    T.tcorr_xcf(x, y, tm, s, method, out=out, ws=ws)
    check_guards(ws_buf, need, out_buf, tm + 1, f"xcf {method} {shape}")
    w = torch.rand(N, dtype=torch.float32, device="cuda") + 0.5
    need = T.tcorr_weighted_workspace_size(Tn, N, tm, s, method)
    ws_buf, ws = guarded_ws(need)
    out_buf, out = guarded_out(tm + 1)
    T.tcorr_msd_weighted(x, w, tm, s, method, out=out, ws=ws)
    check_guards(ws_buf, need, out_buf, tm + 1, f"weighted msd {method} {shape}")
    assert torch.equal(x, x0), "an input was written"
    assert T.tcorr_status_poll() == 0


@pytest.mark.parametrize("method", ["plain", "fp16x3"])
def test_batch_and_stream_stay_inside_their_buffers(T, method):
    rng = np.random.default_rng(5)
    xs, outs, bufs = [], [], []
    for i in range(7):
        Tn = int(rng.integers(100, 3000))
        N = int(rng.integers(1, 300))
        tm = Tn // 4
        xs.append(torch.from_numpy(synth.random_walk_positions(Tn, N, 0.02, 3.0, seed=50 + i)).cuda())
        ob, o = guarded_out(tm + 1)
        outs.append(o)
        bufs.append((ob, tm + 1))
    items = [(i % 2, x, x.shape[0] // 4, 1, o) for i, (x, o) in enumerate(zip(xs, outs))]
    inst = T.make_instances(items)
    need = T.tcorr_batch_workspace_size(inst, method)
    ws_buf, ws = guarded_ws(need)
    T.tcorr_batch(inst, method, ws=ws)
    for ob, n in bufs:
        check_guards(ws_buf, need, ob, n, f"batch {method}")
    xh = torch.from_numpy(synth.random_walk_positions(4000, 60, 0.02, 3.0, seed=77)).pin_memory()
    need = T.tcorr_stream_workspace_size(4000, 60, 700, 1, method, 512)
    ws_buf, ws = guarded_ws(need)
    out_buf, out = guarded_out(701)
    T.tcorr_msd_stream(xh, 700, 1, method, chunk_frames=512, out=out, ws=ws)
    check_guards(ws_buf, need, out_buf, 701, f"stream {method}")
    assert T.tcorr_status_poll() == 0


def test_batch_with_an_injected_host_allocation_failure_writes_nothing(T, monkeypatch):
    """With TCORR_FAULT_INJECT=host_alloc tcorr_batch returns TCORR_ENOMEM and
    nothing reaches the GPU: the outputs and the workspace keep their canary
    bytes; without it the same call runs."""
    xs = [torch.from_numpy(synth.random_walk_positions(500 + 100 * i, 20, 0.02, 3.0, seed=i)).cuda()
          for i in range(3)]
    outs = [torch.full((x.shape[0] // 4 + 1,), 12345.5, dtype=torch.float64, device="cuda") for x in xs]
    inst = T.make_instances([(i % 2, x, x.shape[0] // 4, 1, o) for i, (x, o) in enumerate(zip(xs, outs))])
    for method in ("plain", "fp16x3"):
        need = T.tcorr_batch_workspace_size(inst, method)
        ws = torch.full((need,), PAT, dtype=torch.uint8, device="cuda")
        monkeypatch.setenv("TCORR_FAULT_INJECT", "host_alloc")
        with pytest.raises(T.TcorrError) as ei:
            T.tcorr_batch(inst, method, ws=ws)
        assert ei.value.code == 3
        torch.cuda.synchronize()
        assert bool((ws == PAT).all()) and all(bool((o == 12345.5).all()) for o in outs)
        monkeypatch.delenv("TCORR_FAULT_INJECT")
        T.tcorr_batch(inst, method, ws=ws)
        torch.cuda.synchronize()
        assert all(bool(torch.isfinite(o).all()) and not bool((o == 12345.5).any()) for o in outs)
        for o in outs:
            o.fill_(12345.5)
