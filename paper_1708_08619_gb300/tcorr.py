"""Python binding of libtcorr.so (argument marshalling only).

Every function here has the name of the C entry point it calls
(``include/tcorr.h``).  Tensors are torch tensors; the binding passes their
device pointers, allocates outputs and workspace with torch when the caller
gives none, and passes torch's current CUDA stream.  All arithmetic of the
path runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or the tensors are not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os

PLAIN, TC_TF32X3, TC_BF16X3, TC_BF16X4, TC_FP16X3, AUTO, FFT = range(7)
METHODS = {"plain": PLAIN, "tf32x3": TC_TF32X3, "bf16x3": TC_BF16X3, "bf16x4": TC_BF16X4,
           "fp16x3": TC_FP16X3, "auto": AUTO, "fft": FFT}
STATUS = {0: "TCORR_OK", 1: "TCORR_EINVAL", 2: "TCORR_EALIGN", 3: "TCORR_ENOMEM",
          4: "TCORR_EWORKSPACE", 5: "TCORR_ECUDA", 6: "TCORR_ETIMEOUT", 7: "TCORR_EUNSUPPORTED",
          8: "TCORR_EBOUNDS"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtcorr.so")
_lib = None


class TcorrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class TcorrInstance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d_x", ctypes.c_void_p), ("T", ctypes.c_int64),
                ("N", ctypes.c_int64), ("tau_max", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("d_out", ctypes.c_void_p)]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Open libtcorr.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1708_08619_gb300.build.build()")
    lib = ctypes.CDLL(path)
    i64, vp, dbl, ci, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    lib.tcorr_workspace_size.argtypes = [i64, i64, i64, i64, ci]
    lib.tcorr_workspace_size.restype = sz
    for name in ("tcorr_msd", "tcorr_acf"):
        f = getattr(lib, name)
        f.argtypes = [vp, i64, i64, i64, i64, ci, vp, vp, sz, vp]
        f.restype = ci
    lib.tcorr_xcf_workspace_size.argtypes = [i64, i64, i64, i64, ci]
    lib.tcorr_xcf_workspace_size.restype = sz
    lib.tcorr_xcf.argtypes = [vp, vp, i64, i64, i64, i64, ci, vp, vp, sz, vp]
    lib.tcorr_xcf.restype = ci
    lib.gk_integrate.argtypes = [vp, i64, dbl, dbl, vp, vp]
    lib.gk_integrate.restype = ci
    lib.gk_integrate_batch.argtypes = [vp, i64, i64, i64, dbl, dbl, vp, i64, vp]
    lib.gk_integrate_batch.restype = ci
    lib.tcorr_collective.argtypes = [vp, vp, i64, i64, i64, vp, vp]
    lib.tcorr_collective.restype = ci
    lib.tcorr_weighted_workspace_size.argtypes = [i64, i64, i64, i64, ci]
    lib.tcorr_weighted_workspace_size.restype = sz
    for name in ("tcorr_msd_weighted", "tcorr_acf_weighted"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, i64, i64, i64, i64, ci, vp, vp, sz, vp]
        f.restype = ci
    lib.tcorr_combine_shards.argtypes = [vp, i64, i64, i64, vp, vp]
    lib.tcorr_combine_shards.restype = ci
    lib.tcorr_weight_total.argtypes = [vp, i64, vp, vp]
    lib.tcorr_weight_total.restype = ci
    lib.einstein_slope.argtypes = [vp, i64, dbl, ci, i64, i64, vp, vp]
    lib.einstein_slope.restype = ci
    lib.tcorr_batch_workspace_size.argtypes = [ctypes.POINTER(TcorrInstance), ci, ci]
    lib.tcorr_batch_workspace_size.restype = sz
    lib.tcorr_batch.argtypes = [ctypes.POINTER(TcorrInstance), ci, ci, vp, sz, vp]
    lib.tcorr_batch.restype = ci
    lib.tcorr_stream_workspace_size.argtypes = [i64, i64, i64, i64, ci, i64]
    lib.tcorr_stream_workspace_size.restype = sz
    for name in ("tcorr_msd_stream", "tcorr_acf_stream"):
        f = getattr(lib, name)
        f.argtypes = [vp, i64, i64, i64, i64, ci, i64, vp, vp, sz, vp]
        f.restype = ci
    for name in ("tcorr_msd_stream_chunks", "tcorr_acf_stream_chunks"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, ci, i64, i64, i64, ci, i64, vp, vp, sz, vp]
        f.restype = ci
    lib.tcorr_plain_static.argtypes = [ci, vp, i64, i64, i64, i64, vp, vp]
    lib.tcorr_plain_static.restype = ci
    lib.tcorr_profile_enable.argtypes = [ci]
    lib.tcorr_profile_enable.restype = ci
    lib.tcorr_profile_read.argtypes = [ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.tcorr_profile_read.restype = ci
    lib.tcorr_selftest_timeout.argtypes = [vp]
    lib.tcorr_selftest_timeout.restype = ci
    lib.tcorr_status_poll.argtypes = [vp]
    lib.tcorr_status_poll.restype = ci
    lib.tcorr_strerror.argtypes = [ci]
    lib.tcorr_strerror.restype = ctypes.c_char_p
    lib.tcorr_version.argtypes = []
    lib.tcorr_version.restype = ci
    if path == LIB_PATH:
        _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _method(m) -> int:
    return METHODS[m] if isinstance(m, str) else int(m)


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_traj(x):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("x must be a CUDA torch tensor")
    if x.dtype != torch.float32 or x.dim() != 3 or x.shape[2] != 3 or not x.is_contiguous():
        raise TypeError("x must be a contiguous float32 tensor of shape [T][N][3]")


def _check_out(out, n: int, device, dtype_name: str = "float64"):
    """A caller's output tensor: contiguous, of the result's dtype, on the input's
    device, with room for n values; raises TypeError before any library call."""
    torch = _torch()
    dtype = getattr(torch, dtype_name)
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.device != torch.device(device):
        raise TypeError("out must be a CUDA tensor on the input's device")
    if out.dtype != dtype or not out.is_contiguous() or out.numel() < n:
        raise TypeError(f"out must be a contiguous {dtype_name} tensor of at least {n} values")
    return out


def _check_ws(ws, device):
    torch = _torch()
    if ws is not None and (not isinstance(ws, torch.Tensor) or not ws.is_cuda
                           or ws.device != torch.device(device) or not ws.is_contiguous()):
        raise TypeError("ws must be a contiguous CUDA tensor on the input's device")
    return ws


def tcorr_workspace_size(T: int, N: int, tau_max: int, stride: int = 1, method=AUTO) -> int:
    return int(load().tcorr_workspace_size(T, N, tau_max, stride, _method(method)))


def _alloc_ws(nbytes: int, device):
    torch = _torch()
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _held_by(t, stream):
    """A tensor allocated here for a call on ``stream``: torch's caching allocator
    allocated it on the current stream, so it is marked as used by ``stream`` too;
    otherwise its memory could go to another allocation as soon as the binding
    drops it, while the call's kernels still run."""
    if t is not None and stream is not None:
        t.record_stream(stream)
    return t


def _corr(fname: str, x, tau_max: int, stride: int, method, out, ws, stream):
    torch = _torch()
    _check_traj(x)
    T, N, _ = x.shape
    m = _method(method)
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=x.device), stream)
    _check_out(out, tau_max + 1, x.device)
    _check_ws(ws, x.device)
    need = tcorr_workspace_size(T, N, tau_max, stride, m)
    if ws is None:
        ws = _held_by(_alloc_ws(need, x.device), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = getattr(load(), fname)(x.data_ptr(), T, N, tau_max, stride, m, out.data_ptr(),
                                ws_ptr, ws_bytes, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, fname)
    return out


def tcorr_msd(x, tau_max: int, stride: int = 1, method=AUTO, out=None, ws=None, stream=None):
    """MSD(tau), tau = 0..tau_max, of x[T][N][3] (Eq. 5); returns a float64 tensor."""
    return _corr("tcorr_msd", x, tau_max, stride, method, out, ws, stream)


def tcorr_acf(x, tau_max: int, stride: int = 1, method=AUTO, out=None, ws=None, stream=None):
    """<A(t0).A(t0+tau)>, tau = 0..tau_max, of A[T][N][3] (Eq. 4 integrand)."""
    return _corr("tcorr_acf", x, tau_max, stride, method, out, ws, stream)


def tcorr_xcf_workspace_size(T: int, N: int, tau_max: int, stride: int = 1, method=AUTO) -> int:
    return int(load().tcorr_xcf_workspace_size(T, N, tau_max, stride, _method(method)))


def tcorr_xcf(a, b, tau_max: int, stride: int = 1, method=AUTO, out=None, ws=None, stream=None):
    """<A(t0).B(t0+tau)>, tau = 0..tau_max, of A and B [T][N][3] (same shape)."""
    torch = _torch()
    _check_traj(a)
    _check_traj(b)
    if a.shape != b.shape:
        raise TypeError("a and b must have the same shape")
    T, N, _ = a.shape
    m = _method(method)
    if a.device != b.device:
        raise TypeError("a and b must be on the same device")
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=a.device), stream)
    _check_out(out, tau_max + 1, a.device)
    _check_ws(ws, a.device)
    need = tcorr_xcf_workspace_size(T, N, tau_max, stride, m)
    if ws is None:
        ws = _held_by(_alloc_ws(need, a.device), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = load().tcorr_xcf(a.data_ptr(), b.data_ptr(), T, N, tau_max, stride, m, out.data_ptr(), ws_ptr, ws_bytes,
                          _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_xcf")
    return out


def gk_integrate(c, dt: float, prefactor: float = 1.0, out=None, stream=None):
    """Running trapezoid integral prefactor * int_0^tau C dt (Eq. 4)."""
    torch = _torch()
    if not c.is_cuda or c.dtype != torch.float64 or not c.is_contiguous():
        raise TypeError("c must be a contiguous float64 CUDA tensor")
    if out is None:
        out = _held_by(torch.empty_like(c), stream)
    _check_out(out, c.numel(), c.device)
    rc = load().gk_integrate(c.data_ptr(), c.numel(), dt, prefactor, out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "gk_integrate")
    return out


def gk_integrate_batch(c, dt: float, prefactor: float = 1.0, out=None, stream=None):
    """gk_integrate of every row of a [count][n] float64 CUDA tensor, one launch.

    Rows may be padded (row stride >= n, unit column stride); out gets the
    same shape (a new contiguous tensor by default).
    """
    torch = _torch()
    if not c.is_cuda or c.dtype != torch.float64 or c.dim() != 2 or c.stride(1) != 1:
        raise TypeError("c must be a [count][n] float64 CUDA tensor with unit column stride")
    if out is None:
        out = _held_by(torch.empty(c.shape, dtype=torch.float64, device=c.device), stream)
    if tuple(out.shape) != tuple(c.shape) or out.dtype != torch.float64 or out.stride(1) != 1:
        raise TypeError("out must be a float64 tensor shaped like c with unit column stride")
    count, n = c.shape
    rc = load().gk_integrate_batch(c.data_ptr(), n, count, c.stride(0) if count > 1 else n, dt, prefactor,
                                   out.data_ptr(), out.stride(0) if count > 1 else n, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "gk_integrate_batch")
    return out


def tcorr_weighted_workspace_size(T: int, N: int, tau_max: int, stride: int = 1, method=AUTO) -> int:
    return int(load().tcorr_weighted_workspace_size(T, N, tau_max, stride, _method(method)))


def _corr_weighted(fname: str, x, w, tau_max: int, stride: int, method, out, ws, stream):
    torch = _torch()
    _check_traj(x)
    T, N, _ = x.shape
    if not isinstance(w, torch.Tensor) or not w.is_cuda or w.dtype != torch.float32 or w.numel() != N \
            or not w.is_contiguous():
        raise TypeError("w must be a contiguous float32 CUDA tensor with one weight per atom")
    m = _method(method)
    if w.device != x.device:
        raise TypeError("w must be on the trajectory's device")
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=x.device), stream)
    _check_out(out, tau_max + 1, x.device)
    _check_ws(ws, x.device)
    need = tcorr_weighted_workspace_size(T, N, tau_max, stride, m)
    if ws is None:
        ws = _held_by(_alloc_ws(need, x.device), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = getattr(load(), fname)(x.data_ptr(), w.data_ptr(), T, N, tau_max, stride, m, out.data_ptr(),
                                ws_ptr, ws_bytes, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, fname)
    return out


def tcorr_msd_weighted(x, w, tau_max: int, stride: int = 1, method=AUTO, out=None, ws=None, stream=None):
    """MSD with atom i counted w[i] times (w >= 0): sum_i w_i (...) / (sum_i w_i n_o(tau))."""
    return _corr_weighted("tcorr_msd_weighted", x, w, tau_max, stride, method, out, ws, stream)


def tcorr_acf_weighted(x, w, tau_max: int, stride: int = 1, method=AUTO, out=None, ws=None, stream=None):
    """Autocorrelation with atom i counted w[i] times (w >= 0)."""
    return _corr_weighted("tcorr_acf_weighted", x, w, tau_max, stride, method, out, ws, stream)


def tcorr_collective(x, w=None, ref_frame: int = -1, out=None, stream=None):
    """sum_i w_i (x[t][i] - x[ref_frame][i]) per frame as a [T][1][3] float32 trajectory
    (ref_frame -1: no reference; w None: unit weights)."""
    torch = _torch()
    _check_traj(x)
    T, N, _ = x.shape
    if w is not None and (not w.is_cuda or w.dtype != torch.float32 or w.numel() != N or not w.is_contiguous()):
        raise TypeError("w must be a contiguous float32 CUDA tensor with one weight per atom")
    if w is not None and w.device != x.device:
        raise TypeError("w must be on the trajectory's device")
    if out is None:
        out = _held_by(torch.empty((T, 1, 3), dtype=torch.float32, device=x.device), stream)
    _check_out(out, 3 * T, x.device, "float32")
    rc = load().tcorr_collective(x.data_ptr(), w.data_ptr() if w is not None else None, T, N, ref_frame,
                                 out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_collective")
    return out


def tcorr_combine_shards(rows, n: int, out=None, stream=None):
    """Average over all atoms from gathered shard records: rows is a [count][ld]
    float64 CUDA tensor (unit column stride, ld >= n + 1) whose row r holds
    shard r's n per-lag averages followed by its weight (atom count or weight
    sum); returns sum_r w_r rows[r][:n] / sum_r w_r (FP64, rows in order)."""
    torch = _torch()
    if not isinstance(rows, torch.Tensor) or not rows.is_cuda or rows.dtype != torch.float64 \
            or rows.dim() != 2 or rows.stride(1) != 1:
        raise TypeError("rows must be a [count][ld] float64 CUDA tensor with unit column stride")
    count = rows.shape[0]
    ld = rows.stride(0) if count > 1 else rows.shape[1]
    if rows.shape[1] < n + 1:
        raise TypeError("each row needs n values and a weight")
    if out is None:
        out = _held_by(torch.empty(n, dtype=torch.float64, device=rows.device), stream)
    _check_out(out, n, rows.device)
    rc = load().tcorr_combine_shards(rows.data_ptr(), n, count, ld, out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_combine_shards")
    return out


def tcorr_weight_total(w, out=None, stream=None):
    """sum_i w_i of a float32 CUDA weight vector in FP64 (fixed order); out: one
    double on the device (a new one by default, or a view into a record)."""
    torch = _torch()
    if not isinstance(w, torch.Tensor) or not w.is_cuda or w.dtype != torch.float32 or not w.is_contiguous():
        raise TypeError("w must be a contiguous float32 CUDA tensor")
    if out is None:
        out = _held_by(torch.empty(1, dtype=torch.float64, device=w.device), stream)
    _check_out(out, 1, w.device)
    rc = load().tcorr_weight_total(w.data_ptr(), w.numel(), out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_weight_total")
    return out


def einstein_slope(msd, dt: float, dim: int = 3, lo: int | None = None, hi: int | None = None,
                   out=None, stream=None):
    """[D from the least-squares slope over [lo, hi], D from the ratio at hi] (Eq. 5)."""
    torch = _torch()
    if not msd.is_cuda or msd.dtype != torch.float64 or not msd.is_contiguous():
        raise TypeError("msd must be a contiguous float64 CUDA tensor")
    n = msd.numel()
    if hi is None:
        hi = n - 1
    if lo is None:
        lo = -(-(2 * hi) // 10)
    if out is None:
        out = _held_by(torch.empty(2, dtype=torch.float64, device=msd.device), stream)
    _check_out(out, 2, msd.device)
    rc = load().einstein_slope(msd.data_ptr(), n, dt, dim, lo, hi, out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "einstein_slope")
    return out


def make_instances(items):
    """items: iterable of (kind, x, tau_max, stride, out) -> ctypes array."""
    items = list(items)
    arr = (TcorrInstance * len(items))()
    for i, (kind, x, tau_max, stride, out) in enumerate(items):
        _check_traj(x)
        arr[i] = TcorrInstance(kind, x.data_ptr(), x.shape[0], x.shape[1], tau_max, stride,
                               out.data_ptr())
    return arr


def tcorr_batch_workspace_size(instances, method=AUTO) -> int:
    return int(load().tcorr_batch_workspace_size(instances, len(instances), _method(method)))


def tcorr_batch(instances, method=AUTO, ws=None, stream=None, device=None):
    """Run every instance of a ``make_instances`` array; outputs are written in place."""
    torch = _torch()
    m = _method(method)
    need = tcorr_batch_workspace_size(instances, m)
    if ws is None:
        ws = _held_by(_alloc_ws(need, device or torch.device("cuda")), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = load().tcorr_batch(instances, len(instances), m, ws_ptr, ws_bytes, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_batch")


def tcorr_stream_workspace_size(T: int, N: int, tau_max: int, stride: int = 1, method=AUTO,
                                chunk_frames: int = 0) -> int:
    return int(load().tcorr_stream_workspace_size(T, N, tau_max, stride, _method(method), chunk_frames))


def _corr_stream(fname: str, x, tau_max: int, stride: int, method, chunk_frames: int, out, ws, stream, device):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.is_cuda:
        raise TypeError("x must be a host (CPU) torch tensor; pin it for overlapped copies")
    if x.dtype != torch.float32 or x.dim() != 3 or x.shape[2] != 3 or not x.is_contiguous():
        raise TypeError("x must be a contiguous float32 tensor of shape [T][N][3]")
    T, N, _ = x.shape
    m = _method(method)
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=device), stream)
    _check_out(out, tau_max + 1, device)
    _check_ws(ws, device)
    need = tcorr_stream_workspace_size(T, N, tau_max, stride, m, chunk_frames)
    if ws is None:
        ws = _held_by(_alloc_ws(need, device), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = getattr(load(), fname)(x.data_ptr(), T, N, tau_max, stride, m, chunk_frames, out.data_ptr(),
                                ws_ptr, ws_bytes, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, fname)
    return out


def tcorr_msd_stream(x, tau_max: int, stride: int = 1, method=AUTO, chunk_frames: int = 0, out=None, ws=None,
                     stream=None, device=None):
    """MSD of a host-resident x[T][N][3] streamed through the device in windows
    of chunk_frames origins (0: library default); result on the device."""
    return _corr_stream("tcorr_msd_stream", x, tau_max, stride, method, chunk_frames, out, ws, stream, device)


def tcorr_acf_stream(x, tau_max: int, stride: int = 1, method=AUTO, chunk_frames: int = 0, out=None, ws=None,
                     stream=None, device=None):
    """Autocorrelation of a host-resident A[T][N][3], streamed as tcorr_msd_stream."""
    return _corr_stream("tcorr_acf_stream", x, tau_max, stride, method, chunk_frames, out, ws, stream, device)


def _corr_stream_chunks(fname: str, chunks, tau_max: int, stride: int, method, window_frames: int, out, ws,
                        stream, device):
    torch = _torch()
    chunks = list(chunks)
    if not chunks:
        raise ValueError("chunks: at least one host tensor")
    N = None
    for c in chunks:
        if not isinstance(c, torch.Tensor) or c.is_cuda:
            raise TypeError("every chunk must be a host (CPU) torch tensor; pin each for overlapped copies")
        if c.dtype != torch.float32 or c.dim() != 3 or c.shape[2] != 3 or not c.is_contiguous():
            raise TypeError("every chunk must be a contiguous float32 tensor of shape [frames][N][3]")
        if N is None:
            N = c.shape[1]
        elif c.shape[1] != N:
            raise ValueError("chunks hold different atom counts")
    T = sum(c.shape[0] for c in chunks)
    m = _method(method)
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=device), stream)
    _check_out(out, tau_max + 1, device)
    _check_ws(ws, device)
    need = tcorr_stream_workspace_size(T, N, tau_max, stride, m, window_frames)
    if ws is None:
        ws = _held_by(_alloc_ws(need, device), stream)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    ptrs = (ctypes.c_void_p * len(chunks))(*[c.data_ptr() for c in chunks])
    frames = (ctypes.c_int64 * len(chunks))(*[c.shape[0] for c in chunks])
    rc = getattr(load(), fname)(ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(frames, ctypes.c_void_p),
                                len(chunks), N, tau_max, stride, m, window_frames, out.data_ptr(), ws_ptr,
                                ws_bytes, _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, fname)
    return out


def tcorr_msd_stream_chunks(chunks, tau_max: int, stride: int = 1, method=AUTO, window_frames: int = 0, out=None,
                            ws=None, stream=None, device=None):
    """MSD of a host-resident trajectory given as consecutive frame chunks (host tensors
    [frames][N][3], e.g. each pinned on its own), streamed as tcorr_msd_stream."""
    return _corr_stream_chunks("tcorr_msd_stream_chunks", chunks, tau_max, stride, method, window_frames, out, ws,
                               stream, device)


def tcorr_acf_stream_chunks(chunks, tau_max: int, stride: int = 1, method=AUTO, window_frames: int = 0, out=None,
                            ws=None, stream=None, device=None):
    """Autocorrelation of a host-resident signal given as consecutive frame chunks."""
    return _corr_stream_chunks("tcorr_acf_stream_chunks", chunks, tau_max, stride, method, window_frames, out, ws,
                               stream, device)


def tcorr_plain_static(kind: int, x, tau_max: int, stride: int = 1, out=None, stream=None):
    """Plain path with the library's fixed device scratch (no workspace, nothing allocated
    by the library); kind 0 = MSD, 1 = autocorrelation."""
    torch = _torch()
    _check_traj(x)
    if out is None:
        out = _held_by(torch.empty(tau_max + 1, dtype=torch.float64, device=x.device), stream)
    _check_out(out, tau_max + 1, x.device)
    rc = load().tcorr_plain_static(kind, x.data_ptr(), x.shape[0], x.shape[1], tau_max, stride,
                                   out.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_plain_static")
    return out


def tcorr_profile_enable(on: bool = True) -> None:
    """Record CUDA events around every launch of the dominant kernel (diagnostics)."""
    load().tcorr_profile_enable(1 if on else 0)


def tcorr_profile_read(kind: int):
    """(summed milliseconds, launches) of the recorded dominant-kernel launches of one kind."""
    ms = ctypes.c_double()
    n = ctypes.c_int()
    rc = load().tcorr_profile_read(kind, ctypes.byref(ms), ctypes.byref(n))
    if rc != 0:
        raise TcorrError(rc, "tcorr_profile_read")
    return ms.value, n.value


def tcorr_status_poll(stream=None) -> int:
    return int(load().tcorr_status_poll(_stream_ptr(stream)))


def tcorr_selftest_timeout(stream=None) -> None:
    """Enqueue the device-side timeout self-test (sets TCORR_ETIMEOUT in the status word)."""
    rc = load().tcorr_selftest_timeout(_stream_ptr(stream))
    if rc != 0:
        raise TcorrError(rc, "tcorr_selftest_timeout")


def tcorr_version() -> int:
    return int(load().tcorr_version())


def correlate_host(kind: str, x_host, tau_max: int, stride: int = 1, method=AUTO,
                   device="cuda", ws=None, x_dev=None):
    """End-to-end call from host memory: copy x to the device, run, copy back.

    ``x_host`` is a (preferably pinned) float32 CPU tensor [T][N][3]; returns a
    float64 CPU tensor.  ``x_dev`` / ``ws`` may be given to reuse device buffers.
    """
    torch = _torch()
    if x_dev is None:
        x_dev = torch.empty(x_host.shape, dtype=torch.float32, device=device)
    x_dev.copy_(x_host, non_blocking=True)
    f = tcorr_msd if kind == "msd" else tcorr_acf
    out = f(x_dev, tau_max, stride, method, ws=ws)
    return out.to("cpu")
