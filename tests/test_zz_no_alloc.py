"""The entry point that allocates nothing (tcorr_plain_static), through the C ABI.

Some callers cannot allocate device memory (an analysis hook inside an engine
that owns all device memory through its own pool, or a host that must not call
cudaMalloc because it synchronises the device).  tcorr_plain_static serves them
from one fixed array of device memory inside the library.  These checks call it
twice in a row, on different shapes and data, and compare each result with the
workspace-based entry points (tcorr_msd / tcorr_acf, plain method); a third call
asks for more scratch than the array holds and must be refused.  This file is
collected last so that a run stopping at the first failure has run every other
test first.
"""
import ctypes

import numpy as np
import pytest

from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TCORR_EWORKSPACE = 4


@pytest.fixture(scope="module")
def lib():
    from paper_1708_08619_gb300 import build, tcorr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return tcorr.load()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _static(lib, kind, x, tau_max, stride):
    out = torch.full((tau_max + 1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.tcorr_plain_static(kind, x.data_ptr(), x.shape[0], x.shape[1], tau_max, stride,
                                out.data_ptr(), _stream())
    assert rc == 0, rc
    return out


def _with_workspace(lib, kind, x, tau_max, stride):
    T, N = x.shape[0], x.shape[1]
    need = lib.tcorr_workspace_size(T, N, tau_max, stride, 0)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    out = torch.empty(tau_max + 1, dtype=torch.float64, device="cuda")
    f = lib.tcorr_msd if kind == 0 else lib.tcorr_acf
    rc = f(x.data_ptr(), T, N, tau_max, stride, 0, out.data_ptr(), ws.data_ptr(), need, _stream())
    assert rc == 0, rc
    return out


def test_two_calls_match_workspace_entry_points(lib):
    rng = np.random.default_rng(4242)
    pos = (rng.normal(size=(700, 300, 3)).cumsum(axis=0) * 0.02
           + rng.uniform(0, 3, size=(1, 300, 3))).astype(np.float32)
    vel = rng.normal(size=(500, 77, 3)).astype(np.float32)
    x = torch.from_numpy(pos).cuda()
    v = torch.from_numpy(vel).cuda()

    # first call: MSD; second call right after it: ACF of another shape and stride
    m_static = _static(lib, 0, x, 400, 1)
    c_static = _static(lib, 1, v, 499, 3)
    m_ref = _with_workspace(lib, 0, x, 400, 1)
    c_ref = _with_workspace(lib, 1, v, 499, 3)
    torch.cuda.synchronize()
    m_s, m_r = m_static.cpu().numpy(), m_ref.cpu().numpy()
    c_s, c_r = c_static.cpu().numpy(), c_ref.cpu().numpy()
    # same plan, same kernels, same summation order: the results agree bit for bit
    assert np.array_equal(m_s, m_r), "static msd differs from the workspace msd"
    assert np.array_equal(c_s, c_r), "static acf differs from the workspace acf"
    parity.check_plain_msd(m_s, m_r, what="static msd vs workspace msd")
    parity.check_acf(c_s, c_r, parity.PLAIN_TOL, what="static acf vs workspace acf")

    # the same calls again, in the other order, reuse the array's old contents
    c_again = _static(lib, 1, v, 499, 3).cpu().numpy()
    m_again = _static(lib, 0, x, 400, 1).cpu().numpy()
    assert np.array_equal(m_again, m_r), "static msd, second round"
    assert np.array_equal(c_again, c_r), "static acf, second round"


def test_refuses_shapes_beyond_the_fixed_array(lib):
    # 200000 frames of 10 atoms with tau_max = 100000 need about 1.2M band tiles of
    # partial sums, far beyond the 32 MiB array.  The trajectory and the output have
    # the full size the arguments describe, so no change to the order of the argument
    # checks can make this call read or write past them; the output stays untouched.
    T, N, tm = 200000, 10, 100000
    x = torch.zeros((T, N, 3), dtype=torch.float32, device="cuda")
    out = torch.full((tm + 1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.tcorr_plain_static(0, x.data_ptr(), T, N, tm, 1, out.data_ptr(), _stream())
    torch.cuda.synchronize()
    assert rc == TCORR_EWORKSPACE
    assert torch.isnan(out).all().item(), "a refused call wrote its output"
