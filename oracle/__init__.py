"""FP64 CPU oracle for the multiple-time-origin MSD / autocorrelation path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the CPU-baseline legs of ``bench.py``.  The CUDA library never imports,
links or calls anything here, and nothing here imports the CUDA library.

The arithmetic lives in ``tcorr_oracle.c`` (plain FP64 loops following
Eq. 5 / Algorithm 10 for the MSD, Eq. 4 / Algorithm 8 for the
autocorrelation and its running Green-Kubo integral, the same loop nest
with the later factor taken from a second signal for the cross-correlation,
and the weighted atom sum that forms a collective signal).  This module compiles it
with gcc (no FMA contraction, no fast-math, so x86 and Arm give the same bits)
and marshals numpy arrays through ctypes.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute force, FFT, closed forms, invariants,
statistics) and ``tests/test_oracle_mutants.py`` (planted mistakes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcorr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

KIND_MSD = 0
KIND_ACF = 1


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle into a shared library; returns its path."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build() -> str:
    """Build liboracle.so next to this file if it is missing or stale."""
    if (not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        compile_oracle()
    return _LIB_PATH


def load_library(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    i64, dbl = ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_corr.argtypes = [ctypes.c_int, vp, i64, i64, i64, vp, i64, vp, ctypes.c_int]
    lib.oracle_corr.restype = ctypes.c_int
    lib.oracle_corr_weighted.argtypes = [ctypes.c_int, vp, vp, i64, i64, i64, vp, i64, vp, ctypes.c_int]
    lib.oracle_corr_weighted.restype = ctypes.c_int
    lib.oracle_xcorr.argtypes = [vp, vp, i64, i64, i64, vp, i64, vp, ctypes.c_int]
    lib.oracle_xcorr.restype = ctypes.c_int
    lib.oracle_collective.argtypes = [vp, vp, i64, i64, i64, vp]
    lib.oracle_collective.restype = ctypes.c_int
    lib.oracle_gk_integrate.argtypes = [vp, i64, dbl, dbl, vp]
    lib.oracle_gk_integrate.restype = ctypes.c_int
    lib.oracle_einstein.argtypes = [vp, i64, dbl, ctypes.c_int, i64, i64, vp, vp]
    lib.oracle_einstein.restype = ctypes.c_int
    return lib


def _get_lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def corr(kind: int, x: np.ndarray, tau_max: int | None = None, stride: int = 1,
         lags=None, nthreads: int | None = None, lib=None) -> np.ndarray:
    """MSD (kind 0) or autocorrelation (kind 1) of x[T][N][3] float32.

    Returns FP64 values at ``lags`` (default 0..tau_max).
    """
    lib = lib or _get_lib()
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim != 3 or x.shape[2] != 3:
        raise ValueError("x must have shape [T][N][3]")
    T, N, _ = x.shape
    if lags is None:
        if tau_max is None:
            tau_max = T - 1
        lags = np.arange(tau_max + 1, dtype=np.int64)
    lags = np.ascontiguousarray(lags, dtype=np.int64)
    out = np.zeros(lags.shape[0], dtype=np.float64)
    rc = lib.oracle_corr(kind, x.ctypes.data, T, N, stride, lags.ctypes.data,
                         lags.shape[0], out.ctypes.data, nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle_corr failed with code {rc}")
    return out


def msd(x, tau_max=None, stride=1, lags=None, nthreads=None, lib=None):
    """Mean square displacement, Eq. 5 averaged over atoms and origins."""
    return corr(KIND_MSD, x, tau_max, stride, lags, nthreads, lib)


def acf(x, tau_max=None, stride=1, lags=None, nthreads=None, lib=None):
    """Autocorrelation <A(t0).A(t0+tau)>, the integrand of Eq. 4."""
    return corr(KIND_ACF, x, tau_max, stride, lags, nthreads, lib)


def corr_weighted(kind: int, x: np.ndarray, w: np.ndarray, tau_max: int | None = None, stride: int = 1,
                  lags=None, nthreads=None, lib=None) -> np.ndarray:
    """Weighted atom average: sum_i w_i (atom i's per-lag sum) / (sum_i w_i n_o(tau))."""
    lib = lib or _get_lib()
    x = np.ascontiguousarray(x, dtype=np.float32)
    T, N = x.shape[0], x.shape[1]
    w = np.ascontiguousarray(w, dtype=np.float32)
    if w.shape != (N,):
        raise ValueError("w must hold one weight per atom")
    if lags is None:
        if tau_max is None:
            tau_max = T - 1
        lags = np.arange(tau_max + 1, dtype=np.int64)
    lags = np.ascontiguousarray(lags, dtype=np.int64)
    out = np.zeros(lags.shape[0], dtype=np.float64)
    rc = lib.oracle_corr_weighted(kind, x.ctypes.data, w.ctypes.data, T, N, stride, lags.ctypes.data,
                                  lags.shape[0], out.ctypes.data, nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle_corr_weighted failed with code {rc}")
    return out


def msd_weighted(x, w, tau_max=None, stride=1, lags=None, nthreads=None, lib=None):
    return corr_weighted(KIND_MSD, x, w, tau_max, stride, lags, nthreads, lib)


def acf_weighted(x, w, tau_max=None, stride=1, lags=None, nthreads=None, lib=None):
    return corr_weighted(KIND_ACF, x, w, tau_max, stride, lags, nthreads, lib)


def xcf(a, b, tau_max=None, stride=1, lags=None, nthreads=None, lib=None) -> np.ndarray:
    """Cross-correlation <A(t0).B(t0+tau)> of a[T][N][3] and b[T][N][3] float32."""
    lib = lib or _get_lib()
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    if a.ndim != 3 or a.shape[2] != 3 or b.shape != a.shape:
        raise ValueError("a and b must both have shape [T][N][3]")
    T, N, _ = a.shape
    if lags is None:
        if tau_max is None:
            tau_max = T - 1
        lags = np.arange(tau_max + 1, dtype=np.int64)
    lags = np.ascontiguousarray(lags, dtype=np.int64)
    out = np.zeros(lags.shape[0], dtype=np.float64)
    rc = lib.oracle_xcorr(a.ctypes.data, b.ctypes.data, T, N, stride, lags.ctypes.data,
                          lags.shape[0], out.ctypes.data, nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle_xcorr failed with code {rc}")
    return out


def collective(x, w=None, ref_frame: int = -1, lib=None) -> np.ndarray:
    """J[t][c] = sum_i w_i (x[t][i][c] - x[ref][i][c]) in FP64 ([T][3]); ref_frame -1: no reference."""
    lib = lib or _get_lib()
    x = np.ascontiguousarray(x, dtype=np.float32)
    T, N = x.shape[0], x.shape[1]
    wp = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.shape != (N,):
            raise ValueError("w must hold one weight per atom")
        wp = w.ctypes.data
    out = np.zeros((T, 3), dtype=np.float64)
    if lib.oracle_collective(x.ctypes.data, wp, T, N, ref_frame, out.ctypes.data) != 0:
        raise ValueError("oracle_collective: bad arguments")
    return out


def gk_integrate(c, dt: float, prefactor: float = 1.0, lib=None) -> np.ndarray:
    """Running trapezoid integral prefactor * int_0^tau C, Eq. 4."""
    lib = lib or _get_lib()
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros_like(c)
    if lib.oracle_gk_integrate(c.ctypes.data, c.shape[0], dt, prefactor, out.ctypes.data) != 0:
        raise ValueError("oracle_gk_integrate: bad arguments")
    return out


def einstein(msd_values, dt: float, dim: int = 3, lo: int | None = None,
             hi: int | None = None, lib=None):
    """(D from the least-squares slope over [lo, hi], D from the ratio at hi)."""
    lib = lib or _get_lib()
    m = np.ascontiguousarray(msd_values, dtype=np.float64)
    n = m.shape[0]
    if hi is None:
        hi = n - 1
    if lo is None:
        lo = -(-(2 * hi) // 10)  # ceil(0.2 * hi)
    d_slope = ctypes.c_double()
    d_ratio = ctypes.c_double()
    rc = lib.oracle_einstein(m.ctypes.data, n, dt, dim, lo, hi,
                             ctypes.addressof(d_slope), ctypes.addressof(d_ratio))
    if rc != 0:
        raise ValueError("oracle_einstein: bad arguments")
    return d_slope.value, d_ratio.value


def n_origins(T: int, tau, stride: int = 1):
    """n_o(tau) = floor((T-1-tau)/s) + 1, the number of origins for lag tau."""
    tau = np.asarray(tau, dtype=np.int64)
    return (T - 1 - tau) // stride + 1
