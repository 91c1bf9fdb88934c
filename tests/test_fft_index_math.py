"""Index math of the FFT route's own transforms, checked on the CPU.

The route (fft.cu) transforms two real columns at once as one complex signal,
factors the length as L = L1 L2 (four-step: column transforms of length L1
with the twiddle W_L^(n2 k1), then row transforms of length L2, the spectrum
left in the transposed order [k1][k2]), forms the power spectrum point by
point, and runs the inverse in the opposite order.  Each transform in shared
memory is a Stockham FFT: butterfly idx of a radix-R stage (after transforms
of length Ns are done) reads elements idx + r P/R, multiplies by
W_(Ns R)^(r (idx mod Ns)) and writes element (idx // Ns) Ns R + idx mod Ns +
r Ns.  This test restates those index rules in numpy (complex128) and checks
the stages against numpy's FFT and the whole chain against the direct lag
sums of two real columns, for the lengths and factorisations the route uses.
"""
import numpy as np
import pytest


def dft_small(a, dirn):
    R = len(a)
    w = np.exp(dirn * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    return w @ a


def stockham(x, dirn):
    P = len(x)
    m = 3 if P % 3 == 0 else 5 if P % 5 == 0 else 1
    rem = P // m
    radices = []
    if rem > 1 and (rem.bit_length() - 1) % 2 == 1:
        radices.append(2)
        rem //= 2
    while rem >= 4:
        radices.append(4)
        rem //= 4
    if m > 1:
        radices.append(m)
    buf = x.astype(np.complex128).copy()
    Ns = 1
    for R in radices:
        nb = P // R
        out = np.empty_like(buf)
        for idx in range(nb):
            k = idx % Ns
            a = np.array([buf[idx + r * nb] for r in range(R)])
            if Ns > 1:
                a = a * np.exp(dirn * 2j * np.pi * np.arange(R) * k / (Ns * R))
            b = dft_small(a, dirn)
            base = (idx // Ns) * Ns * R + k
            for r in range(R):
                out[base + r * Ns] = b[r]
        buf = out
        Ns *= R
    return buf


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 160, 384, 640])
def test_stockham_stages_match_numpy(P):
    rng = np.random.default_rng(P)
    x = rng.normal(size=P) + 1j * rng.normal(size=P)
    np.testing.assert_allclose(stockham(x, -1), np.fft.fft(x), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(stockham(x, +1), np.fft.ifft(x) * P, rtol=1e-12, atol=1e-12)


def split(L, max_l2):
    if L <= max_l2:
        return 1, L
    l1 = 2
    while L // l1 > max_l2:
        l1 *= 2
    return l1, L // l1


def four_step(z, L1, L2, dirn, twiddle_after_cols):
    """Column pass (length L1 over n1, stride L2) then row pass (length L2)."""
    L = L1 * L2
    Y = z.reshape(L1, L2).copy()
    for n2 in range(L2):
        Y[:, n2] = stockham(Y[:, n2], dirn)
    k1 = np.arange(L1)[:, None]
    n2 = np.arange(L2)[None, :]
    Y *= np.exp(dirn * 2j * np.pi * (n2 * k1) / L)
    for r in range(L1):
        Y[r, :] = stockham(Y[r, :], dirn)
    return Y


def inverse_four_step(X, L1, L2):
    L = L1 * L2
    Y = X.copy()
    for r in range(L1):
        Y[r, :] = stockham(Y[r, :], +1)
    k1 = np.arange(L1)[:, None]
    n2 = np.arange(L2)[None, :]
    Y *= np.exp(+2j * np.pi * (n2 * k1) / L)
    for n2_ in range(L2):
        Y[:, n2_] = stockham(Y[:, n2_], +1)
    return Y.reshape(L)


@pytest.mark.parametrize("L,max_l2", [(48, 16), (160, 32), (96, 96), (320, 40), (384, 64), (640, 128)])
def test_transposed_spectrum_and_back(L, max_l2):
    """The forward chain gives X[k1 + L1 k2] at [k1][k2]; the inverse chain
    takes that order back to L times the input."""
    L1, L2 = split(L, max_l2)
    rng = np.random.default_rng(L)
    z = rng.normal(size=L) + 1j * rng.normal(size=L)
    X = four_step(z, L1, L2, -1, True)
    F = np.fft.fft(z)
    k1 = np.arange(L1)[:, None]
    k2 = np.arange(L2)[None, :]
    np.testing.assert_allclose(X, F[k1 + L1 * k2], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(inverse_four_step(X, L1, L2), L * z, rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("T,tm,s,max_l2", [(30, 29, 1, 16), (50, 20, 3, 16), (21, 20, 2, 8)])
def test_two_columns_per_complex_signal(T, tm, s, max_l2):
    """Re IFFT(conj(F w) F z) with z = a + i b and w the origin-masked copy is
    the sum of the two columns' lag sums over origins in sZ."""
    rng = np.random.default_rng(T + tm)
    a, b = rng.normal(size=T), rng.normal(size=T)
    n = T + tm
    L = min(m * 2 ** int(np.ceil(np.log2(n / m))) for m in (1, 3, 5))
    L1, L2 = split(L, max_l2)
    z = np.zeros(L, complex)
    z[:T] = a + 1j * b
    w = z.copy()
    w[np.arange(L) % s != 0] = 0
    Z = four_step(z, L1, L2, -1, True)
    W = four_step(w, L1, L2, -1, True)
    lag = inverse_four_step(Z * np.conj(W), L1, L2).real / L
    want = [sum(a[t] * a[t + tau] + b[t] * b[t + tau] for t in range(0, T - tau, s)) for tau in range(tm + 1)]
    np.testing.assert_allclose(lag[:tm + 1], want, rtol=1e-10, atol=1e-10)
