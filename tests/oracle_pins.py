"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each ``pin_*`` function takes a loaded oracle library (``oracle.load_library``)
and raises AssertionError when the oracle disagrees with what the paper's
definitions and plain mathematics fix:

* a hand-worked example (``tests/golden/hand_worked_T4_N2.json``);
* brute force over every ordered frame pair, binned by lag;
* the Wiener-Khinchin route (numpy FFT) for correlations and the FFT form of
  the MSD (|a-b|^2 = |a|^2 + |b|^2 - 2 a.b summed over origins);
* closed forms: constant velocity (MSD = <|v|^2> tau^2, constant correlation),
  the trapezoid of a constant and of a geometric series, the least-squares
  slope of an exactly linear MSD;
* invariants: per-atom shifts, time reversal, atom permutation, scaling, and
  the split of stride-1 origins into two stride-2 sets;
* statistics: random walk (E[MSD] = 3 sigma^2 tau), Ornstein-Uhlenbeck
  (C(tau)/C(0) = phi^tau within Bartlett errors), and Einstein D = Green-Kubo D
  for positions integrated from OU velocities;
* the collective (weighted atom-sum) signal: one-hot selection, linearity,
  shift invariance, the ballistic closed form and its Einstein-Helfand MSD.

The same functions run against planted-mistake copies of the oracle in
``test_oracle_mutants.py``; each copy must fail at least one of them.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
from paper_1708_08619_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _close(a, b, rtol, atol=0.0, what=""):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    err = np.abs(a - b)
    lim = atol + rtol * np.abs(b)
    if not np.all(err <= lim):
        k = int(np.argmax(err - lim))
        raise AssertionError(f"{what}: mismatch at {k}: got {a.flat[k]!r}, want {b.flat[k]!r}")


# ----------------------------------------------------------------- hand worked

def pin_hand_worked(lib):
    with open(os.path.join(GOLDEN, "hand_worked_T4_N2.json")) as f:
        g = json.load(f)
    x = np.array(g["x"], dtype=np.float32)
    for s, key in ((1, "stride1"), (2, "stride2")):
        _close(oracle.msd(x, 3, s, lib=lib), g[key]["msd"], 1e-15, what=f"hand msd s={s}")
        _close(oracle.acf(x, 3, s, lib=lib), g[key]["acf"], 1e-15, what=f"hand acf s={s}")


# ----------------------------------------------------------------- brute force

def _brute_pairs(x, tau_max, s, kind):
    """Every ordered frame pair (t, t') with t a multiple of s, binned by lag."""
    x = x.astype(np.float64)
    T = x.shape[0]
    t = np.arange(0, T, s)
    tp = np.arange(T)
    tt, ttp = np.meshgrid(t, tp, indexing="ij")
    keep = (ttp >= tt) & (ttp - tt <= tau_max)
    tt, ttp = tt[keep], ttp[keep]
    if kind == "msd":
        val = ((x[ttp] - x[tt]) ** 2).sum(axis=2)      # [pairs][N]
    else:
        val = (x[ttp] * x[tt]).sum(axis=2)
    sums = np.zeros(tau_max + 1)
    counts = np.zeros(tau_max + 1)
    np.add.at(sums, ttp - tt, val.sum(axis=1))
    np.add.at(counts, ttp - tt, val.shape[1])
    return sums / counts


def pin_brute_force(lib):
    rng = np.random.default_rng(11)
    for T in (1, 2, 3, 5, 8, 12):
        for N in (1, 2, 3):
            x = rng.normal(size=(T, N, 3)).astype(np.float32)
            for s in (1, 2, 3, T + 1):
                for tau_max in range(T):
                    for kind, f in (("msd", oracle.msd), ("acf", oracle.acf)):
                        want = _brute_pairs(x, tau_max, s, kind)
                        got = f(x, tau_max, s, lib=lib)
                        _close(got, want, 1e-13, 1e-15, what=f"brute {kind} T={T} N={N} s={s} tm={tau_max}")


def pin_lag_subset(lib):
    """Evaluating a subset of lags gives the same values as the full range."""
    rng = np.random.default_rng(12)
    x = rng.normal(size=(40, 7, 3)).astype(np.float32)
    full_m = oracle.msd(x, 39, 2, lib=lib)
    full_c = oracle.acf(x, 39, 2, lib=lib)
    lags = np.array([39, 0, 17, 1, 38, 5])
    _close(oracle.msd(x, stride=2, lags=lags, lib=lib), full_m[lags], 0.0, what="msd subset")
    _close(oracle.acf(x, stride=2, lags=lags, lib=lib), full_c[lags], 0.0, what="acf subset")


# ------------------------------------------------------------------------- FFT

def _fft_lag_products(a):
    """sum_t a[t] a[t+tau] for every tau, per column, by Wiener-Khinchin."""
    T = a.shape[0]
    n = 1 << (2 * T - 1).bit_length()
    f = np.fft.rfft(a, n=n, axis=0)
    return np.fft.irfft(f * np.conj(f), n=n, axis=0)[:T]


def pin_fft(lib):
    rng = np.random.default_rng(13)
    for T, N in ((64, 5), (97, 3)):
        x = rng.uniform(-2.0, 2.0, size=(T, N, 3)).astype(np.float32)
        xd = x.astype(np.float64).reshape(T, -1)
        tau = np.arange(T)
        n_o = T - tau
        prod = _fft_lag_products(xd).sum(axis=1)
        _close(oracle.acf(x, T - 1, 1, lib=lib), prod / (N * n_o), 1e-10, 1e-12, what="fft acf")
        sq = (xd ** 2).sum(axis=1)
        cs = np.concatenate([[0.0], np.cumsum(sq)])
        first = cs[T - tau]            # sum_{t0 < T - tau} |x_t0|^2
        second = cs[T] - cs[tau]       # sum_{t0 >= tau} |x_t0|^2
        msd = (first + second - 2.0 * prod) / (N * n_o)
        _close(oracle.msd(x, T - 1, 1, lib=lib), msd, 1e-9, 1e-11, what="fft msd")


# --------------------------------------------------------------- closed forms

def pin_constant_velocity(lib):
    x, v = synth.constant_velocity(300, 50, seed=14)
    tau = np.arange(300)
    v2 = (v ** 2).sum(axis=1).mean()
    _close(oracle.msd(x, 299, 1, lib=lib), v2 * tau.astype(np.float64) ** 2, 1e-14,
           what="constant velocity msd")
    _close(oracle.msd(x, 150, 7, lib=lib), v2 * tau[:151].astype(np.float64) ** 2, 1e-14,
           what="constant velocity msd s=7")
    # A_t = v for every t: the correlation is <|v|^2> at every lag
    a = np.broadcast_to(v.astype(np.float32)[None], (300, 50, 3)).copy()
    _close(oracle.acf(a, 299, 1, lib=lib), np.full(300, v2), 1e-14, what="constant acf")
    _close(oracle.acf(a, 299, 4, lib=lib), np.full(300, v2), 1e-14, what="constant acf s=4")


def pin_zero_lag(lib):
    rng = np.random.default_rng(15)
    x = rng.normal(size=(33, 9, 3)).astype(np.float32)
    assert oracle.msd(x, 5, 1, lib=lib)[0] == 0.0
    assert oracle.msd(x, 5, 3, lib=lib)[0] == 0.0
    want = (x.astype(np.float64) ** 2).sum(axis=2).mean()
    _close(oracle.acf(x, 0, 1, lib=lib), [want], 1e-13, what="C(0) = <|A|^2>")
    want3 = (x[::3].astype(np.float64) ** 2).sum(axis=2).mean()
    _close(oracle.acf(x, 0, 3, lib=lib), [want3], 1e-13, what="C(0) stride 3")


def pin_single_origin(lib):
    """With stride >= T only t0 = 0 is an origin: MSD(tau) = <|x_tau - x_0|^2>."""
    rng = np.random.default_rng(16)
    x = rng.normal(size=(20, 6, 3)).astype(np.float32)
    xd = x.astype(np.float64)
    want_m = ((xd - xd[0:1]) ** 2).sum(axis=2).mean(axis=1)
    want_c = (xd * xd[0:1]).sum(axis=2).mean(axis=1)
    _close(oracle.msd(x, 19, 20, lib=lib), want_m, 1e-13, what="single origin msd")
    _close(oracle.acf(x, 19, 25, lib=lib), want_c, 1e-13, 1e-15, what="single origin acf")


# ----------------------------------------------------------------- invariants

def pin_invariants(lib):
    rng = np.random.default_rng(17)
    T, N = 50, 11
    q = 2.0 ** -10
    x = (rng.integers(-4096, 4096, size=(T, N, 3)) * q).astype(np.float32)
    shift = (rng.integers(-1024, 1024, size=(1, N, 3)) * q).astype(np.float32)
    m = oracle.msd(x, T - 1, 1, lib=lib)
    # per-atom constant shift (exact in float32 here)
    _close(oracle.msd(x + shift, T - 1, 1, lib=lib), m, 1e-13, what="shift invariance")
    # time reversal: the same frame pairs at every lag (stride 1)
    _close(oracle.msd(x[::-1].copy(), T - 1, 1, lib=lib), m, 1e-13, what="time reversal msd")
    c = oracle.acf(x, T - 1, 1, lib=lib)
    _close(oracle.acf(x[::-1].copy(), T - 1, 1, lib=lib), c, 1e-12, 1e-14, what="time reversal acf")
    # atom permutation
    p = rng.permutation(N)
    _close(oracle.msd(x[:, p].copy(), T - 1, 2, lib=lib), oracle.msd(x, T - 1, 2, lib=lib),
           1e-13, what="permutation")
    # scaling by 2 multiplies both by 4 exactly
    _close(oracle.acf(2 * x, T - 1, 3, lib=lib), 4 * oracle.acf(x, T - 1, 3, lib=lib), 0.0,
           what="acf scaling")
    _close(oracle.msd(2 * x, T - 1, 3, lib=lib), 4 * oracle.msd(x, T - 1, 3, lib=lib), 0.0,
           what="msd scaling")
    # components are independent: permuting x,y,z changes nothing
    _close(oracle.msd(x[:, :, ::-1].copy(), T - 1, 1, lib=lib), m, 1e-13, what="component order")


def pin_stride_split(lib):
    """Origins {0,1,2,...} = {0,2,4,...} + {1,3,5,...}: the sums must add up."""
    rng = np.random.default_rng(18)
    T, N = 41, 5
    x = rng.normal(size=(T, N, 3)).astype(np.float32)
    tm = 30
    tau = np.arange(tm + 1)
    for f in (oracle.msd, oracle.acf):
        s1 = f(x, tm, 1, lib=lib) * (T - tau)
        even = f(x, tm, 2, lib=lib)
        odd = f(x[1:].copy(), tm, 2, lib=lib)
        n_even = np.array([len(range(0, T - t, 2)) for t in tau])
        n_odd = np.array([len(range(1, T - t, 2)) for t in tau])
        comb = even * n_even + odd * n_odd
        _close(s1, comb, 1e-12, 1e-12, what=f"stride split {f.__name__}")


# ------------------------------------------------------------------ quadrature

def pin_gk_closed_forms(lib):
    n, dt = 101, 0.25
    c = np.full(n, 3.0)
    _close(oracle.gk_integrate(c, dt, 2.0, lib=lib), 2.0 * 3.0 * dt * np.arange(n), 1e-15,
           what="trapezoid of a constant")
    phi = 0.9
    g = phi ** np.arange(n)
    k = np.arange(n)
    want = dt * (1 + phi) / 2 * (1 - phi ** k) / (1 - phi)
    _close(oracle.gk_integrate(g, dt, 1.0, lib=lib), want, 1e-13, 1e-16, what="trapezoid of phi^k")
    # a straight line is integrated exactly by the trapezoid rule
    lin = 1.5 + 0.5 * k
    _close(oracle.gk_integrate(lin, 1.0, 1.0, lib=lib), 1.5 * k + 0.25 * k ** 2, 1e-14,
           what="trapezoid of a line")


def pin_einstein_exact(lib):
    tau = np.arange(201, dtype=np.float64)
    dt, a, b = 0.5, 0.3, 0.01
    m = a * tau * dt + b
    d_slope, d_ratio = oracle.einstein(m, dt, 3, 40, 200, lib=lib)
    assert abs(d_slope - a / 6) <= 1e-13, d_slope
    assert abs(d_ratio - (a * 200 * dt + b) / (6 * 200 * dt)) <= 1e-15, d_ratio
    d2, _ = oracle.einstein(m, dt, 2, 40, 200, lib=lib)
    assert abs(d2 - a / 4) <= 1e-13, d2


# ------------------------------------------------------------------ statistics

def pin_random_walk(lib):
    sigma, T, N = 0.05, 200, 3000
    x = synth.random_walk_positions(T, N, sigma, 3.0, seed=19)
    m = oracle.msd(x, 20, 1, lib=lib)
    tau = np.arange(1, 21)
    ratio = m[1:] / (3 * sigma ** 2 * tau)
    assert np.all(np.abs(ratio - 1.0) < 0.03), ratio


def pin_ou(lib):
    gamma, sigma, T, N = 0.1, 1.0, 400, 2000
    v = synth.ou_velocities(T, N, gamma, sigma, seed=20)
    c = oracle.acf(v, 20, 1, lib=lib)
    phi = math.exp(-gamma)
    tau = np.arange(21)
    r = c / c[0]
    # Bartlett variance of the sample autocorrelation of an AR(1) series,
    # averaged over 3N independent series of length T
    var = ((1 + phi ** 2) * (1 - phi ** (2 * tau)) / (1 - phi ** 2) - 2 * tau * phi ** (2 * tau)) / (3 * N * T)
    se = np.sqrt(np.maximum(var, 1e-30))
    assert np.all(np.abs(r - phi ** tau) <= 5 * se + 1e-12), (r, phi ** tau, se)
    assert abs(c[0] / (3 * sigma ** 2) - 1) < 0.01, c[0]


def pin_einstein_vs_green_kubo(lib):
    """Positions x_{t+1} = x_t + v_t dt with OU velocities v: Einstein D = GK D.

    For this discrete model MSD(tau) = dt^2 [tau C(0) + 2 sum_{m<tau} (tau-m) C(m)],
    whose slope per unit time tends to dt [C(0) + 2 sum_{m>=1} C(m)]; the
    trapezoid integral of C is dt [C(0)/2 + sum_{m>=1} C(m)]; with d = 3 and C
    summed over components the two D agree, both equal to
    dt sigma^2 (1 + phi) / (2 (1 - phi)).
    """
    gamma, sigma, T, N, dt = 0.2, 1.0, 2000, 1000, 0.5
    v = synth.ou_velocities(T, N, gamma, sigma, seed=21)
    x = np.concatenate([np.zeros((1, N, 3)), np.cumsum(v.astype(np.float64) * dt, axis=0)[:-1]], axis=0)
    x = x.astype(np.float32)
    tm = 100
    m = oracle.msd(x, tm, 1, lib=lib)
    c = oracle.acf(v, tm, 1, lib=lib)
    d_e, _ = oracle.einstein(m, dt, 3, 40, tm, lib=lib)
    d_gk = oracle.gk_integrate(c, dt, 1.0 / 3.0, lib=lib)[-1]
    phi = math.exp(-gamma)
    d_true = dt * sigma ** 2 * (1 + phi) / (2 * (1 - phi))
    assert abs(d_e / d_true - 1) < 0.05, (d_e, d_true)
    assert abs(d_gk / d_true - 1) < 0.05, (d_gk, d_true)
    assert abs(d_e / d_gk - 1) < 0.05, (d_e, d_gk)


# ------------------------------------------------------- cross-correlation

def _brute_cross(a, b, tau_max, s):
    """sum over origins t0 (multiples of s) of a[t0] . b[t0 + tau], over every
    ordered frame pair, binned by lag and averaged over atoms and origins."""
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    T, N, _ = a.shape
    sums = np.zeros(tau_max + 1)
    counts = np.zeros(tau_max + 1)
    for t0 in range(0, T, s):
        for t1 in range(t0, min(T, t0 + tau_max + 1)):
            sums[t1 - t0] += float((a[t0] * b[t1]).sum())
            counts[t1 - t0] += N
    return sums / counts


def pin_xcf_brute_force(lib):
    rng = np.random.default_rng(31)
    for T in (1, 2, 5, 9):
        for N in (1, 3):
            a = rng.normal(size=(T, N, 3)).astype(np.float32)
            b = rng.normal(size=(T, N, 3)).astype(np.float32)
            for s in (1, 2, T + 1):
                for tau_max in range(T):
                    _close(oracle.xcf(a, b, tau_max, s, lib=lib), _brute_cross(a, b, tau_max, s), 1e-13, 1e-15,
                           what=f"brute xcf T={T} N={N} s={s} tm={tau_max}")


def pin_xcf_fft(lib):
    """sum_t a[t] b[t+tau] per column = irfft(conj(rfft a) rfft b) (zero padded)."""
    rng = np.random.default_rng(32)
    T, N = 80, 4
    a = rng.uniform(-1.0, 1.0, size=(T, N, 3)).astype(np.float32)
    b = rng.uniform(-1.0, 1.0, size=(T, N, 3)).astype(np.float32)
    n = 1 << (2 * T - 1).bit_length()
    fa = np.fft.rfft(a.astype(np.float64).reshape(T, -1), n=n, axis=0)
    fb = np.fft.rfft(b.astype(np.float64).reshape(T, -1), n=n, axis=0)
    lagged = np.fft.irfft(np.conj(fa) * fb, n=n, axis=0)[:T].sum(axis=1)
    want = lagged / (N * (T - np.arange(T)))
    _close(oracle.xcf(a, b, T - 1, lib=lib), want, 1e-10, 1e-13, what="xcf fft")


def pin_xcf_closed_forms(lib):
    """A constant (p) and B linear in time (v t), dyadic so every product is
    exact: X(tau) = <p.v> (tau + s (n_o - 1) / 2); the reverse order gives
    <p.v> s (n_o - 1) / 2, so the two signals' roles are pinned.  And X(A, A)
    is the autocorrelation, bit for bit."""
    rng = np.random.default_rng(33)
    T, N = 60, 5
    p = (rng.integers(-64, 64, size=(N, 3)) / 64.0).astype(np.float32)
    v = (rng.integers(-64, 64, size=(N, 3)) / 1024.0).astype(np.float32)
    a = np.repeat(p[None], T, axis=0)
    t = np.arange(T, dtype=np.float32)[:, None, None]
    b = (v[None] * t).astype(np.float32)
    pv = float((p.astype(np.float64) * v.astype(np.float64)).sum()) / N
    for s in (1, 3):
        tau = np.arange(T)
        n_o = (T - 1 - tau) // s + 1
        _close(oracle.xcf(a, b, T - 1, s, lib=lib), pv * (tau + s * (n_o - 1) / 2.0), 1e-13, 1e-14,
               what=f"xcf const x linear s={s}")
        _close(oracle.xcf(b, a, T - 1, s, lib=lib), pv * (s * (n_o - 1) / 2.0), 1e-13, 1e-14,
               what=f"xcf linear x const s={s}")
    x = rng.normal(size=(30, 6, 3)).astype(np.float32)
    if not np.array_equal(oracle.xcf(x, x, 29, 2, lib=lib), oracle.acf(x, 29, 2, lib=lib)):
        raise AssertionError("xcf(A, A) differs from acf(A)")


# ----------------------------------------------------------------- collective signal

def pin_collective(lib):
    """The weighted atom sum J[t] = sum_i w_i (x[t][i] - x[ref][i]) on dyadic data
    (every product and partial sum exact in FP64, so each check is bit for bit):
    one-hot weights select one atom; J is linear in the weights; with a reference
    frame J does not change when each atom is shifted by a constant; unit weights
    (no weight array) are the plain atom sum; and a constant-velocity system gives
    J(t) = (sum_i w_i v_i)(t - ref), whose MSD is |sum_i w_i v_i|^2 tau^2 (the
    Einstein-Helfand MSD of a ballistic system)."""
    rng = np.random.default_rng(41)
    T, N = 40, 7
    x = (rng.integers(-4096, 4096, size=(T, N, 3)) / 1024.0).astype(np.float32)
    w1 = (rng.integers(-16, 16, size=N) / 8.0).astype(np.float32)
    w2 = (rng.integers(-16, 16, size=N) / 8.0).astype(np.float32)
    for ref in (-1, 0, 17, T - 1):
        for j in (0, 3, N - 1):
            e = np.zeros(N, dtype=np.float32)
            e[j] = 1.0
            want = x[:, j, :].astype(np.float64) - (x[ref, j].astype(np.float64) if ref >= 0 else 0.0)
            if not np.array_equal(oracle.collective(x, e, ref, lib=lib), want):
                raise AssertionError(f"collective one-hot atom {j} ref {ref}")
        lin = oracle.collective(x, w1, ref, lib=lib) + oracle.collective(x, w2, ref, lib=lib)
        if not np.array_equal(oracle.collective(x, w1 + w2, ref, lib=lib), lin):
            raise AssertionError(f"collective not linear in the weights (ref {ref})")
        plain = (x.astype(np.float64) - (x[ref].astype(np.float64) if ref >= 0 else 0.0)).sum(axis=1)
        if not np.array_equal(oracle.collective(x, None, ref, lib=lib), plain):
            raise AssertionError(f"collective with unit weights (ref {ref})")
    shift = (rng.integers(-64, 64, size=(1, N, 3)) / 4.0).astype(np.float32)
    for ref in (0, 9):
        if not np.array_equal(oracle.collective(x + shift, w1, ref, lib=lib), oracle.collective(x, w1, ref, lib=lib)):
            raise AssertionError(f"collective with a reference frame changed under per-atom shifts (ref {ref})")
    x0 = (rng.integers(-64, 64, size=(N, 3)) / 8.0).astype(np.float32)
    v = (rng.integers(-64, 64, size=(N, 3)) / 256.0).astype(np.float32)
    t = np.arange(T, dtype=np.float64)
    xc = (x0[None].astype(np.float64) + v[None].astype(np.float64) * t[:, None, None]).astype(np.float32)
    wv = (w1[:, None].astype(np.float64) * v.astype(np.float64)).sum(axis=0)
    for ref in (0, 11):
        J = oracle.collective(xc, w1, ref, lib=lib)
        if not np.array_equal(J, wv[None] * (t - ref)[:, None]):
            raise AssertionError(f"collective constant-velocity closed form (ref {ref})")
        m = oracle.msd(J.astype(np.float32)[:, None, :], T - 1, lib=lib)
        _close(m, float((wv ** 2).sum()) * t ** 2, 1e-15, what=f"Einstein-Helfand MSD, ballistic (ref {ref})")


# ----------------------------------------------------------------- weighted atom averages

def pin_weighted(lib):
    """Weighted atom averages: unit weights are the plain average bit for bit;
    a one-hot weight is that atom alone; weights scaled by a power of two leave
    the result unchanged bit for bit; integer weights equal the plain average
    over a trajectory holding atom i w_i times."""
    rng = np.random.default_rng(43)
    T, N = 36, 9
    x = rng.normal(size=(T, N, 3)).astype(np.float32)
    wi = rng.integers(0, 4, size=N).astype(np.float32)
    wi[0] = 2.0
    for kind, f, fw in ((0, oracle.msd, oracle.msd_weighted), (1, oracle.acf, oracle.acf_weighted)):
        for s in (1, 2):
            plain = f(x, T - 1, s, lib=lib)
            if not np.array_equal(fw(x, np.ones(N, np.float32), T - 1, s, lib=lib), plain):
                raise AssertionError(f"weighted kind {kind} s={s}: unit weights differ from the plain average")
            e = np.zeros(N, np.float32)
            e[4] = 1.0
            if not np.array_equal(fw(x, e, T - 1, s, lib=lib), f(x[:, 4:5, :], T - 1, s, lib=lib)):
                raise AssertionError(f"weighted kind {kind} s={s}: one-hot weight is not the single atom")
            a = fw(x, wi, T - 1, s, lib=lib)
            if not np.array_equal(fw(x, wi * 8.0, T - 1, s, lib=lib), a):
                raise AssertionError(f"weighted kind {kind} s={s}: not invariant under weight scaling")
            rep = np.repeat(x, wi.astype(np.int64), axis=1)
            _close(a, f(rep, T - 1, s, lib=lib), 1e-12, 1e-15, what=f"weighted kind {kind} s={s} vs repetition")


ALL_PINS = [
    pin_hand_worked, pin_brute_force, pin_lag_subset, pin_fft, pin_constant_velocity,
    pin_zero_lag, pin_single_origin, pin_invariants, pin_stride_split,
    pin_gk_closed_forms, pin_einstein_exact, pin_random_walk, pin_ou,
    pin_einstein_vs_green_kubo, pin_xcf_brute_force, pin_xcf_fft, pin_xcf_closed_forms,
    pin_collective, pin_weighted,
]
