"""Host-side check of the band tiling used by every kernel (CPU only).

The kernels split a lag as tau = rho + m*s (rho = tau mod s) and cover, for
each residue rho, the band 0 <= k - o <= m_max(rho) of the origin x frame-index
plane with tiles (rho, r, c): origins [r*BO, r*BO+BO), frame indices
[r*BO + c*BF, ... + BF).  A tile keeps per-offset sums in a window indexed by
w = m - c*BF + BO - 1, and the reduction for lag tau visits the column tiles
c_lo = m // BF .. c_hi = (m + BO - 1) // BF of every row tile.  This test
enumerates the scheme on small shapes and checks that every (origin, lag)
pair with t0 + tau <= T-1 is counted exactly once, at the right window slot.
"""
import itertools

import pytest


def ceil_div(a, b):
    return -(-a // b)


def plan(T, tau_max, s, BO, BF):
    n_orig = (T - 1) // s + 1
    n_res = min(s, tau_max + 1)
    m_max0 = tau_max // s
    return dict(n_orig=n_orig, n_res=n_res, n_rows=ceil_div(n_orig, BO),
                n_cols=ceil_div(BO + m_max0, BF))


@pytest.mark.parametrize("T,tau_max,s,BO,BF", [
    (1, 0, 1, 4, 4), (10, 9, 1, 4, 4), (10, 3, 1, 4, 8), (17, 16, 3, 4, 4), (30, 12, 5, 4, 8),
    (40, 39, 7, 8, 4), (23, 5, 30, 4, 4), (64, 63, 64, 8, 8), (50, 20, 2, 8, 16), (70, 40, 1, 8, 12), (45, 30, 4, 4, 6),
])
def test_band_tiles_cover_each_pair_once(T, tau_max, s, BO, BF):
    p = plan(T, tau_max, s, BO, BF)
    seen = {}
    window = {}
    for rho, r, c in itertools.product(range(p["n_res"]), range(p["n_rows"]), range(p["n_cols"])):
        n_rho = 0 if rho > T - 1 else (T - 1 - rho) // s + 1
        m_max = (tau_max - rho) // s
        for i, j in itertools.product(range(BO), range(BF)):
            o = r * BO + i
            k = r * BO + c * BF + j
            m = k - o
            if not (o < p["n_orig"] and k < n_rho and 0 <= m <= m_max):
                continue
            tau = rho + m * s
            t0 = o * s
            assert t0 + tau == rho + k * s <= T - 1
            assert 0 <= tau <= tau_max
            seen[(t0, tau)] = seen.get((t0, tau), 0) + 1
            w = m - c * BF + BO - 1
            assert 0 <= w <= BO + BF - 2
            assert w == j - i + BO - 1
            window.setdefault((rho, r, c, w), set()).add(tau)
    want = {(t0, tau) for tau in range(tau_max + 1) for t0 in range(0, T - tau, s)}
    assert set(seen) == want
    assert all(v == 1 for v in seen.values())
    # one lag per (tile, window slot)
    assert all(len(v) == 1 for v in window.values())
    # the reduction visits exactly the tiles whose window holds the lag
    for tau in range(tau_max + 1):
        rho, m = tau % s, tau // s
        c_lo = m // BF
        c_hi = min(p["n_cols"] - 1, (m + BO - 1) // BF)
        holders = {(r, c) for (rr, r, c, w), taus in window.items() if rr == rho and tau in taus}
        assert all(c_lo <= c <= c_hi for _, c in holders)
        for r, c in holders:
            assert tau in window[(rho, r, c, m - c * BF + BO - 1)]
