"""Host-side check of the polyphase recast used for small K (CPU only).

With L phases, Y[j][(series, p)] = a_series(p L + j) (zero past T, each series
padded to Pp >= P + nq slots) and M_q = sum_p Y[.][p] Y[.][p+q]^T, entry (j, j')
of M_q sums a(t) a(t + tau) over origins t = p L + j with tau = q L + j' - j.
The kernel reads M_q's B operand from copy r = q mod 8 of Y pre-shifted by r
elements at aligned offset q - r, tiles M_q into 3 x 2 blocks of 128 x 192, and
the reduction finds lag tau in block (q, h, c) at window slot
w = tau - (q L + 192 c - 128 h) + 127.  This test rebuilds all of that with
numpy on a small case (scaled-down tiles) and compares with brute force.
"""
import numpy as np
import pytest


def brute_acf_sums(a, tau_max):
    T = a.shape[0]
    return np.array([(a[:T - tau] * a[tau:]).sum() for tau in range(tau_max + 1)])


@pytest.mark.parametrize("T,nser,tau_max,BO,BF", [
    (200, 3, 60, 4, 6), (97, 2, 40, 4, 6), (300, 1, 299, 8, 12), (120, 3, 30, 2, 3),
])
def test_polyphase_blocks_reproduce_lag_sums(T, nser, tau_max, BO, BF):
    L = 3 * BO
    assert L == 2 * BF
    rng = np.random.default_rng(T + nser)
    a = rng.normal(size=(T, nser))
    P = -(-T // L)
    nq = (tau_max + L - 1) // L + 1
    Pp = P + nq + 1
    Kp = nser * Pp
    Kalloc = Kp + nq + 8
    Y = np.zeros((L, Kalloc))
    for ser in range(nser):
        for p in range(P):
            for j in range(L):
                t = p * L + j
                if t < T:
                    Y[j, ser * Pp + p] = a[t, ser]
    copies = [np.concatenate([Y[:, r:], np.zeros((L, r))], axis=1) for r in range(8)]
    WP = BO + BF - 1
    windows = {}
    for q in range(nq):
        r, bx = q % 8, q - q % 8
        B = copies[r][:, bx:bx + Kp]                      # Y[j'][k + q] for k < Kp
        M = Y[:, :Kp] @ B.T                               # M_q[j][j']
        for h in range(3):
            for c in range(2):
                blk = M[BO * h:BO * h + BO, BF * c:BF * c + BF]
                moff = q * L + BF * c - BO * h
                win = np.zeros(WP)
                for i in range(BO):
                    for j in range(BF):
                        m = moff + j - i
                        if 0 <= m <= tau_max:
                            win[j - i + BO - 1] += blk[i, j]
                windows[(q, h, c)] = win
    got = np.zeros(tau_max + 1)
    for tau in range(tau_max + 1):
        for h in range(3):
            for c in range(2):
                base = tau + BO * h - BF * c + (BO - 1)
                for cand in range(2):
                    q = base // L - cand
                    if q < 0 or q >= nq:
                        continue
                    w = base - q * L
                    if 0 <= w <= BO + BF - 2:
                        got[tau] += windows[(q, h, c)][w]
    want = brute_acf_sums(a, tau_max)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
