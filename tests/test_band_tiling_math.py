"""Host-side checks of the band tiling's index arithmetic (CPU only).

The tensor-core band kernel sums the origin x frame Gram entries
x_o . x_f (o an origin, f a frame of residue rho, lag m = f - o) tile by tile
into per-tile windows of band offsets, and the lag reduction reads the
windows back.  Two tilings exist:
* one CTA per 128 x 192 tile: row tile r, column tile c, frames
  k0 = r BO + c BF, entry (i, j) at lag m = c BF + j - i;
* CTA pairs (cta_group::2): row tiles 2 rp and 2 rp + 1 share the frames
  k0 = 2 rp BO + c BF, so the odd row tile holds lag m at offset
  c BF - BO + j - i; the layout has an even number of row tiles and one more
  column tile per band row, and the reduction reads odd row tiles at m + BO.
Both are rebuilt here with numpy at the kernel's tile sizes and compared with
the brute-force sum D(tau) = sum_o x_o . x_{o + tau}.  The operand layout
(tile images: K-block planes, residue-major rows, 64B swizzle) is checked to
be a bijection in which every tile is one contiguous piece.
"""
import numpy as np
import pytest

BO, BF, WP = 128, 192, 320


def cdiv(a, b):
    return -(-a // b)


def tiled_sums(x, tau_max, s, pair):
    """D(tau) through the kernel's tiling, windows and lag reduction."""
    T, K = x.shape
    n_orig = (T - 1) // s + 1
    n_res = min(s, tau_max + 1)
    m0 = tau_max // s
    n_rows = cdiv(n_orig, BO)
    if pair:
        n_rows = cdiv(n_rows, 2) * 2
        n_cols = cdiv(2 * BO + m0, BF)
    else:
        n_cols = cdiv(BO + m0, BF)
    n_k = cdiv(T, s)
    nkp = cdiv(n_k + 2 * BO, 8) * 8
    win = np.zeros((n_res, n_rows, n_cols, WP))
    i_idx = np.arange(BO)[:, None]
    for rho in range(n_res):
        n_rho = (T - 1 - rho) // s + 1 if rho <= T - 1 else 0
        m_max = (tau_max - rho) // s
        fr = np.zeros((nkp, K))            # frames of residue rho, zero past the series
        fr[:n_rho] = x[rho::s][:n_rho]
        org = np.zeros((nkp, K))           # origins o -> frame o s, zero past the last origin
        org[:n_orig] = x[0::s][:n_orig]
        for r in range(n_rows):
            for c in range(n_cols):
                if pair:
                    rp, cr = divmod(r, 2)
                    k0 = 2 * rp * BO + c * BF
                    if c * BF - 2 * BO + 1 > m_max or k0 >= n_rho:
                        continue
                    need = m_max - c * BF + 2 * BO
                    ncol = BF if need >= BF else (32 if need <= 32 else (need + 31) & ~31)
                else:
                    k0 = r * BO + c * BF
                    if c * BF - BO + 1 > m_max or k0 >= n_rho:
                        continue
                    need = m_max - c * BF + BO
                    ncol = BF if need >= BF else (16 if need <= 16 else (need + 15) & ~15)
                o0 = r * BO
                assert o0 + BO <= nkp and k0 + ncol <= nkp        # every load stays in its residue's rows
                G = org[o0:o0 + BO] @ fr[k0:k0 + ncol].T
                j_idx = np.arange(ncol)[None, :]
                m = (k0 - o0) + j_idx - i_idx
                keep = (m >= 0) & (m <= m_max) & (o0 + i_idx < n_orig)
                w = j_idx - i_idx + BO - 1
                assert w.min() >= 0 and w.max() < WP
                np.add.at(win[rho, r, c], w[keep], G[keep])
    out = np.zeros(tau_max + 1)
    for tau in range(tau_max + 1):
        rho, m = tau % s, tau // s
        parities = ((0, 2, 0), (1, 2, BO)) if pair else ((0, 1, 0),)   # (first row, row step, lag shift)
        total = 0.0
        for cr, step, shift in parities:
            mp = m + shift
            c_lo, c_hi = mp // BF, min((mp + BO - 1) // BF, n_cols - 1)
            rows = range(cr, n_rows, step)
            for rr in rows:
                for c in range(c_lo, c_hi + 1):
                    total += win[rho, rr, c, mp - c * BF + BO - 1]
        out[tau] = total
    return out


def brute_sums(x, tau_max, s):
    T = x.shape[0]
    n_orig = (T - 1) // s + 1
    out = np.zeros(tau_max + 1)
    for tau in range(tau_max + 1):
        no = min((T - 1 - tau) // s + 1, n_orig)
        o = np.arange(no) * s
        out[tau] = np.sum(x[o] * x[o + tau])
    return out


SHAPES = [  # (T, K, tau_max, stride): odd and even row-tile counts, narrow last columns, residues
    (1, 3, 0, 1), (129, 6, 128, 1), (300, 6, 299, 1), (300, 6, 50, 1), (500, 9, 200, 3),
    (700, 3, 650, 1), (900, 6, 700, 2), (257, 3, 256, 200), (400, 3, 399, 7), (1000, 3, 380, 1),
]


@pytest.mark.parametrize("pair", [False, True], ids=["one_cta", "cta_pair"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda t: "T%d_K%d_tm%d_s%d" % t)
def test_tiling_reproduces_lag_sums(shape, pair):
    T, K, tm, s = shape
    rng = np.random.default_rng(T * 31 + K * 7 + tm + s)
    x = rng.normal(size=(T, K))
    got = tiled_sums(x, tm, s, pair)
    ref = brute_sums(x, tm, s)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9 * max(1.0, np.abs(ref).max()))


def tile_byte(t, k, s, nkp, rows, esize):
    """Byte of element (frame t, K index k) in the tile images (the split kernel's store)."""
    bke = 64 // esize
    R = (t % s) * nkp + t // s
    kb, kin = k // bke, k % bke
    chunk, within = (kin * esize) // 16, (kin * esize) % 16
    return (kb * rows + R) * 64 + ((chunk ^ ((R >> 1) & 3)) << 4) + within


@pytest.mark.parametrize("esize", [2, 4], ids=["fp16_bf16", "tf32"])
@pytest.mark.parametrize("T,K,s", [(37, 70, 1), (50, 33, 3), (20, 64, 7)])
def test_tile_images_are_a_bijection_with_contiguous_tiles(T, K, s, esize):
    bke = 64 // esize
    Kp = cdiv(K, 64) * 64
    n_k = cdiv(T, s)
    nkp = cdiv(n_k + 2 * BO, 8) * 8
    rows = s * nkp
    t = np.arange(T)[:, None]
    k = np.arange(Kp)[None, :]
    b = tile_byte(t, k, s, nkp, rows, esize)
    assert len(np.unique(b)) == b.size                         # no two elements share a byte
    assert b.min() >= 0 and b.max() + esize <= (Kp // bke) * rows * 64
    # a tile: rows R0 .. R0 + n - 1 of one residue (R0 a multiple of 8) in one K-block is the
    # contiguous range [(kb rows + R0) 64, + n 64), each row's chunks permuted within its 64 bytes
    for rho in range(min(s, T)):
        for kb in range(Kp // bke):
            kk = np.arange(n_k)
            tt = rho + kk * s
            live = tt < T
            R = rho * nkp + kk[live]
            kcols = kb * bke + np.arange(bke)
            bb = tile_byte(tt[live][:, None], kcols[None, :], s, nkp, rows, esize)
            first = (kb * rows + rho * nkp) * 64
            starts = (bb.min(axis=1) - first) // 64
            assert np.array_equal(starts, R - rho * nkp)        # row R of the tile at 64 (R - R0)
            assert np.all(bb.max(axis=1) - bb.min(axis=1) == 64 - esize)
