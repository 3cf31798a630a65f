"""CPU model of the register-wavefront update on height bits (the algorithm of the GPU kernel
k_wave, restated in numpy), checked against the oracle bit for bit.

The model keeps, per row, one word of h mod 4 bits per sublattice (b = ((h - parity)/2) mod 2),
integrates the first row of a warp tile along x and every further row down y from the sy-
slopes, runs 2K half-steps as a wavefront over a band with 2K + 2 halo rows above and 2K below,
tests local minima / maxima as "b xor b(n) == s for all four neighbours" and converts the final
rows back to canonical slope words.  32-lane tiles with one halo word on each side and bands
that wrap the torus are modelled as on the GPU, with one or four words per lane.  A mistake in the representation (a wrong
parity, a swapped minimum / maximum, a wrong shifted neighbour, a missing halo row) changes
the result and fails here without a GPU.
"""
import numpy as np
import pytest

import oracle as o

M = 0xFFFFFFFF


def _fsr(lo, hi):
    return ((lo >> 1) | (hi << 31)) & M


def _fsl(lo, hi):
    return ((hi << 1) | (lo >> 31)) & M


def _prefix_xor(g):
    for d in (1, 2, 4, 8, 16):
        g = g ^ ((g << d) & M)
    return g


def _prev_w(v, V):
    """Word w-1 of a tile's 32 V words (lane 0's first word reads its own lane's last word,
    as the lane shuffle gives lane 0 its own value)."""
    return np.concatenate([v[V - 1:V], v[:-1]])


def _next_w(v, V):
    """Word w+1 (lane 31's last word reads its own lane's first word)."""
    return np.concatenate([v[1:], v[31 * V:31 * V + 1]])


def wave_model(src, L, K, nbands, dp, dq, V=1):
    """V words per lane: a tile is 32 V consecutive words, lanes 0 and 31 (V words each) halo."""
    W = L // 64
    S = 2 * K
    plane = L * W
    dst = np.zeros_like(src)
    written = np.zeros(src.shape, np.int64)
    ncols = (W + 30 * V - 1) // (30 * V)
    words = np.arange(32 * V)
    lanes = words // V
    for band in range(nbands):
        y0 = 2 * ((band * (L // 2)) // nbands)
        y1 = 2 * (((band + 1) * (L // 2)) // nbands)
        NR = y1 - y0 + 4 * K + 2
        first = (y0 + 2 * L - 2 * K - 2) % L
        for col in range(ncols):
            jj = col * 30 * V - V + words
            j = jj % W
            own = (lanes >= 1) & (lanes <= 30) & (jj < W)
            rows = [None] * NR
            # first row (even): b_e(k) = b_e(k-1) ^ sx0(k) ^ ~sx1(k-1), prefix across the tile
            sx0 = src[0 * plane + first * W + j]
            nsx1 = (~src[2 * plane + first * W + j]) & M
            pre = _prefix_xor(sx0 ^ _fsl(_prev_w(nsx1, V), nsx1))
            par = pre >> 31
            incl = np.bitwise_xor.accumulate(par)        # parity of the words up to this one
            pre = pre ^ np.where((incl ^ par) == 1, M, 0).astype(np.uint64)
            rows[0] = [pre, pre ^ nsx1]
            for R in range(1, NR):
                y = (first + R) % L
                sy0 = src[1 * plane + y * W + j]
                sy1 = src[3 * plane + y * W + j]
                rows[R] = [rows[R - 1][1] ^ sy0, (~(rows[R - 1][0] ^ sy1)) & M]
            # wavefront: at position R, half-step i on row R - i
            for R in range(NR):
                rs = ((R + 1) & 1) == 1
                for i in range(1, S + 1):
                    r = R - i
                    if r - 1 < 0:
                        continue            # rows above the band: never valid, not needed
                    s = (i - 1) & 1
                    ns = s ^ 1
                    b = rows[r][s]
                    up, dn, mid = rows[r - 1][ns], rows[r + 1][ns], rows[r][ns]
                    side = _fsr(mid, _next_w(mid, V)) if rs else _fsl(_prev_w(mid, V), mid)
                    e_or = (b ^ up) | (b ^ dn) | (b ^ mid) | (b ^ side)
                    e_and = (b ^ up) & (b ^ dn) & (b ^ mid) & (b ^ side)
                    is_min = ((~e_or) & M) if s == 0 else e_and
                    is_max = e_and if s == 0 else ((~e_or) & M)
                    m = (is_min if dp else 0) | (is_max if dq else 0)
                    rows[r][s] = b ^ m
            for r in range(4 * K + 2 - S, NR - S):
                y = y0 + r - 2 * K - 2
                hr, hp = rows[r], rows[r - 1]
                sy0 = hr[0] ^ hp[1]
                sy1 = (~(hr[1] ^ hp[0])) & M
                if (r & 1) == 0:
                    sx0 = hr[0] ^ _fsl(_prev_w(hr[1], V), hr[1])
                    sx1 = (~(hr[1] ^ hr[0])) & M
                else:
                    sx0 = hr[0] ^ hr[1]
                    sx1 = (~(hr[1] ^ _fsl(_prev_w(hr[0], V), hr[0]))) & M
                for pl, v in ((0, sx0), (1, sy0), (2, sx1), (3, sy1)):
                    idx = pl * plane + y * W + j[own]
                    dst[idx] = v[own]
                    written[idx] += 1
    assert (written == 1).all()
    return dst


@pytest.mark.parametrize("L,K,nbands,dp,dq,V", [
    (64, 4, 2, 1, 0, 1), (128, 2, 3, 1, 0, 1), (192, 8, 1, 1, 1, 1), (320, 8, 7, 0, 1, 1),
    (2048, 4, 5, 1, 0, 1), (448, 4, 3, 1, 1, 1), (256, 1, 128, 1, 0, 1),
    # four words per lane (sector-aligned 120-word tiles): one tile wider than the row, exactly
    # one tile, and columns that wrap around the lattice
    (256, 1, 4, 1, 0, 4), (512, 2, 3, 0, 1, 4), (768, 2, 2, 1, 1, 4), (8192, 1, 4, 1, 0, 4),
])
def test_height_bit_wavefront_equals_oracle(L, K, nbands, dp, dq, V):
    bx, by = o.init_flat(L)
    o.run(bx, by, 5, 0.75, 0.25, t0=0, n_mcs=7 if L <= 2048 else 2)   # a rough surface
    start = o.pack(bx, by).astype(np.uint64)
    got = wave_model(start.copy(), L, K, nbands, dp, dq, V)
    bx2, by2 = o.unpack(L, start.astype(np.uint32))
    o.run(bx2, by2, 5, float(dp), float(dq), t0=100, n_mcs=K)
    assert np.array_equal(got.astype(np.uint32), o.pack(bx2, by2))


def test_model_catches_a_swapped_extremum():
    """The same model with local minima and maxima swapped disagrees with the oracle."""
    L, K = 128, 2
    bx, by = o.init_flat(L)
    o.run(bx, by, 5, 0.75, 0.25, t0=0, n_mcs=7)
    start = o.pack(bx, by).astype(np.uint64)
    wrong = wave_model(start.copy(), L, K, 2, 0, 1)      # removal only, where p = 1 was meant
    bx2, by2 = o.unpack(L, start.astype(np.uint32))
    o.run(bx2, by2, 5, 1.0, 0.0, t0=100, n_mcs=K)
    assert not np.array_equal(wrong.astype(np.uint32), o.pack(bx2, by2))
