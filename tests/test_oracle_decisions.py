"""Exact, site-by-site prediction of the first MCS from the flat surface (CPU only).

From h = (x+y)&1 every even site is a local minimum and every odd site a local maximum.  The
even half-step deposits at each even site whose draw accepts with p; an odd site is then a
minimum iff all four even neighbours deposited and a maximum iff none did.  This test rebuilds
each decision from the raw Philox draws with the and/or construction of Sec. III (digits of p,
draw 1 most significant) or the per-site 32-bit compare, in height variables, and checks the
oracle's state after one MCS.  It pins which draw bit belongs to which site and in which order
the draws combine, which the statistical tests cannot see.
"""
import math

import numpy as np
import pytest

import oracle as o


def xi_and_or(p, draw_bits):
    """Sec. III construction for dyadic p = 0.b_1 b_2 ... b_n (b_n = 1)."""
    if p in (0.0, 1.0):
        return int(p)
    P, n = o.dyadic_split(p)
    b = [(P >> (n - i)) & 1 for i in range(1, n + 1)]
    xi = draw_bits[n - 1]
    for i in range(n - 1, 0, -1):
        xi = (draw_bits[i - 1] | xi) if b[i - 1] else (draw_bits[i - 1] & xi)
    return xi


def accept(L, seed, t, s, x, y, r, mode, n_draws):
    if mode == o.DYADIC:
        bits = [o.word_draw_bit(L, seed, t, s, i, x, y) for i in range(1, n_draws + 1)]
        return xi_and_or(r, bits)
    return int(o.site_uniform(L, seed, t, s, x, y) < math.floor(r * 2.0 ** 32))


def predicted_first_mcs(L, seed, p, q, mode):
    n_draws = 0
    if mode == o.DYADIC:
        n_draws = max(o.dyadic_split(p)[1], o.dyadic_split(q)[1])
    h = ((np.arange(L)[None, :] + np.arange(L)[:, None]) & 1).astype(np.int64)
    for y in range(L):
        for x in range(L):
            if (x + y) & 1 == 0 and accept(L, seed, 0, 0, x, y, p, mode, n_draws):
                h[y, x] += 2
    g = h.copy()
    for y in range(L):
        for x in range(L):
            if (x + y) & 1 == 1:
                nb = [h[y, (x + 1) % L], h[y, (x - 1) % L], h[(y + 1) % L, x], h[(y - 1) % L, x]]
                if all(v == h[y, x] + 1 for v in nb) and accept(L, seed, 0, 1, x, y, p, mode, n_draws):
                    g[y, x] += 2
                elif all(v == h[y, x] - 1 for v in nb) and accept(L, seed, 0, 1, x, y, q, mode, n_draws):
                    g[y, x] -= 2
    dx = g - np.roll(g, 1, axis=1)
    dy = g - np.roll(g, 1, axis=0)
    return ((dx + 1) // 2).astype(np.uint8), ((dy + 1) // 2).astype(np.uint8)


@pytest.mark.parametrize("L,p,q,mode", [
    (64, 0.75, 0.25, o.DYADIC),
    (64, 0.625, 0.375, o.DYADIC),
    (128, 0.5, 0.0, o.DYADIC),
    (64, 0.8125, 0.0625, o.DYADIC),
    (66, 0.6, 0.3, o.UNIFORM32),
    (64, 0.875, 0.125, o.UNIFORM32),
])
def test_first_mcs_matches_site_by_site_prediction(L, p, q, mode):
    for seed in (1, 0xDEADBEEF12345):
        bx, by = o.init_flat(L)
        o.run(bx, by, seed, p, q, mode=mode, t0=0, n_mcs=1)
        ex, ey = predicted_first_mcs(L, seed, p, q, mode)
        assert np.array_equal(bx, ex) and np.array_equal(by, ey)


def test_uniform_threshold_is_strict():
    """Per-site acceptance is u < floor(p * 2^32): a probability whose threshold equals the
    site's own uniform rejects it, one ulp of 2^-32 more accepts it."""
    L, seed = 64, 77
    x, y = 10, 4                       # an even site, a minimum of the flat surface
    u = o.site_uniform(L, seed, 0, 0, x, y)
    for p, expect in ((u / 2.0 ** 32, 0), ((u + 1) / 2.0 ** 32, 1)):
        bx, by = o.init_flat(L)
        o.run(bx, by, seed, p, 0.0, mode=o.UNIFORM32, t0=0, n_mcs=1)
        ex, ey = predicted_first_mcs(L, seed, p, 0.0, o.UNIFORM32)
        assert np.array_equal(bx, ex) and np.array_equal(by, ey)
        # the even site itself: sx-(x,y) is 1 iff it deposited (its odd left neighbour cannot
        # have deposited unless all four of that site's even neighbours did)
        assert int(bx[y, x]) == expect or int(bx[y, (x - 1) % L]) == 0
