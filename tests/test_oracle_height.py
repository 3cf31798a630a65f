"""Pins for the oracle's height-change counters: the origin's absolute height and the total
(CPU only).

Slopes fix heights only up to a constant (the roughness sets h(0,0) = 0), so the growth
velocity, the rate of change of the absolute mean height, needs one absolute height carried
along: the origin's, counted +2 per deposition and -2 per removal at site (0, 0).  From the
flat start h(x,y) = (x + y) & 1 (h(0,0) = 0) the absolute mean height is then
<h> = h00 + S1/N with S1 the roughness sum (relative to h(0,0)).  Pinned by: the p = 1 closed
form (every site deposits once per MCS: h00 = 2t, total 2Nt); the site-by-site prediction of
the first MCS in height variables from the raw draws; and the conservation identity
N h00 + S1 = N/2 + (total height change), which ties the local counter to the global one
through the slope state.
"""
import math

import numpy as np
import pytest

import oracle as o


def flat_heights(X, Y):
    return ((np.arange(X)[None, :] + np.arange(Y)[:, None]) & 1).astype(np.int64)


@pytest.mark.parametrize("X,Y", [(64, 64), (34, 130)])
@pytest.mark.parametrize("mode", [o.DYADIC, o.UNIFORM32])
def test_p1_closed_form(X, Y, mode):
    bx, by = o.init_flat_rect(X, Y)
    h00 = tot = 0
    for t in range(1, 5):
        a, b = o.run_rect_counted(bx, by, 1, 1.0, 0.25, mode=mode, t0=t - 1, n_mcs=1)
        h00 += a
        tot += b
        assert h00 == 2 * t and tot == 2 * X * Y * t


@pytest.mark.parametrize("X,Y,p,q,mode", [(64, 64, 0.75, 0.25, o.DYADIC), (66, 10, 0.6, 0.3, o.UNIFORM32),
                                          (128, 6, 0.5, 0.0, o.DYADIC)])
def test_first_mcs_heights_match_prediction(X, Y, p, q, mode):
    """After one MCS from flat, the counters equal the absolute heights rebuilt site by site
    from the raw draws (even sites deposit with p; an odd site then deposits if all four even
    neighbours did, is removed with q if none did)."""
    n_draws = max(o.dyadic_split(p)[1], o.dyadic_split(q)[1]) if mode == o.DYADIC else 0

    def acc(seed, s, x, y, r):
        if mode == o.DYADIC:
            if r in (0.0, 1.0):
                return int(r)
            P, n = o.dyadic_split(r)
            bits = [o.word_draw_bit(X, seed, 0, s, i, x, y) for i in range(1, n + 1)]
            R = 0
            for b in bits:
                R = 2 * R + b
            return int(R >= 2 ** n - P)
        return int(o.site_uniform(X, seed, 0, s, x, y) < math.floor(r * 2.0 ** 32))

    seed = 17
    h = flat_heights(X, Y)
    for y in range(Y):
        for x in range(X):
            if (x + y) % 2 == 0 and acc(seed, 0, x, y, p):
                h[y, x] += 2
    g = h.copy()
    for y in range(Y):
        for x in range(X):
            if (x + y) % 2 == 1:
                nb = [h[y, (x + 1) % X], h[y, (x - 1) % X], h[(y + 1) % Y, x], h[(y - 1) % Y, x]]
                if all(v == h[y, x] + 1 for v in nb) and acc(seed, 1, x, y, p):
                    g[y, x] += 2
                elif all(v == h[y, x] - 1 for v in nb) and acc(seed, 1, x, y, q):
                    g[y, x] -= 2
    assert n_draws >= 0
    bx, by = o.init_flat_rect(X, Y)
    org, tot = o.run_rect_counted(bx, by, seed, p, q, mode=mode, t0=0, n_mcs=1)
    assert org == g[0, 0]
    assert tot == int((g - flat_heights(X, Y)).sum())


@pytest.mark.parametrize("X,Y,p,q", [(64, 64, 0.75, 0.25), (96, 34, 0.5, 0.0), (34, 66, 0.3, 0.7),
                                     (130, 12, 0.6, 0.35)])
def test_conservation_identity(X, Y, p, q):
    """N h00 + S1 = N/2 + total: the absolute height sum from the origin's counter and the
    relative sum S1 equals the flat start's sum (N/2) plus every height change."""
    bx, by = o.init_flat_rect(X, Y)
    N = X * Y
    h00 = tot = t = 0
    for tt in (1, 3, 8, 20):
        a, b = o.run_rect_counted(bx, by, 23, p, q, t0=t, n_mcs=tt - t)
        t = tt
        h00 += a
        tot += b
        S1 = o.observe_rect(bx, by)["S1"]
        assert N * h00 + S1 == N // 2 + tot, tt
    assert h00 != 0 and tot != 0


def test_counted_run_equals_plain_run():
    a = o.init_flat_rect(64, 40)
    b = tuple(v.copy() for v in a)
    o.run_rect(*a, 5, 0.625, 0.375, t0=0, n_mcs=6)
    o.run_rect_counted(*b, 5, 0.625, 0.375, t0=0, n_mcs=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
