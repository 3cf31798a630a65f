"""Pins for the oracle on X x Y lattices, X != Y (CPU only).

The paper names the two lateral sizes X and Y (Sec. II.B: the effective SIMD word spans X, and a
wide-system variant handles X >= 2^17) and benchmarks X = Y = L (Sec. III, Fig. 4).  These
tests check the oracle's X x Y functions against what the model fixes, independently of the
oracle's own code: the p = 1 closed form from the flat surface; the invariants of a surface
(row and column slope sums, closed plaquettes, single-valued heights of the parity of x + y);
the symmetry of the model under exchanging x and y (Eq. 1 and the sublattice schedule treat
the two directions alike), which a row count and a row length confused with each other break;
the packed layout restated in numpy; the site-by-site prediction of the first MCS from raw
draws with the counter layout's unit y * W + word (W from the row length X); the band runner;
and the enumerated Markov chain of a 6 x 4 torus.  The first tests use X < Y, so that a mutant
that wraps rows at X stays inside the arrays.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import oracle as o


def flat_heights(X, Y):
    return ((np.arange(X)[None, :] + np.arange(Y)[:, None]) & 1).astype(np.int64)


def slopes_from_heights(h):
    dx = h - np.roll(h, 1, axis=1)
    dy = h - np.roll(h, 1, axis=0)
    assert np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1)
    return ((dx + 1) // 2).astype(np.uint8), ((dy + 1) // 2).astype(np.uint8)


def heights_numpy(bx, by):
    sx = 2 * bx.astype(np.int64) - 1
    sy = 2 * by.astype(np.int64) - 1
    col0 = np.concatenate([[0], np.cumsum(sy[1:, 0])])
    rows = np.concatenate([np.zeros((bx.shape[0], 1), np.int64), np.cumsum(sx[:, 1:], axis=1)],
                          axis=1)
    return col0[:, None] + rows


def pack_numpy(bx, by):
    """The canonical layout restated: Y rows of X sites; site k of sublattice s in row y is
    x = 2k + ((s + y) & 1); word j = k >> 5, bit k & 31; order [s][d][y][j]; W = ceil(X/64)."""
    Y, X = bx.shape
    W = (X // 2 + 31) // 32
    words = np.zeros((2, 2, Y, W), dtype=np.uint64)
    for s in (0, 1):
        for y in range(Y):
            for k in range(X // 2):
                x = 2 * k + ((s + y) & 1)
                words[s, 0, y, k >> 5] |= int(bx[y, x]) << (k & 31)
                words[s, 1, y, k >> 5] |= int(by[y, x]) << (k & 31)
    return words.astype(np.uint32).reshape(-1)


def rough(X, Y, seed=3, n=5, p=0.625, q=0.375, mode=None):
    bx, by = o.init_flat_rect(X, Y)
    o.run_rect(bx, by, seed, p, q, mode=mode, n_mcs=n)
    return bx, by


def transpose(bx, by):
    """h'(x', y') = h(y', x') on the Y x X lattice: sx-' = sy- transposed and sy-' = sx-
    transposed (sublattice parity x + y is unchanged)."""
    return np.ascontiguousarray(by.T), np.ascontiguousarray(bx.T)


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("X,Y", [(4, 8), (10, 128), (64, 6), (66, 4)])
@pytest.mark.parametrize("mode", [o.DYADIC, o.UNIFORM32])
def test_p1_closed_form_from_flat(X, Y, mode):
    """p = 1 from flat on an X x Y torus: every even site deposits, then every odd site, so the
    slopes return to the flat ones after every MCS and W^2 = 1/4, i.e. num = N^2/4 with
    N = X * Y."""
    bx, by = o.init_flat_rect(X, Y)
    ex, ey = slopes_from_heights(flat_heights(X, Y))
    assert np.array_equal(bx, ex) and np.array_equal(by, ey)
    w0 = o.pack_rect(bx, by)
    for t in range(4):
        o.run_rect(bx, by, 1, 1.0, 0.25, mode=mode, t0=t, n_mcs=1)
        assert np.array_equal(o.pack_rect(bx, by), w0)
        r = o.observe_rect(bx, by)
        assert r["N"] == X * Y and 4 * r["num"] == (X * Y) ** 2


@pytest.mark.parametrize("X,Y", [(6, 10), (130, 4), (64, 2), (2, 64)])
def test_flat_pack_closed_form(X, Y):
    """Flat: sublattice 0 words all zero, sublattice 1 words with their X/2 valid bits set."""
    bx, by = o.init_flat_rect(X, Y)
    W = o.words_per_row(X)
    w = o.pack_rect(bx, by).reshape(2, 2, Y, W)
    assert np.all(w[0] == 0)
    full = np.zeros(W, dtype=np.uint64)
    for k in range(X // 2):
        full[k >> 5] |= 1 << (k & 31)
    assert np.all(w[1] == full.astype(np.uint32)[None, None, :])


@pytest.mark.parametrize("X,Y", [(10, 34), (96, 6), (130, 12)])
def test_pack_matches_layout_definition_and_round_trips(X, Y):
    bx, by = rough(X, Y)
    w = o.pack_rect(bx, by)
    assert np.array_equal(w, pack_numpy(bx, by))
    bx2, by2 = o.unpack_rect(X, Y, w)
    assert np.array_equal(bx, bx2) and np.array_equal(by, by2)


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("X,Y,p,q,mode", [(34, 96, 0.75, 0.25, o.DYADIC), (96, 34, 0.5, 0.0, o.DYADIC),
                                          (66, 20, 0.7, 0.3, o.UNIFORM32)])
def test_invariants_hold_every_step(X, Y, p, q, mode):
    """Every row's sx- slopes sum to zero (X/2 ones), every column's sy- slopes too (Y/2 ones),
    every plaquette closes, heights are single-valued and have the parity of x + y, and the
    exact sums equal their definition over the numpy heights."""
    bx, by = o.init_flat_rect(X, Y)
    for t in range(6):
        o.run_rect(bx, by, 11, p, q, mode=mode, t0=t, n_mcs=1)
        assert np.all(bx.sum(axis=1) == X // 2)
        assert np.all(by.sum(axis=0) == Y // 2)
        sx = 2 * bx.astype(np.int64) - 1
        sy = 2 * by.astype(np.int64) - 1
        # plaquette with corners (x-1, y-1), (x, y): sx(x, y) + sy(x-1, y) == sy(x, y) + sx(x, y-1)
        assert np.array_equal(sx + np.roll(sy, 1, axis=1), sy + np.roll(sx, 1, axis=0))
        h = o.heights_rect(bx, by)
        assert np.array_equal(h, heights_numpy(bx, by))
        assert np.all((h - flat_heights(X, Y)) % 2 == 0)
        r = o.observe_rect(bx, by)
        S1, S2, N = int(h.sum()), int((h.astype(object) ** 2).sum()), X * Y
        assert (r["S1"], r["S2"], r["num"]) == (S1, S2, N * S2 - S1 * S1)


# ----------------------------------------------------------------------------- x <-> y symmetry

@pytest.mark.parametrize("X,Y", [(12, 20), (20, 12), (64, 66), (130, 6)])
@pytest.mark.parametrize("p,q", [(1.0, 0.0), (0.0, 1.0), (1.0, 1.0)])
def test_transpose_commutes_with_deterministic_dynamics(X, Y, p, q):
    """Eq. (1) and the even-then-odd schedule treat x and y alike, so with deterministic rules
    (no draws) evolving a rough X x Y surface and exchanging x and y gives the same as exchanging
    first and evolving on the Y x X torus; the sums are the same too (same multiset of heights
    up to the common shift fixed by h(0,0) = 0)."""
    bx, by = rough(X, Y, seed=7, n=4)
    tx, ty = transpose(bx, by)
    for n in (1, 3):
        o.run_rect(bx, by, 5, p, q, t0=0, n_mcs=n)
        o.run_rect(tx, ty, 5, p, q, t0=0, n_mcs=n)
        ex, ey = transpose(bx, by)
        assert np.array_equal(tx, ex) and np.array_equal(ty, ey)
        a, b = o.observe_rect(bx, by), o.observe_rect(tx, ty)
        assert (a["S1"], a["S2"], a["num"]) == (b["S1"], b["S2"], b["num"])


def test_rough_surfaces_really_differ_between_shapes():
    """Guard for the symmetry test: a random rule does not commute with the exchange (the draws
    are keyed by the row-major unit), so the test above is not trivially true."""
    bx, by = rough(12, 20, seed=7, n=4)
    tx, ty = transpose(bx, by)
    o.run_rect(bx, by, 5, 0.5, 0.25, t0=0, n_mcs=2)
    o.run_rect(tx, ty, 5, 0.5, 0.25, t0=0, n_mcs=2)
    ex, ey = transpose(bx, by)
    assert not (np.array_equal(tx, ex) and np.array_equal(ty, ey))


# ----------------------------------------------------------------------------- draws

def _xi_and_or(p, draw_bits):
    if p in (0.0, 1.0):
        return int(p)
    P, n = o.dyadic_split(p)
    b = [(P >> (n - i)) & 1 for i in range(1, n + 1)]
    xi = draw_bits[n - 1]
    for i in range(n - 1, 0, -1):
        xi = (draw_bits[i - 1] | xi) if b[i - 1] else (draw_bits[i - 1] & xi)
    return xi


def _draw_bit(X, seed, t, s, draw, x, y):
    """Restated from the counter layout: unit = y * W + (k >> 5), W = ceil(X/64), k = x >> 1."""
    W = (X // 2 + 31) // 32
    k = x >> 1
    unit = y * W + (k >> 5)
    ctr = [unit >> 2, t, s | ((draw - 1) << 1), 0]
    out = o.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    return (int(out[unit & 3]) >> (k & 31)) & 1


def _site_uniform(X, seed, t, s, x, y):
    unit = y * (X // 2) + (x >> 1)
    out = o.philox4x32_10([unit >> 2, t, s, 1], [seed & 0xFFFFFFFF, seed >> 32])
    return int(out[unit & 3])


def _accept(X, seed, s, x, y, r, mode, n_draws):
    if mode == o.DYADIC:
        return _xi_and_or(r, [_draw_bit(X, seed, 0, s, i, x, y) for i in range(1, n_draws + 1)])
    return int(_site_uniform(X, seed, 0, s, x, y) < math.floor(r * 2.0 ** 32))


def _predicted_first_mcs(X, Y, seed, p, q, mode):
    n_draws = max(o.dyadic_split(p)[1], o.dyadic_split(q)[1]) if mode == o.DYADIC else 0
    h = flat_heights(X, Y)
    for y in range(Y):
        for x in range(X):
            if (x + y) & 1 == 0 and _accept(X, seed, 0, x, y, p, mode, n_draws):
                h[y, x] += 2
    g = h.copy()
    for y in range(Y):
        for x in range(X):
            if (x + y) & 1 == 1:
                nb = [h[y, (x + 1) % X], h[y, (x - 1) % X], h[(y + 1) % Y, x], h[(y - 1) % Y, x]]
                if all(v == h[y, x] + 1 for v in nb) and _accept(X, seed, 1, x, y, p, mode, n_draws):
                    g[y, x] += 2
                elif all(v == h[y, x] - 1 for v in nb) and _accept(X, seed, 1, x, y, q, mode, n_draws):
                    g[y, x] -= 2
    return slopes_from_heights(g)


@pytest.mark.parametrize("X,Y,p,q,mode", [(128, 6, 0.75, 0.25, o.DYADIC), (6, 130, 0.5, 0.0, o.DYADIC),
                                          (192, 4, 0.625, 0.125, o.DYADIC), (66, 10, 0.6, 0.3, o.UNIFORM32)])
def test_first_mcs_matches_site_by_site_prediction(X, Y, p, q, mode):
    """Each decision of the first MCS rebuilt from raw Philox draws whose counter unit uses the
    row length X (and never the row count Y)."""
    for seed in (2, 0xC0FFEE123):
        bx, by = o.init_flat_rect(X, Y)
        o.run_rect(bx, by, seed, p, q, mode=mode, t0=0, n_mcs=1)
        ex, ey = _predicted_first_mcs(X, Y, seed, p, q, mode)
        assert np.array_equal(bx, ex) and np.array_equal(by, ey)


def test_draw_functions_use_the_row_length():
    for (X, x, y) in [(128, 100, 5), (6, 3, 100), (192, 190, 3)]:
        s = (x + y) & 1
        assert o.word_draw_bit(X, 9, 0, s, 2, x, y) == _draw_bit(X, 9, 0, s, 2, x, y)
        assert o.site_uniform(X, 9, 0, s, x, y) == _site_uniform(X, 9, 0, s, x, y)


# ----------------------------------------------------------------------------- band runner

@pytest.mark.parametrize("n_mcs", [1, 2])
def test_band_run_equals_full_run_interior(n_mcs):
    X, Y, p, q = 40, 22, 0.75, 0.25
    bx, by = o.init_flat_rect(X, Y)
    o.run_rect(bx, by, 4, p, q, t0=0, n_mcs=n_mcs)
    for y_first in (0, 9, 18):
        nrows = 4 * n_mcs + 6
        gx, gy = o.init_flat_band_rect(X, Y, y_first, nrows)
        o.run_band_rect(X, Y, y_first, gx, gy, 4, p, q, t0=0, n_mcs=n_mcs)
        for i in range(2 * n_mcs, nrows - 2 * n_mcs):
            y = (y_first + i) % Y
            assert np.array_equal(gx[i], bx[y]) and np.array_equal(gy[i], by[y]), (y_first, i)


# ----------------------------------------------------------------------------- brute force

def _half_step(h, s, p, q):
    Y, X = h.shape
    cand = []
    for y in range(Y):
        for x in range(X):
            if (x + y) & 1 != s:
                continue
            nb = [h[y, (x + 1) % X], h[y, (x - 1) % X], h[(y + 1) % Y, x], h[(y - 1) % Y, x]]
            if all(v == h[y, x] + 1 for v in nb):
                cand.append((x, y, 2, p))
            elif all(v == h[y, x] - 1 for v in nb):
                cand.append((x, y, -2, q))
    out = {}
    for flips in itertools.product((0, 1), repeat=len(cand)):
        pr, g = 1.0, h.copy()
        for f, (x, y, dh, r) in zip(flips, cand):
            pr *= r if f else 1 - r
            if f:
                g[y, x] += dh
        if pr:
            out[g.tobytes()] = out.get(g.tobytes(), 0.0) + pr
    return out


def test_6x4_transition_frequencies_match_enumerated_chain():
    """6 x 4 torus (X = 6 sites per row, Y = 4 rows), one MCS from flat: the exact distribution
    over slope configurations, enumerated in height variables, against the oracle's frequencies
    over many seeds (chi-square)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    X, Y, p, q, n_seeds = 6, 4, 0.75, 0.25, 20000
    dist = {flat_heights(X, Y).tobytes(): 1.0}
    for s in (0, 1):
        nd = {}
        for key, pr in dist.items():
            for k2, p2 in _half_step(np.frombuffer(key, dtype=np.int64).reshape(Y, X), s, p, q).items():
                nd[k2] = nd.get(k2, 0.0) + pr * p2
        dist = nd
    exact = {}
    for key, pr in dist.items():
        bx, by = slopes_from_heights(np.frombuffer(key, dtype=np.int64).reshape(Y, X))
        k = bx.tobytes() + by.tobytes()
        exact[k] = exact.get(k, 0.0) + pr
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    counts = Counter()
    for seed in range(n_seeds):
        bx, by = o.init_flat_rect(X, Y)
        o.run_rect(bx, by, seed, p, q, n_mcs=1)
        counts[bx.tobytes() + by.tobytes()] += 1
    assert set(counts) <= set(exact), "oracle reached a state the chain cannot reach"
    obs, exp, rest_o, rest_e = [], [], 0, 0.0
    for k in sorted(exact, key=lambda k: -exact[k]):
        e = exact[k] * n_seeds
        if e >= 5:
            obs.append(counts.get(k, 0))
            exp.append(e)
        else:
            rest_o += counts.get(k, 0)
            rest_e += e
    if rest_e > 0:
        obs.append(rest_o)
        exp.append(rest_e)
    chi2 = sum((a - b) ** 2 / b for a, b in zip(obs, exp))
    assert len(obs) > 10
    assert scipy_stats.chi2.sf(chi2, len(obs) - 1) > 1e-4, (chi2, len(obs))
