"""Pins for the oracle's dynamics, layout and observables (CPU only).

Each test checks the oracle against something other than itself: a closed form, an invariant
that the model fixes, a symmetry, a brute-force enumeration of the Markov chain written in
height variables (not slope bits), or an independent numpy restatement of a definition.

Paper passages (arXiv 1606.00310): Sec. I.A Eq. (1) (Kawasaki rules, p/q, periodic boundaries),
Sec. I.A (even sublattice first, then odd), Sec. II.A (slope bits, sx+(x,y) = sx-(x+1,y),
sy+(x,y) = sy-(x,y+1)), Sec. II.B Eqs. (2)-(4) (update masks), Sec. III (dyadic and/or
construction of random bits), Sec. I.A (KPZ roughening for q = 0, Edwards-Wilkinson for p = q).
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import oracle as o


# ----------------------------------------------------------------------------- helpers (test)

def slopes_from_heights(h):
    """bx(x,y) = (h(x,y) - h(x-1,y) + 1)/2, by(x,y) = (h(x,y) - h(x,y-1) + 1)/2 (periodic)."""
    dx = h - np.roll(h, 1, axis=1)
    dy = h - np.roll(h, 1, axis=0)
    assert np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1)
    return ((dx + 1) // 2).astype(np.uint8), ((dy + 1) // 2).astype(np.uint8)


def heights_numpy(bx, by):
    """Independent restatement: h(0,0)=0, column 0 from sy-, rows from sx-."""
    sx = 2 * bx.astype(np.int64) - 1
    sy = 2 * by.astype(np.int64) - 1
    col0 = np.concatenate([[0], np.cumsum(sy[1:, 0])])
    rows = np.concatenate([np.zeros((bx.shape[0], 1), np.int64), np.cumsum(sx[:, 1:], axis=1)],
                          axis=1)
    return col0[:, None] + rows


def pack_numpy(bx, by):
    """Independent restatement of the canonical layout: site k of sublattice s in row y is
    x = 2k + ((s + y) & 1); word j = k >> 5, bit k & 31; order [s][d][y][j]."""
    L = bx.shape[0]
    W = (L // 2 + 31) // 32
    words = np.zeros((2, 2, L, W), dtype=np.uint64)
    for s in (0, 1):
        for y in range(L):
            for k in range(L // 2):
                x = 2 * k + ((s + y) & 1)
                words[s, 0, y, k >> 5] |= int(bx[y, x]) << (k & 31)
                words[s, 1, y, k >> 5] |= int(by[y, x]) << (k & 31)
    return words.astype(np.uint32).reshape(-1)


def rough_state(L, seed=3, n=7, p=0.5, q=0.25):
    bx, by = o.init_flat(L)
    o.run(bx, by, seed, p, q, n_mcs=n)
    return bx, by


# ----------------------------------------------------------------------------- layout

@pytest.mark.parametrize("L", [2, 4, 6, 64, 130])
def test_flat_pack_closed_form(L):
    """Flat h = (x+y)&1: every even site has sx- = sy- = -1, every odd site +1, so sublattice 0
    words are all zero and sublattice 1 words have their L/2 valid bits set."""
    bx, by = o.init_flat(L)
    h = (np.arange(L)[None, :] + np.arange(L)[:, None]) & 1
    ebx, eby = slopes_from_heights(h)
    assert np.array_equal(bx, ebx) and np.array_equal(by, eby)
    W = o.words_per_row(L)
    w = o.pack(bx, by).reshape(2, 2, L, W)
    assert np.all(w[0] == 0)
    full = np.zeros(W, dtype=np.uint64)
    for k in range(L // 2):
        full[k >> 5] |= 1 << (k & 31)
    assert np.all(w[1] == full.astype(np.uint32)[None, None, :])


@pytest.mark.parametrize("L", [4, 10, 64, 96])
def test_pack_matches_layout_definition_and_round_trips(L):
    bx, by = rough_state(L)
    w = o.pack(bx, by)
    assert np.array_equal(w, pack_numpy(bx, by))
    bx2, by2 = o.unpack(L, w)
    assert np.array_equal(bx, bx2) and np.array_equal(by, by2)


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("q", [0.0, 0.25, 1.0])
@pytest.mark.parametrize("mode", [o.DYADIC, o.UNIFORM32])
def test_p1_closed_form_from_flat(q, mode):
    """p = 1 from flat: every even site is a minimum and deposits, then every odd site is a
    minimum and deposits, so after each whole MCS the slopes equal the initial slopes and
    W^2 = 1/4 (num = N^2 / 4) at every t, whatever q is."""
    L = 64
    bx, by = o.init_flat(L)
    w0 = o.pack(bx, by)
    for t in range(6):
        o.run(bx, by, 1, 1.0, q, mode=mode, t0=t, n_mcs=1)
        assert np.array_equal(o.pack(bx, by), w0)
        r = o.observe(bx, by)
        assert r["num"] == r["N"] ** 2 // 4 and 4 * r["num"] == r["N"] ** 2


def test_p0_q0_is_identity():
    bx, by = rough_state(32)
    w = o.pack(bx, by)
    o.run(bx, by, 5, 0.0, 0.0, t0=7, n_mcs=5)
    assert np.array_equal(o.pack(bx, by), w)


@pytest.mark.parametrize("p,q", [(0.75, 0.25), (0.5, 0.0), (0.6, 0.3), (0.875, 0.125)])
def test_complement_symmetry(p, q):
    """Complementing every slope bit swaps minima and maxima, so running (q, p) on the
    complement is the complement of running (p, q), draw for draw (the two processes share
    their random numbers)."""
    L = 48
    bx, by = rough_state(L, seed=11)
    cx, cy = 1 - bx, 1 - by
    o.run(bx, by, 21, p, q, t0=3, n_mcs=4)
    o.run(cx, cy, 21, q, p, t0=3, n_mcs=4)
    assert np.array_equal(cx, 1 - bx) and np.array_equal(cy, 1 - by)


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("p,q,mode", [(0.5, 0.0, o.DYADIC), (0.75, 0.25, o.DYADIC),
                                      (0.7, 0.2, o.UNIFORM32)])
def test_invariants_hold_every_step(p, q, mode):
    """Slope sums vanish around every row and column (periodic surface), every plaquette
    closes, heights are single-valued and h = x + y (mod 2)."""
    L = 40
    bx, by = o.init_flat(L)
    for t in range(12):
        o.run(bx, by, 8, p, q, mode=mode, t0=t, n_mcs=1)
        assert np.all(bx.sum(axis=1) == L // 2)
        assert np.all(by.sum(axis=0) == L // 2)
        sx = 2 * bx.astype(int) - 1
        sy = 2 * by.astype(int) - 1
        # sx(x+1,y) + sy(x+1,y+1) == sy(x,y+1) + sx(x+1,y+1)
        lhs = np.roll(sx, -1, 1) + np.roll(np.roll(sy, -1, 1), -1, 0)
        rhs = np.roll(sy, -1, 0) + np.roll(np.roll(sx, -1, 1), -1, 0)
        assert np.array_equal(lhs, rhs)
        h = o.heights(bx, by)
        assert np.array_equal(h, heights_numpy(bx, by))
        xy = np.arange(L)[None, :] + np.arange(L)[:, None]
        assert np.all((h - xy) % 2 == 0)
        bx2, by2 = slopes_from_heights(h)
        assert np.array_equal(bx, bx2) and np.array_equal(by, by2)


def test_observe_matches_exact_integer_definition():
    for L, n in [(16, 3), (40, 9), (64, 20)]:
        bx, by = rough_state(L, n=n)
        h = heights_numpy(bx, by)
        S1 = int(h.sum())
        S2 = int((h.astype(object) ** 2).sum())
        N = L * L
        r = o.observe(bx, by)
        assert (r["S1"], r["S2"], r["num"], r["N"]) == (S1, S2, N * S2 - S1 * S1, N)
        assert math.isclose(r["num"] / N ** 2, float(np.var(h)), rel_tol=1e-12)


def test_observe_rejects_non_closing_slopes():
    bx, by = o.init_flat(8)
    bx[3, 2] ^= 1
    with pytest.raises(ValueError):
        o.observe(bx, by)


# ----------------------------------------------------------------------------- random bits

@pytest.mark.parametrize("n", range(1, 9))
def test_dyadic_and_or_construction_equals_integer_compare(n):
    """Sec. III builds xi_r for dyadic r from a few random words with and/or.  With binary
    digits b_1..b_n of p (b_n = 1): xi = r_n; for i = n-1..1: xi = b_i ? (r_i | xi) : (r_i & xi).
    For every P and every draw pattern this equals the oracle's test R >= 2^n - P."""
    for P in range(1, 2 ** n, 2):
        b = [(P >> (n - i)) & 1 for i in range(1, n + 1)]
        for R in range(2 ** n):
            r = [(R >> (n - i)) & 1 for i in range(1, n + 1)]
            xi = r[n - 1]
            for i in range(n - 1, 0, -1):
                xi = (r[i - 1] | xi) if b[i - 1] else (r[i - 1] & xi)
            assert xi == (1 if R >= 2 ** n - P else 0)
    assert sum(1 for R in range(2 ** n) if R >= 2 ** n - 1) == 1


def test_dyadic_split():
    assert o.dyadic_split(0.75) == (3, 2)
    assert o.dyadic_split(0.125) == (1, 3)
    assert o.dyadic_split(0.875) == (7, 3)
    assert o.dyadic_split(1.0) == (1, 0)
    assert o.dyadic_split(0.0) == (0, 0)
    assert o.dyadic_split(2.0 ** -32) == (1, 32)
    assert o.dyadic_split(0.3) is None
    assert o.dyadic_split(2.0 ** -33) is None


@pytest.mark.parametrize("p,mode", [(0.75, o.DYADIC), (0.375, o.DYADIC), (0.3, o.UNIFORM32),
                                    (0.95, o.UNIFORM32)])
def test_one_mcs_acceptance_frequency(p, mode):
    """From flat with q = 0, every even site is a minimum and deposits with probability p; an
    odd site then deposits (probability p) only if all four even neighbours did, which flips
    the shared slope back.  So after one MCS sx-(x,y) = 1 at an even site with probability
    p - p^5 exactly."""
    L = 128
    hits = 0
    n = 0
    ev = ((np.arange(L)[None, :] + np.arange(L)[:, None]) & 1) == 0
    for seed in range(4):
        bx, by = o.init_flat(L)
        o.run(bx, by, seed, p, 0.0, mode=mode, n_mcs=1)
        hits += int(bx[ev].sum())
        n += int(ev.sum())
    expect = p - p ** 5
    sigma = math.sqrt(expect * (1 - expect) / n)
    assert abs(hits / n - expect) < 6 * sigma, (hits / n, expect)


# ----------------------------------------------------------------------------- brute force

def _neighbours(x, y, L):
    return [((x + 1) % L, y), ((x - 1) % L, y), (x, (y + 1) % L), (x, (y - 1) % L)]


def _half_step_distribution(h, s, p, q):
    """Exact distribution after updating sublattice s of height field h (dict: heights -> prob).
    A site is a local minimum if its four neighbours are one higher (deposit with p, h += 2),
    a local maximum if they are one lower (remove with q, h -= 2)."""
    L = h.shape[0]
    cand = []
    for y in range(L):
        for x in range(L):
            if (x + y) & 1 != s:
                continue
            nb = [h[yy, xx] for (xx, yy) in _neighbours(x, y, L)]
            if all(v == h[y, x] + 1 for v in nb):
                cand.append((x, y, +2, p))
            elif all(v == h[y, x] - 1 for v in nb):
                cand.append((x, y, -2, q))
    out = {}
    for flips in itertools.product((0, 1), repeat=len(cand)):
        pr = 1.0
        g = h.copy()
        for f, (x, y, dh, r) in zip(flips, cand):
            pr *= r if f else (1 - r)
            if f:
                g[y, x] += dh
        if pr == 0.0:
            continue
        key = g.tobytes()
        out[key] = out.get(key, 0.0) + pr
    return out


def _exact_mcs_distribution(h0, p, q, n_mcs):
    L = h0.shape[0]
    dist = {h0.tobytes(): 1.0}
    for _ in range(n_mcs):
        for s in (0, 1):
            nd = {}
            for key, pr in dist.items():
                h = np.frombuffer(key, dtype=np.int64).reshape(L, L)
                for k2, p2 in _half_step_distribution(h, s, p, q).items():
                    nd[k2] = nd.get(k2, 0.0) + pr * p2
            dist = nd
    # states are slope configurations: heights modulo a global shift
    sl = {}
    for key, pr in dist.items():
        h = np.frombuffer(key, dtype=np.int64).reshape(L, L)
        bx, by = slopes_from_heights(h)
        k = bx.tobytes() + by.tobytes()
        sl[k] = sl.get(k, 0.0) + pr
    return sl


@pytest.mark.parametrize("p,q,mode", [(0.75, 0.25, o.DYADIC), (0.6, 0.3, o.UNIFORM32)])
def test_4x4_transition_frequencies_match_enumerated_chain(p, q, mode):
    """4x4 torus, two MCS from flat: the exact distribution over slope configurations is
    enumerated in height variables; the oracle's frequencies over many seeds must pass a
    chi-square test against it."""
    scipy_stats = pytest.importorskip("scipy.stats")
    L, n_mcs, n_seeds = 4, 2, 20000
    h0 = ((np.arange(L)[None, :] + np.arange(L)[:, None]) & 1).astype(np.int64)
    exact = _exact_mcs_distribution(h0, p, q, n_mcs)
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    counts = Counter()
    for seed in range(n_seeds):
        bx, by = o.init_flat(L)
        o.run(bx, by, seed, p, q, mode=mode, n_mcs=n_mcs)
        counts[bx.tobytes() + by.tobytes()] += 1
    assert set(counts) <= set(exact), "oracle reached a state the chain cannot reach"
    keys = sorted(exact, key=lambda k: -exact[k])
    obs, exp = [], []
    rest_o, rest_e = 0, 0.0
    for k in keys:
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
    pval = scipy_stats.chi2.sf(chi2, len(obs) - 1)
    assert len(obs) > 10
    assert pval > 1e-4, (chi2, len(obs), pval)


# ----------------------------------------------------------------------------- band variant

@pytest.mark.parametrize("n_mcs", [1, 2, 3])
def test_band_run_equals_full_run_interior(n_mcs):
    L, p, q = 64, 0.75, 0.25
    bx, by = o.init_flat(L)
    o.run(bx, by, 4, p, q, t0=0, n_mcs=n_mcs)
    for y_first in (0, 50, 60):
        nrows = 4 * n_mcs + 6
        gx, gy = o.init_flat_band(L, y_first, nrows)
        o.run_band(L, y_first, gx, gy, 4, p, q, t0=0, n_mcs=n_mcs)
        for i in range(2 * n_mcs, nrows - 2 * n_mcs):
            y = (y_first + i) % L
            assert np.array_equal(gx[i], bx[y]) and np.array_equal(gy[i], by[y]), (y_first, i)


# ----------------------------------------------------------------------------- statistics

def _w2_curve(L, p, q, times, seeds):
    w2 = np.zeros(len(times))
    for seed in seeds:
        bx, by = o.init_flat(L)
        t = 0
        for i, tt in enumerate(times):
            o.run(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
            t = tt
            r = o.observe(bx, by)
            w2[i] += r["num"] / r["N"] ** 2
    return w2 / len(seeds)


def test_kpz_growth_exponent():
    """q = 0 gives KPZ roughening, W^2 ~ t^(2 beta) with beta ~ 0.24 in 2+1 dimensions
    (Sec. I.A).  Fit W^2 = A t^(2 beta) + c (c absorbs the intrinsic width) for 16 <= t <= 1024
    at L = 512 (far from saturation, t_x ~ L^1.6 ~ 2e4)."""
    optimize = pytest.importorskip("scipy.optimize")
    times = [2 ** k for k in range(11)]
    w2 = _w2_curve(512, 0.5, 0.0, times, seeds=range(1, 5))
    t = np.array(times, float)
    m = t >= 16
    popt, _ = optimize.curve_fit(lambda t, A, b, c: A * t ** (2 * b) + c, t[m], w2[m],
                                 p0=(0.3, 0.24, 0.3))
    assert abs(popt[1] - 0.24) < 0.02, popt


def test_edwards_wilkinson_log_growth():
    """p = q gives Edwards-Wilkinson roughening, which is logarithmic (Sec. I.A): W^2 rises by
    about the same amount per factor of t, unlike the KPZ power law."""
    times = [2 ** k for k in range(2, 11, 2)]
    ew = _w2_curve(256, 0.5, 0.5, times, seeds=range(1, 4))
    inc = np.diff(ew)
    assert np.all(inc > 0)
    assert inc.max() / inc.min() < 1.6, inc
    kpz = _w2_curve(256, 0.5, 0.0, times, seeds=range(1, 4))
    kinc = np.diff(kpz)
    assert kinc[-1] / kinc[0] > 2.0, kinc
