"""Pins for the oracle's random-sequential dynamics on the local 4 x 4 encoding (CPU only).

The paper's non-vectorized comparison keeps 4 x 4 sites per 32-bit word, the encoding of choice
when sites are selected at random (Sec. II.A).  The reading taken (the paper gives no schedule):
random-sequential attempts decomposed over the 4 x 4 words, words in a checkerboard of two
phases per MCS, 16 attempts per active word, each at a uniformly drawn site of the word,
accepted with p at a local minimum and q at a local maximum (Eq. 1).

Pinned by: on a 4 x 4 torus (one word) the process is plain random-sequential dynamics, whose
one-MCS law is P1^16 with P1 the one-attempt transition (site uniform among 16), enumerated in
height variables and compared with the oracle's frequencies (chi-square); the attempts rebuilt
one by one from the raw Philox draws in height variables on multi-word lattices; the surface
invariants every step.
"""
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


def attempt(h, x, y, u, Tp, Tq):
    """One attempt at site (x, y) in height variables, acceptance number u."""
    Y, X = h.shape
    nb = [h[y, (x + 1) % X], h[y, (x - 1) % X], h[(y + 1) % Y, x], h[(y - 1) % Y, x]]
    if all(v == h[y, x] + 1 for v in nb) and u < Tp:
        h[y, x] += 2
    elif all(v == h[y, x] - 1 for v in nb) and u < Tq:
        h[y, x] -= 2


def predicted(X, Y, seed, p, q, n_mcs):
    """The process restated: MCS t, phases 0 and 1, active words (wx + wy) & 1 == phase, 16
    attempts each; attempt a of word w uses the Philox call (w, t, ph | a << 1, 2), site
    out[0] >> 28 (column i & 3, row i >> 2 of the word), acceptance out[1]."""
    Tp, Tq = math.floor(p * 2.0 ** 32), math.floor(q * 2.0 ** 32)
    h = flat_heights(X, Y)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(n_mcs):
        for ph in (0, 1):
            for wy in range(Y // 4):
                for wx in range(X // 4):
                    if (wx + wy) % 2 != ph:
                        continue
                    w = wy * (X // 4) + wx
                    for a in range(16):
                        out = o.philox4x32_10([w, t, ph | (a << 1), 2], key)
                        i = int(out[0]) >> 28
                        attempt(h, 4 * wx + (i & 3), 4 * wy + (i >> 2), int(out[1]), Tp, Tq)
    return slopes_from_heights(h)


@pytest.mark.parametrize("X,Y,p,q,n", [(8, 8, 0.75, 0.25, 2), (16, 8, 1.0, 0.0, 2), (8, 16, 0.6, 0.3, 3),
                                       (24, 16, 0.5, 0.5, 1)])
def test_attempts_match_prediction(X, Y, p, q, n):
    for seed in (3, 0xABCDEF0123):
        bx, by = o.init_flat_rect(X, Y)
        o.rs_run(bx, by, seed, p, q, t0=0, n_mcs=n)
        ex, ey = predicted(X, Y, seed, p, q, n)
        assert np.array_equal(bx, ex) and np.array_equal(by, ey)


@pytest.mark.parametrize("X,Y,p,q", [(64, 32, 0.75, 0.25), (32, 64, 0.5, 0.0)])
def test_invariants_hold_every_step(X, Y, p, q):
    bx, by = o.init_flat_rect(X, Y)
    for t in range(6):
        o.rs_run(bx, by, 5, p, q, t0=t, n_mcs=1)
        assert np.all(bx.sum(axis=1) == X // 2) and np.all(by.sum(axis=0) == Y // 2)
        sx, sy = 2 * bx.astype(np.int64) - 1, 2 * by.astype(np.int64) - 1
        assert np.array_equal(sx + np.roll(sy, 1, axis=1), sy + np.roll(sx, 1, axis=0))
        h = o.heights_rect(bx, by)
        assert np.all((h - flat_heights(X, Y)) % 2 == 0)


def test_p0_q0_is_identity_and_bad_sizes_are_refused():
    bx, by = o.init_flat_rect(16, 8)
    o.rs_run(bx, by, 1, 0.0, 0.0, n_mcs=3)
    ex, ey = o.init_flat_rect(16, 8)
    assert np.array_equal(bx, ex) and np.array_equal(by, ey)
    for X, Y in ((12, 8), (8, 6)):
        bx, by = o.init_flat_rect(X, Y)
        with pytest.raises(ValueError):
            o.rs_run(bx, by, 1, 0.5, 0.0)


def _one_attempt_law(h, p, q):
    """Plain random-sequential step: a site uniform among the 16, flipped with p (minimum) or
    q (maximum)."""
    out = {}
    for y in range(4):
        for x in range(4):
            nb = [h[y, (x + 1) % 4], h[y, (x - 1) % 4], h[(y + 1) % 4, x], h[(y - 1) % 4, x]]
            r = p if all(v == h[y, x] + 1 for v in nb) else q if all(v == h[y, x] - 1 for v in nb) else 0.0
            if r > 0:
                g = h.copy()
                g[y, x] += 2 if r == p and all(v == h[y, x] + 1 for v in nb) else -2
                out[g.tobytes()] = out.get(g.tobytes(), 0.0) + r / 16
            if r < 1:
                out[h.tobytes()] = out.get(h.tobytes(), 0.0) + (1 - r) / 16
    return out


def test_4x4_torus_is_plain_random_sequential():
    """One MCS on the 4 x 4 torus = 16 plain random-sequential attempts: exact law P1^16 from
    flat (in height variables, states taken as slope configurations) against the oracle's
    frequencies over many seeds."""
    scipy_stats = pytest.importorskip("scipy.stats")
    p, q, n_seeds = 0.8, 0.3, 20000
    Tp, Tq = math.floor(p * 2.0 ** 32), math.floor(q * 2.0 ** 32)
    pe, qe = Tp / 2.0 ** 32, Tq / 2.0 ** 32          # the exact acceptance probabilities
    dist = {flat_heights(4, 4).tobytes(): 1.0}
    for _ in range(16):
        nd = {}
        for key, pr in dist.items():
            for k2, p2 in _one_attempt_law(np.frombuffer(key, dtype=np.int64).reshape(4, 4), pe, qe).items():
                nd[k2] = nd.get(k2, 0.0) + pr * p2
        # heights modulo a global shift of 2 (slopes do not see it): fold to keep the map small
        folded = {}
        for key, pr in nd.items():
            h = np.frombuffer(key, dtype=np.int64).reshape(4, 4)
            h = h - 2 * (h[0, 0] // 2)
            folded[h.tobytes()] = folded.get(h.tobytes(), 0.0) + pr
        dist = folded
    exact = {}
    for key, pr in dist.items():
        bx, by = slopes_from_heights(np.frombuffer(key, dtype=np.int64).reshape(4, 4))
        k = bx.tobytes() + by.tobytes()
        exact[k] = exact.get(k, 0.0) + pr
    assert abs(sum(exact.values()) - 1.0) < 1e-9
    counts = Counter()
    for seed in range(n_seeds):
        bx, by = o.init_flat_rect(4, 4)
        o.rs_run(bx, by, seed, p, q, n_mcs=1)
        counts[bx.tobytes() + by.tobytes()] += 1
    assert set(counts) <= set(exact)
    obs, exp, ro, re = [], [], 0, 0.0
    for k in sorted(exact, key=lambda k: -exact[k]):
        e = exact[k] * n_seeds
        if e >= 5:
            obs.append(counts.get(k, 0))
            exp.append(e)
        else:
            ro += counts.get(k, 0)
            re += e
    if re > 0:
        obs.append(ro)
        exp.append(re)
    chi2 = sum((a - b) ** 2 / b for a, b in zip(obs, exp))
    assert len(obs) > 10
    assert scipy_stats.chi2.sf(chi2, len(obs) - 1) > 1e-4, (chi2, len(obs))
