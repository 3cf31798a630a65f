"""Pins for the oracle's Philox4x32-10 and its counter layout (CPU only).

Philox4x32-10 is defined by Salmon, Moraes, Dror and Shaw (SC'11).  The oracle's copy is checked
against an independent implementation (Triton's, run on the CPU by Triton's interpreter) and
against the statistical properties the paper needs from single random bits (Sec. II.B: the r = 1/2
case uses every bit of a word directly).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as o

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_outputs(items):
    pytest.importorskip("triton")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_ref.py")],
                          input=json.dumps(items), capture_output=True, text=True, timeout=300)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr.strip().splitlines()[-1])
    return json.loads(proc.stdout)


def test_philox_matches_triton_reference():
    rng = np.random.default_rng(12345)
    items = []
    keys = [(0, 0), (1, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x89ABCDEF, 0x01234567)]
    keys += [tuple(int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)) for _ in range(4)]
    for k in keys:
        ctrs = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
                [0xFFFFFFFF] * 4]
        ctrs += rng.integers(0, 2**32, (10, 4), dtype=np.uint64).tolist()
        items.append({"key": list(k), "ctrs": ctrs})
    ref = _triton_outputs(items)
    for item, out in zip(items, ref):
        for ctr, expect in zip(item["ctrs"], out):
            got = o.philox4x32_10(ctr, item["key"]).tolist()
            assert got == expect, (item["key"], ctr)


def test_philox_is_not_identity_and_key_sensitive():
    a = o.philox4x32_10([0, 0, 0, 0], [0, 0])
    b = o.philox4x32_10([0, 0, 0, 0], [1, 0])
    c = o.philox4x32_10([1, 0, 0, 0], [0, 0])
    assert len({tuple(a), tuple(b), tuple(c)}) == 3
    # Avalanche: one flipped counter bit changes about half of the 128 output bits.
    rng = np.random.default_rng(7)
    flips = []
    for _ in range(200):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        w = int(rng.integers(0, 4))
        bit = int(rng.integers(0, 32))
        ctr2 = ctr.copy()
        ctr2[w] ^= np.uint32(1 << bit)
        d = o.philox4x32_10(ctr, key) ^ o.philox4x32_10(ctr2, key)
        flips.append(sum(bin(int(v)).count("1") for v in d))
    assert 60 < np.mean(flips) < 68


def test_word_draw_bits_are_fair_and_uncorrelated():
    """Every bit position of the packed-word draws is set with frequency 1/2 and neighbouring
    sites / successive draws are uncorrelated (paper Sec. II.B: single-bit quality matters)."""
    L = 64
    n = 0
    ones = np.zeros(32)
    pair = 0
    draws12 = 0
    samples = []
    for t in range(4):
        for s in (0, 1):
            for y in range(L):
                for x in range(s ^ (y & 1), L, 2):
                    b1 = o.word_draw_bit(L, 99, t, s, 1, x, y)
                    b2 = o.word_draw_bit(L, 99, t, s, 2, x, y)
                    samples.append(b1)
                    ones[(x >> 1) & 31] += b1
                    draws12 += b1 ^ b2
                    n += 1
    samples = np.array(samples, dtype=np.float64)
    # n = 4 * 2 * 64 * 32 = 16384 site-draws; 5 sigma bounds
    assert abs(samples.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    assert abs(draws12 / n - 0.5) < 5 * 0.5 / np.sqrt(n)
    per_bit = ones / (n / 32)
    assert np.all(np.abs(per_bit - 0.5) < 5 * 0.5 / np.sqrt(n / 32))
    corr = np.corrcoef(samples[:-1], samples[1:])[0, 1]
    assert abs(corr) < 5 / np.sqrt(n)


def test_counter_layout_units():
    """The packed-word draw of site (x,y) is bit k & 31 of lane (unit & 3) of the Philox call
    with counter (unit >> 2, t, s | (draw-1) << 1, 0): re-derived here from the layout text."""
    L, seed = 256, 0x1234_5678_9ABC
    W = L // 64
    for (x, y, t, s, draw) in [(0, 0, 0, 0, 1), (3, 0, 5, 1, 2), (200, 17, 9, (200 + 17) & 1, 3),
                               (255, 255, 1, 0, 1), (130, 64, 2**33 + 3, 0, 4)]:
        s = (x + y) & 1
        k = x >> 1
        unit = y * W + (k >> 5)
        ctr = [unit >> 2, t & 0xFFFFFFFF, s | ((draw - 1) << 1) | ((t >> 32) << 6), 0]
        out = o.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        expect = (int(out[unit & 3]) >> (k & 31)) & 1
        assert o.word_draw_bit(L, seed, t, s, draw, x, y) == expect
        site_unit = y * (L // 2) + k
        ctr = [site_unit >> 2, t & 0xFFFFFFFF, s | ((t >> 32) << 6), 1]
        out = o.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert o.site_uniform(L, seed, t, s, x, y) == int(out[site_unit & 3])
