"""The bit-vectorized CPU baseline (w = 64, OpenMP; the paper's CPU implementation, Sec. II.B)
against the oracle, bit for bit (CPU only).

The benchmark reports this implementation beside the GPU numbers as the like-for-like CPU
baseline of the paper's GPU/CPU comparison (Sec. III); these cases pin it to the oracle on the
canonical words: square and X x Y lattices, an odd count of 64-bit words per row, two rows,
one to three dyadic draws, p = q, per-site uniforms, the {0, 1} rules from a rough surface.
"""
import numpy as np
import pytest

import cpu_bitvec as bv
import oracle as o


@pytest.mark.parametrize("X,Y,p,q,n", [
    (128, 128, 0.75, 0.25, 5), (384, 130, 0.5, 0.0, 4), (256, 2, 0.625, 0.375, 7),
    (128, 64, 0.875, 0.125, 6), (256, 256, 0.5, 0.5, 3), (384, 66, 0.7, 0.3, 4),
    (128, 96, 0.95, 0.0, 3)])
def test_bitvec_equals_oracle(X, Y, p, q, n):
    mode = o.rng_mode(p, q)
    bx, by = o.init_flat_rect(X, Y)
    w = bv.flat_words(X, Y)
    assert np.array_equal(w, o.pack_rect(bx, by))
    for t in range(n):
        o.run_rect(bx, by, 21, p, q, mode=mode, t0=t, n_mcs=1)
        bv.run(w, X, 21, p, q, mode, t0=t, n_mcs=1, Y=Y)
        assert np.array_equal(w, o.pack_rect(bx, by)), t


@pytest.mark.parametrize("p,q", [(1.0, 0.0), (0.0, 1.0), (1.0, 1.0)])
def test_bitvec_deterministic_rules_from_rough(p, q):
    X, Y = 256, 128
    bx, by = o.init_flat_rect(X, Y)
    o.run_rect(bx, by, 3, 0.625, 0.375, t0=0, n_mcs=5)
    w = o.pack_rect(bx, by)
    o.run_rect(bx, by, 9, p, q, t0=0, n_mcs=7)
    bv.run(w, X, 9, p, q, o.DYADIC, t0=0, n_mcs=7, Y=Y)
    assert np.array_equal(w, o.pack_rect(bx, by))


def test_bitvec_threads_do_not_change_results():
    X = 512
    a, b = bv.flat_words(X), bv.flat_words(X)
    n0 = bv.threads()
    try:
        bv.threads(1)
        bv.run(a, X, 4, 0.5, 0.0, o.DYADIC, n_mcs=5)
        bv.threads(max(2, n0))
        bv.run(b, X, 4, 0.5, 0.0, o.DYADIC, n_mcs=5)
    finally:
        bv.threads(n0)
    assert np.array_equal(a, b)


def test_bitvec_refuses_rows_of_odd_32_bit_words():
    with pytest.raises(ValueError):
        bv.run(bv.flat_words(192), 192, 1, 0.5, 0.0, o.DYADIC)
