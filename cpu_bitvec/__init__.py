"""Bit-vectorized CPU implementation (w = 64, OpenMP): the like-for-like CPU baseline.

The paper compares its GPU kernel with a CPU implementation of the same bit-vectorized update
on 64-bit words over all cores (Sec. II.B, Sec. III).  This package is that baseline: the
benchmark times it beside the GPU path, and the tests check it bit for bit against the oracle.
It is not part of the GPU library, which neither imports nor loads it, and it shares no code
with the library or the oracle.  ctypes marshalling only; the arithmetic is in sca_bitvec.c.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

DYADIC, UNIFORM32 = 1, 2


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        L.bitvec_run.argtypes = [u32p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_double,
                                 C.c_int, C.c_uint64, C.c_uint64]
        L.bitvec_run.restype = C.c_int
        L.bitvec_threads.argtypes = [C.c_int]
        L.bitvec_threads.restype = C.c_int
        _lib = L
    return _lib


def threads(n: int = 0) -> int:
    return lib().bitvec_threads(int(n))


def flat_words(X, Y=None):
    """Canonical words of the flat surface h = (x + y) & 1: sublattice 0 all zero, sublattice 1
    with the X/2 valid bits of every row set (X a multiple of 64, so every bit is valid)."""
    Y = X if Y is None else Y
    w = np.zeros(4 * Y * (X // 64), dtype=np.uint32)
    w[w.size // 2:] = 0xFFFFFFFF
    return w


def run(words, X, seed, p, q, mode, t0=0, n_mcs=1, Y=None):
    """Advance the canonical words in place (X a multiple of 128; Y rows, default X)."""
    Y = X if Y is None else Y
    assert words.dtype == np.uint32 and words.flags["C_CONTIGUOUS"] and words.size == 4 * Y * (X // 64)
    if lib().bitvec_run(words, X, Y, int(seed), float(p), float(q), int(mode), int(t0), int(n_mcs)) != 0:
        raise ValueError("bitvec_run: bad parameters")
