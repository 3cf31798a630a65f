"""CPU oracle for the octahedron-model SCA: TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this package.
The GPU library never imports it, and it imports nothing from the GPU library.  The arithmetic
lives in ``sca_oracle.c`` (see its header for the paper passages each function follows); this
module only marshals numpy arrays through ctypes.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_word_draw_bit.argtypes = [C.c_int64, C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                                           C.c_int64, C.c_int64]
        L.oracle_word_draw_bit.restype = C.c_uint32
        L.oracle_site_uniform.argtypes = [C.c_int64, C.c_uint64, C.c_uint64, C.c_int,
                                          C.c_int64, C.c_int64]
        L.oracle_site_uniform.restype = C.c_uint32
        L.oracle_dyadic_split.argtypes = [C.c_double, C.POINTER(C.c_uint64), C.POINTER(C.c_int)]
        L.oracle_dyadic_split.restype = C.c_int
        L.oracle_init_flat.argtypes = [C.c_int64, u8p, u8p]
        L.oracle_init_flat.restype = None
        L.oracle_init_flat_band.argtypes = [C.c_int64, C.c_int64, C.c_int64, u8p, u8p]
        L.oracle_init_flat_band.restype = None
        L.oracle_run.argtypes = [C.c_int64, u8p, u8p, C.c_uint64, C.c_double, C.c_double,
                                 C.c_int, C.c_uint64, C.c_uint64]
        L.oracle_run.restype = C.c_int
        L.oracle_run_band.argtypes = [C.c_int64, C.c_int64, C.c_int64, u8p, u8p, C.c_uint64,
                                      C.c_double, C.c_double, C.c_int, C.c_uint64, C.c_uint64]
        L.oracle_run_band.restype = C.c_int
        L.oracle_heights.argtypes = [C.c_int64, u8p, u8p, i64p]
        L.oracle_heights.restype = C.c_int
        L.oracle_observe.argtypes = [C.c_int64, u8p, u8p, C.POINTER(C.c_int64), u64p, u64p]
        L.oracle_observe.restype = C.c_int
        L.oracle_pack.argtypes = [C.c_int64, u8p, u8p, u32p]
        L.oracle_pack.restype = None
        L.oracle_unpack.argtypes = [C.c_int64, u32p, u8p, u8p]
        L.oracle_unpack.restype = None
        L.oracle_threads.argtypes = [C.c_int]
        L.oracle_threads.restype = C.c_int
        _lib = L
    return _lib


DYADIC = 1
UNIFORM32 = 2


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the oracle's OpenMP thread count."""
    return lib().oracle_threads(int(n))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(c, k, out)
    return out


def word_draw_bit(L, seed, t, s, draw, x, y) -> int:
    return int(lib().oracle_word_draw_bit(L, seed, t, s, draw, x, y))


def site_uniform(L, seed, t, s, x, y) -> int:
    return int(lib().oracle_site_uniform(L, seed, t, s, x, y))


def dyadic_split(p):
    """(P, n) with p = P / 2^n, P odd (n = 0 for p in {0, 1}); None if not dyadic."""
    P = C.c_uint64()
    n = C.c_int()
    ok = lib().oracle_dyadic_split(float(p), C.byref(P), C.byref(n))
    return (int(P.value), int(n.value)) if ok else None


def rng_mode(p, q):
    """Dyadic if both probabilities are multiples of 2^-32, else per-site uniform."""
    return DYADIC if (dyadic_split(p) is not None and dyadic_split(q) is not None) else UNIFORM32


def init_flat(L):
    bx = np.empty((L, L), dtype=np.uint8)
    by = np.empty((L, L), dtype=np.uint8)
    lib().oracle_init_flat(L, bx, by)
    return bx, by


def init_flat_band(L, y_first, nrows):
    bx = np.empty((nrows, L), dtype=np.uint8)
    by = np.empty((nrows, L), dtype=np.uint8)
    lib().oracle_init_flat_band(L, y_first, nrows, bx, by)
    return bx, by


def run(bx, by, seed, p, q, mode=None, t0=0, n_mcs=1):
    """Advance (bx, by) in place by n_mcs MCS starting at MCS index t0."""
    L = bx.shape[0]
    if mode is None:
        mode = rng_mode(p, q)
    rc = lib().oracle_run(L, bx, by, seed, float(p), float(q), mode, t0, n_mcs)
    if rc != 0:
        raise ValueError("oracle_run: bad parameters")


def run_band(L, y_first, bx, by, seed, p, q, mode=None, t0=0, n_mcs=1):
    nrows = bx.shape[0]
    if mode is None:
        mode = rng_mode(p, q)
    rc = lib().oracle_run_band(L, y_first, nrows, bx, by, seed, float(p), float(q), mode, t0,
                               n_mcs)
    if rc != 0:
        raise ValueError("oracle_run_band: bad parameters")


def heights(bx, by):
    L = bx.shape[0]
    h = np.empty((L, L), dtype=np.int64)
    if lib().oracle_heights(L, bx, by, h) != 0:
        raise ValueError("slopes do not close: heights are not single-valued")
    return h


def observe(bx, by):
    """Exact roughness sums: dict(S1, S2, num, N) with Python ints; W^2 = num / N^2."""
    L = bx.shape[0]
    S1 = C.c_int64()
    S2 = np.zeros(2, dtype=np.uint64)
    num = np.zeros(2, dtype=np.uint64)
    if lib().oracle_observe(L, bx, by, C.byref(S1), S2, num) != 0:
        raise ValueError("slopes do not close: heights are not single-valued")
    N = L * L
    return {"S1": int(S1.value), "S2": int(S2[0]) | (int(S2[1]) << 64),
            "num": int(num[0]) | (int(num[1]) << 64), "N": N}


def words_per_row(L):
    return (L // 2 + 31) // 32


def pack(bx, by):
    L = bx.shape[0]
    w = np.empty(4 * L * words_per_row(L), dtype=np.uint32)
    lib().oracle_pack(L, bx, by, w)
    return w


def unpack(L, words):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    assert words.size == 4 * L * words_per_row(L)
    bx = np.empty((L, L), dtype=np.uint8)
    by = np.empty((L, L), dtype=np.uint8)
    lib().oracle_unpack(L, words, bx, by)
    return bx, by
