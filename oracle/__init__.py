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
        L.oracle_init_flat_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p]
        L.oracle_init_flat_rect.restype = None
        L.oracle_init_flat_band_rect.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64, u8p, u8p]
        L.oracle_init_flat_band_rect.restype = None
        L.oracle_run_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, C.c_uint64, C.c_double,
                                      C.c_double, C.c_int, C.c_uint64, C.c_uint64]
        L.oracle_run_rect.restype = C.c_int
        L.oracle_run_band_rect.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64, u8p, u8p,
                                           C.c_uint64, C.c_double, C.c_double, C.c_int, C.c_uint64,
                                           C.c_uint64]
        L.oracle_run_band_rect.restype = C.c_int
        L.oracle_heights_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, i64p]
        L.oracle_heights_rect.restype = C.c_int
        L.oracle_observe_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, C.POINTER(C.c_int64),
                                          u64p, u64p]
        L.oracle_observe_rect.restype = C.c_int
        L.oracle_pack_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, u32p]
        L.oracle_pack_rect.restype = None
        L.oracle_unpack_rect.argtypes = [C.c_int64, C.c_int64, u32p, u8p, u8p]
        L.oracle_unpack_rect.restype = None
        L.oracle_run_rect_counted.argtypes = [C.c_int64, C.c_int64, u8p, u8p, C.c_uint64, C.c_double,
                                              C.c_double, C.c_int, C.c_uint64, C.c_uint64,
                                              C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.oracle_run_rect_counted.restype = C.c_int
        L.oracle_rs_run_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, C.c_uint64, C.c_double,
                                         C.c_double, C.c_uint64, C.c_uint64]
        L.oracle_rs_run_rect.restype = C.c_int
        L.oracle_corr_rect.argtypes = [C.c_int64, C.c_int64, u8p, u8p, u8p, u8p,
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int64), i64p, i64p]
        L.oracle_corr_rect.restype = C.c_int
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


def word_draw_bit(X, seed, t, s, draw, x, y) -> int:
    """Draw bit of site (x, y) for rows of X sites (X = L on a square lattice)."""
    return int(lib().oracle_word_draw_bit(X, seed, t, s, draw, x, y))


def site_uniform(X, seed, t, s, x, y) -> int:
    """Per-site 32-bit uniform of site (x, y) for rows of X sites."""
    return int(lib().oracle_site_uniform(X, seed, t, s, x, y))


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


# ----------------------------------------------------------------------------- X x Y lattices
# Arrays are (Y, X): Y rows of X sites.  The square functions above are the case X = Y = L.

def init_flat_rect(X, Y):
    bx = np.empty((Y, X), dtype=np.uint8)
    by = np.empty((Y, X), dtype=np.uint8)
    lib().oracle_init_flat_rect(X, Y, bx, by)
    return bx, by


def init_flat_band_rect(X, Y, y_first, nrows):
    bx = np.empty((nrows, X), dtype=np.uint8)
    by = np.empty((nrows, X), dtype=np.uint8)
    lib().oracle_init_flat_band_rect(X, Y, y_first, nrows, bx, by)
    return bx, by


def run_rect(bx, by, seed, p, q, mode=None, t0=0, n_mcs=1):
    Y, X = bx.shape
    if mode is None:
        mode = rng_mode(p, q)
    if lib().oracle_run_rect(X, Y, bx, by, seed, float(p), float(q), mode, t0, n_mcs) != 0:
        raise ValueError("oracle_run_rect: bad parameters")


def run_band_rect(X, Y, y_first, bx, by, seed, p, q, mode=None, t0=0, n_mcs=1):
    nrows = bx.shape[0]
    if mode is None:
        mode = rng_mode(p, q)
    if lib().oracle_run_band_rect(X, Y, y_first, nrows, bx, by, seed, float(p), float(q), mode, t0,
                                  n_mcs) != 0:
        raise ValueError("oracle_run_band_rect: bad parameters")


def heights_rect(bx, by):
    Y, X = bx.shape
    h = np.empty((Y, X), dtype=np.int64)
    if lib().oracle_heights_rect(X, Y, bx, by, h) != 0:
        raise ValueError("slopes do not close: heights are not single-valued")
    return h


def observe_rect(bx, by):
    """Exact roughness sums of an X x Y lattice: dict(S1, S2, num, N), N = X*Y."""
    Y, X = bx.shape
    S1 = C.c_int64()
    S2 = np.zeros(2, dtype=np.uint64)
    num = np.zeros(2, dtype=np.uint64)
    if lib().oracle_observe_rect(X, Y, bx, by, C.byref(S1), S2, num) != 0:
        raise ValueError("slopes do not close: heights are not single-valued")
    return {"S1": int(S1.value), "S2": int(S2[0]) | (int(S2[1]) << 64),
            "num": int(num[0]) | (int(num[1]) << 64), "N": X * Y}


def pack_rect(bx, by):
    Y, X = bx.shape
    w = np.empty(4 * Y * words_per_row(X), dtype=np.uint32)
    lib().oracle_pack_rect(X, Y, bx, by, w)
    return w


def unpack_rect(X, Y, words):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    assert words.size == 4 * Y * words_per_row(X)
    bx = np.empty((Y, X), dtype=np.uint8)
    by = np.empty((Y, X), dtype=np.uint8)
    lib().oracle_unpack_rect(X, Y, words, bx, by)
    return bx, by


def corr(a, b):
    """Two-time height correlation of states a = (ax, ay) and b = (bx, by) of one lattice:
    dict(Sa, Sb, Sab, cnum, N) with Python ints; C = cnum / N^2 (cnum may be negative)."""
    ax, ay = a
    bx, by = b
    Y, X = ax.shape
    Sa = C.c_int64()
    Sb = C.c_int64()
    Sab = np.zeros(2, dtype=np.int64)
    cn = np.zeros(2, dtype=np.int64)
    if lib().oracle_corr_rect(X, Y, ax, ay, bx, by, C.byref(Sa), C.byref(Sb), Sab, cn) != 0:
        raise ValueError("slopes do not close: heights are not single-valued")

    def i128(v):
        return (int(v[1]) << 64) + (int(v[0]) & 0xFFFFFFFFFFFFFFFF)
    return {"Sa": int(Sa.value), "Sb": int(Sb.value), "Sab": i128(Sab), "cnum": i128(cn),
            "N": X * Y}


def run_rect_counted(bx, by, seed, p, q, mode=None, t0=0, n_mcs=1):
    """As run_rect; returns (origin_dh, total_dh): the summed height changes (+2 per deposition,
    -2 per removal) of site (0, 0) and of all sites over these MCS."""
    Y, X = bx.shape
    if mode is None:
        mode = rng_mode(p, q)
    org = C.c_int64(0)
    tot = C.c_int64(0)
    if lib().oracle_run_rect_counted(X, Y, bx, by, seed, float(p), float(q), mode, t0, n_mcs,
                                     C.byref(org), C.byref(tot)) != 0:
        raise ValueError("oracle_run_rect_counted: bad parameters")
    return int(org.value), int(tot.value)


def rs_run(bx, by, seed, p, q, t0=0, n_mcs=1):
    """Random-sequential dynamics over the 4 x 4 words (see sca_oracle.c) on (Y, X) arrays."""
    Y, X = bx.shape
    if lib().oracle_rs_run_rect(X, Y, bx, by, seed, float(p), float(q), t0, n_mcs) != 0:
        raise ValueError("oracle_rs_run_rect: bad parameters")
