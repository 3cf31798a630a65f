"""CPU model of the observation kernel's word-pair arithmetic (k_obs_rows), checked against the
definition of the sums it forms.

For 64 consecutive sites of a row (the even-x word e and the odd-x word o, x order e0, o0, e1,
o1, ...) appended to a run whose offset is d, the kernel adds to the run's sum of offsets and
sum of squared offsets, with offsets the running sums of the slopes s = 2b - 1 (the height
relative to the run's start, Sec. I.A roughness through exact heights).  It does so through a
256-entry table over 8-site blocks with biased fields, byte permutes, a multiply by 0x01010101
for the in-word prefix sums and byte dot products (dp4a), with every bias taken out in closed
form.  This model restates those steps (byte permute and dp4a as their PTX definitions) and
compares them with the plain sums over the 64 offsets, on edge words and random words at
several starting offsets, so that a wrong bias constant, a wrong byte selector or a dropped
term fails without a GPU.
"""
import random

import pytest

M = 0xFFFFFFFF


def entry(i):
    """Table entry of block index i (bits 0-3: the four even-x sites, bits 4-7 the odd-x ones):
    byte 0 = S + 8, bits 8-23 = B, byte 3 = A + 36 for the block's running offsets d_k
    (S = d_7, A = sum d_k, B = sum d_k^2)."""
    d = a = b = 0
    for k in range(4):
        for bit in ((i >> k) & 1, (i >> (4 + k)) & 1):
            d += 2 * bit - 1
            a += d
            b += d * d
    assert 0 <= d + 8 <= 16 and 0 <= b <= 204 and 0 <= a + 36 <= 72
    return (d + 8) | (b << 8) | ((a + 36) << 24)


TABLE = [entry(i) for i in range(256)]


def byte_perm(x, y, s):
    """PTX prmt (default mode): result byte n is byte (selector nibble n & 7) of {y, x}."""
    src = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(src[(s >> (4 * n)) & 7] << (8 * n) for n in range(4))


def dp4a(a, b, c):
    """PTX dp4a.u32.u32: c plus the sum of the four unsigned byte products."""
    return (c + sum(((a >> (8 * i)) & 0xFF) * ((b >> (8 * i)) & 0xFF) for i in range(4))) & M


def pair_model(e, o, d, sd, sd2):
    x0 = (e & 0x0F0F0F0F) | ((o << 4) & 0xF0F0F0F0)
    x1 = ((e >> 4) & 0x0F0F0F0F) | (o & 0xF0F0F0F0)
    ent = [TABLE[byte_perm(x1 if k & 1 else x0, 0, 0x4440 + (k >> 1))] for k in range(8)]
    P = sum(ent) & M
    l0, h0 = byte_perm(ent[0], ent[1], 0x7340), byte_perm(ent[2], ent[3], 0x7340)
    l1, h1 = byte_perm(ent[4], ent[5], 0x7340), byte_perm(ent[6], ent[7], 0x7340)
    S0, A0 = byte_perm(l0, h0, 0x5410), byte_perm(l0, h0, 0x7632)
    S1, A1 = byte_perm(l1, h1, 0x5410), byte_perm(l1, h1, 0x7632)
    I0, I1 = (S0 * 0x01010101) & M, (S1 * 0x01010101) & M
    D0 = ((I0 << 8) + 0x28303840) & M
    D1 = ((I1 << 8) + (I0 >> 24) * 0x01010101 + 0x08101820) & M
    for D in (D0, D1):       # every biased offset stays inside its byte
        assert all(8 <= (D >> (8 * i)) & 0xFF <= 120 for i in range(4))
    q = dp4a(D1, D1, dp4a(D0, D0, 0))
    r = dp4a(D1, A1, dp4a(D0, A0, 0))
    u = dp4a((D0 + D1) & M, 0x01010101, 0)
    a = dp4a((A0 + A1) & M, 0x01010101, 0)
    SB = (P >> 8) & 0xFFFF
    X = 8 * u + a - 4384
    Z = 8 * q + 2 * r - 1096 * u - 128 * a + 299008 + SB
    return d + (I0 >> 24) + (I1 >> 24) - 64, sd + 64 * d + X, sd2 + d * (64 * d + 2 * X) + Z


def pair_definition(e, o, d, sd, sd2):
    for k in range(32):
        for bit in ((e >> k) & 1, (o >> k) & 1):
            d += 2 * bit - 1
            sd += d
            sd2 += d * d
    return d, sd, sd2


def test_table_fields_fit():
    # eight entries add without carrying out of the fields read from their sum (byte 0: S + 8,
    # bits 8-23: B); byte 3 (A + 36) is read per entry, never from the sum
    assert max(t & 0xFF for t in TABLE) * 8 <= 0xFF
    assert max((t >> 8) & 0xFFFF for t in TABLE) * 8 <= 0xFFFF


@pytest.mark.parametrize("d0", [0, 3, -37, 4000, -4096])
def test_pair_model_equals_definition(d0):
    rng = random.Random(d0 + 12345)
    words = [(0, 0), (M, M), (M, 0), (0, M), (0x55555555, 0xAAAAAAAA), (0x0F0F0F0F, 0xF0F0F0F0),
             (0x80000000, 0x00000001)]
    words += [(rng.getrandbits(32), rng.getrandbits(32)) for _ in range(3000)]
    for e, o in words:
        assert pair_model(e, o, d0, 11, -7) == pair_definition(e, o, d0, 11, -7), (hex(e), hex(o))
