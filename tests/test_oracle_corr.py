"""Pins for the oracle's two-time height correlation (CPU only).

The paper motivates the implementation by two-time functions and aging studies (Sec. I; Sec. IV
cites the aging study its code enabled) without printing a definition; the one used here is
the covariance over the sites of the height fields at two times,
    C(t, s) = (1/N) sum_x [h(x, t) - <h(t)>] [h(x, s) - <h(s)>] = cnum / N^2,
    cnum = N sum h_t h_s - (sum h_t)(sum h_s),
exact in integers.  Pinned by: an independent numpy restatement with Python integers;
C(t, t) = W^2(t) (the same numerator as the roughness); symmetry; the Cauchy-Schwarz bound
cnum^2 <= num_t num_s; and a closed form with a negative correlation (the flat surface against
the surface after one even half-step of deposition, C = -1/4).
"""
import numpy as np
import pytest

import oracle as o


def heights_numpy(bx, by):
    sx = 2 * bx.astype(np.int64) - 1
    sy = 2 * by.astype(np.int64) - 1
    col0 = np.concatenate([[0], np.cumsum(sy[1:, 0])])
    rows = np.concatenate([np.zeros((bx.shape[0], 1), np.int64), np.cumsum(sx[:, 1:], axis=1)],
                          axis=1)
    return col0[:, None] + rows


def slopes_from_heights(h):
    dx = h - np.roll(h, 1, axis=1)
    dy = h - np.roll(h, 1, axis=0)
    assert np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1)
    return ((dx + 1) // 2).astype(np.uint8), ((dy + 1) // 2).astype(np.uint8)


def cov_numpy(a, b):
    ha = heights_numpy(*a).astype(object).ravel()
    hb = heights_numpy(*b).astype(object).ravel()
    n = ha.size
    Sa, Sb, Sab = int(ha.sum()), int(hb.sum()), int((ha * hb).sum())
    return {"Sa": Sa, "Sb": Sb, "Sab": Sab, "cnum": n * Sab - Sa * Sb, "N": n}


def trajectory(X, Y, seed, p, q, times):
    bx, by = o.init_flat_rect(X, Y)
    out, t = [], 0
    for tt in times:
        o.run_rect(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
        t = tt
        out.append((bx.copy(), by.copy()))
    return out


@pytest.mark.parametrize("X,Y,p,q", [(64, 64, 0.75, 0.25), (96, 34, 0.5, 0.0), (34, 130, 0.7, 0.3)])
def test_corr_matches_numpy_restatement(X, Y, p, q):
    states = trajectory(X, Y, 7, p, q, [2, 5, 11])
    for a in states:
        for b in states:
            assert o.corr(a, b) == cov_numpy(a, b)


@pytest.mark.parametrize("X,Y", [(64, 64), (130, 24)])
def test_equal_times_give_the_roughness(X, Y):
    for a in trajectory(X, Y, 3, 0.625, 0.375, [1, 4, 9]):
        r, w = o.corr(a, a), o.observe_rect(*a)
        assert r["cnum"] == w["num"] and r["Sa"] == r["Sb"] == w["S1"] and r["Sab"] == w["S2"]


def test_symmetry_and_cauchy_schwarz():
    states = trajectory(128, 64, 5, 0.5, 0.0, [3, 8, 20])
    for a in states:
        for b in states:
            ab, ba = o.corr(a, b), o.corr(b, a)
            assert ab["cnum"] == ba["cnum"] and ab["Sab"] == ba["Sab"]
            assert (ab["Sa"], ab["Sb"]) == (ba["Sb"], ba["Sa"])
            assert ab["cnum"] ** 2 <= o.observe_rect(*a)["num"] * o.observe_rect(*b)["num"]
    # the surface keeps a memory of its past: positive correlation between two rough times
    assert o.corr(states[1], states[2])["cnum"] > 0


@pytest.mark.parametrize("X,Y", [(8, 8), (64, 6), (10, 130)])
def test_half_step_closed_form_is_negative(X, Y):
    """Flat h_a = (x + y) & 1 = 1 - E (E: even sites) against h_b = h_a + 2E = 1 + E (every even
    site deposited once): cov(1 - E, 1 + E) = -var(E) = -1/4, so cnum = -N^2 / 4; against
    itself +N^2/4."""
    E = (((np.arange(X)[None, :] + np.arange(Y)[:, None]) & 1) == 0).astype(np.int64)
    a = slopes_from_heights(1 - E)
    b = slopes_from_heights(1 + E)
    N = X * Y
    assert 4 * o.corr(a, b)["cnum"] == -N * N
    assert 4 * o.corr(a, a)["cnum"] == N * N
    assert 4 * o.corr(b, b)["cnum"] == N * N


def test_corr_rejects_states_that_do_not_close():
    a = o.init_flat_rect(64, 8)
    b = tuple(v.copy() for v in a)
    b[0][3, 5] ^= 1
    with pytest.raises(ValueError):
        o.corr(a, b)
