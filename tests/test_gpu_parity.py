"""GPU path vs the CPU oracle: bit-exact lattice state and exact roughness sums.

Every case calls the CUDA library through its C ABI (binding in paper_1606_00310_gb300/sca.py)
and compares, element by element, the canonical packed words and the integer sums S1, S2 and
num = N*S2 - S1^2 with the oracle run on the same seeded inputs.  Integer work, so the bar is
exact equality.  Sizes span several row teams and ragged word counts (W = L/64 odd, even, or a
multiple of 4); the largest lattices are checked on sampled rows (band oracle) and through
closed forms that hold at any size.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle as o

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sca():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00310_gb300 import build
    build.build()
    import paper_1606_00310_gb300.sca as mod
    mod.load()
    return mod


def oracle_run_obs(L, seed, p, q, times, mode=None, start=None, t0=0):
    if start is None:
        bx, by = o.init_flat(L)
    else:
        bx, by = o.unpack(L, start)
    res = []
    t = t0
    for tt in times:
        o.run(bx, by, seed, p, q, mode=mode, t0=t, n_mcs=tt - t)
        t = tt
        res.append(o.observe(bx, by))
    return o.pack(bx, by), res


def assert_obs_equal(gpu_obs, ora_obs):
    assert len(gpu_obs) == len(ora_obs)
    for g, r in zip(gpu_obs, ora_obs):
        assert g.status == 0
        assert (g.S1, g.S2, g.num, g.N) == (r["S1"], r["S2"], r["num"], r["N"]), (g, r)
        assert g.w2 == pytest.approx(r["num"] / r["N"] ** 2, rel=1e-15)


GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))


@pytest.mark.parametrize("case", GOLDEN["cases"], ids=[c["name"] for c in GOLDEN["cases"]])
@pytest.mark.parametrize("kernel", [1, 0])
def test_golden_cases(sca, case, kernel):
    if case["L"] % 64:
        pytest.skip("GPU lattices are multiples of 64")
    with sca.Sim(case["L"], seed=case["seed"], p=case["p"], q=case["q"], rng=case["mode"]) as sim:
        if kernel:
            sim.set_kernel(kernel)
        obs = sim.run([ob["t"] for ob in case["obs"]])
        words = sim.get_state()
    for g, ob in zip(obs, case["obs"]):
        assert (g.t, g.S1, str(g.S2), str(g.num)) == (ob["t"], ob["S1"], ob["S2"], ob["num"])
    assert hashlib.sha256(words.tobytes()).hexdigest() == case["final_words_sha256"]


def test_small_lattice_config(sca):
    """L = 64, p = 1, q = 0, seed 1, 1000 MCS, W^2 at 1, 2, 4, ..., 512: oracle and closed form
    (slopes return to the flat pattern every MCS, num = N^2 / 4)."""
    times = [2 ** k for k in range(10)] + [1000]
    with sca.Sim(64, seed=1, p=1.0, q=0.0) as sim:
        flat = sim.get_state()
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(64, 1, 1.0, 0.0, times)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o) and np.array_equal(words, flat)
    assert all(4 * g.num == g.N ** 2 for g in obs)


CASES = [
    # L, p, q, mode, seed, times
    (64, 0.5, 0.0, 1, 3, [1, 2, 3, 7, 20]),
    (128, 0.75, 0.25, 1, 9, [1, 2, 5, 30]),
    (192, 0.875, 0.125, 1, 0, [1, 2, 3, 17]),          # W = 3 (odd word count)
    (256, 0.3125, 0.0625, 1, 5, [1, 4, 9]),            # 4 and 5 draws
    (320, 0.5, 0.5, 1, 77, [1, 2, 13]),                # W = 5, Edwards-Wilkinson point
    (384, 2.0 ** -20 * 999_999, 0.0, 1, 8, [1, 3]),    # 20 draws
    (512, 0.7, 0.3, 2, 4, [1, 2, 6]),                  # per-site uniform
    (576, 0.95, 0.0, 2, 6, [1, 5]),                    # W = 9
    (1024, 0.5, 0.0, 1, 1, [1, 2, 8]),
    (1024, 0.6180339887, 0.1, 2, 2, [1, 3]),
    (2048, 0.75, 0.25, 1, 12, [1, 2]),
    (4096, 0.875, 0.125, 1, 3, [1]),
    (2880, 0.7, 0.3, 2, 21, [1, 2]),                   # W = 45: uniform teams across warps
    (5120, 0.55, 0.45, 2, 22, [1]),                    # W = 80: 20-thread teams, 240-thread blocks
    (128, 1.0, 1.0, 1, 5, [1, 2, 3]),                  # deterministic both ways
    (128, 0.0, 0.0, 1, 5, [1, 4]),                     # identity
]


@pytest.mark.parametrize("L,p,q,mode,seed,times", CASES)
@pytest.mark.parametrize("kernel", [1, 0])
def test_parity_vs_oracle(sca, L, p, q, mode, seed, times, kernel):
    with sca.Sim(L, seed=seed, p=p, q=q, rng=mode) as sim:
        if kernel:
            sim.set_kernel(kernel)
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, times, mode=mode)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)


def test_every_mcs_state_matches(sca):
    """Compare the whole state after every single MCS, not only at observation times."""
    L, seed, p, q = 256, 42, 0.75, 0.25
    bx, by = o.init_flat(L)
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        for t in range(12):
            sim.step(1)
            o.run(bx, by, seed, p, q, t0=t, n_mcs=1)
            assert np.array_equal(sim.get_state(), o.pack(bx, by)), t


def test_resume_from_set_state(sca):
    """A state set from the host at MCS t0 continues exactly like the oracle from t0: the
    counter-based generator makes resume bit-exact (checkpoint / restart)."""
    L, seed, p, q = 320, 5, 0.625, 0.375
    bx, by = o.init_flat(L)
    o.run(bx, by, seed, p, q, t0=0, n_mcs=9)
    start = o.pack(bx, by)
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        sim.set_state(start, t=9)
        assert sim.t == 9
        obs = sim.run([10, 15])
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, [10, 15], start=start, t0=9)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)
    # n + n with a save/restore in between equals 2n
    with sca.Sim(L, seed=seed, p=p, q=q) as a, sca.Sim(L, seed=seed, p=p, q=q) as b:
        a.step(6)
        mid = a.get_state()
        a.step(6)
        b.set_state(mid, t=6)
        b.step(6)
        assert np.array_equal(a.get_state(), b.get_state())


def test_bad_state_is_reported(sca):
    L = 128
    bx, by = o.init_flat(L)
    w = o.pack(bx, by)
    w[5] ^= 1          # one slope flipped: row 5 of sublattice 0 no longer closes
    with sca.Sim(L, seed=1, p=0.5, q=0.0) as sim:
        sim.set_state(w, t=0)
        ob = sim.observe()
        assert ob.status == sca.ESTATE


def test_mid_size_first_mcs_against_oracle(sca):
    """L = 4096 (16.8 M sites), dyadic (3/4, 1/4), seed 1: the whole state and the exact sums
    after each of the first 3 MCS."""
    L, seed, p, q = 4096, 1, 0.75, 0.25
    times = [1, 2, 3]
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, times)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)


def test_mid_size_p1_closed_form_long_run(sca):
    """L = 4096, p = 1, q = 0, 10^4 MCS at log-spaced times: the closed form holds at any size
    (state equals the flat state after every MCS, num = N^2/4)."""
    times = sorted({max(1, int(round(10 ** (4 * i / 39)))) for i in range(40)})
    with sca.Sim(4096, seed=1, p=1.0, q=0.0) as sim:
        flat = sim.get_state()
        obs = sim.run(times)
        assert np.array_equal(sim.get_state(), flat)
    assert all(4 * g.num == g.N ** 2 and g.status == 0 for g in obs)


def _rows_from_words(words, L, rows):
    """Unpack selected rows of canonical words to (bx, by) bytes (restating the layout)."""
    W = L // 64
    w = words.reshape(2, 2, L, W)
    bx = np.zeros((len(rows), L), np.uint8)
    by = np.zeros((len(rows), L), np.uint8)
    k = np.arange(L // 2)
    for i, y in enumerate(rows):
        for s in (0, 1):
            x = 2 * k + ((s + y) & 1)
            bx[i, x] = (w[s, 0, y, k >> 5] >> (k & 31)) & 1
            by[i, x] = (w[s, 1, y, k >> 5] >> (k & 31)) & 1
    return bx, by


@pytest.mark.parametrize("p,q", [(0.5, 0.0), (0.7, 0.3)])
def test_large_lattice_sampled_rows(sca, p, q):
    """L = 65536 (4.3 G sites, 1 GiB of packed slopes): after 2 MCS from flat, sampled rows
    (at the start, a team boundary and the periodic wrap) equal the band oracle's rows, which
    evolves exactly the rows that can influence them."""
    L, seed, n = 65536, 7, 2
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        sim.step(n)
        words = sim.get_state()
    for y_first in (0, 31000, L - 6):
        nrows = 4 * n + 4
        gx, gy = o.init_flat_band(L, y_first, nrows)
        o.run_band(L, y_first, gx, gy, seed, p, q, t0=0, n_mcs=n)
        rows = [(y_first + i) % L for i in range(2 * n, nrows - 2 * n)]
        bx, by = _rows_from_words(words, L, rows)
        assert np.array_equal(bx, gx[2 * n:nrows - 2 * n])
        assert np.array_equal(by, gy[2 * n:nrows - 2 * n])


def test_large_lattice_p1_closed_form(sca):
    """L = 65536, p = 1, q = 0: the state returns to flat every MCS and num = N^2/4 at every
    observation time (checked on the device state without copying the 1 GiB back)."""
    import torch
    with sca.Sim(65536, seed=1, p=1.0, q=0.0) as sim:
        flat = sim.state_tensor().clone()
        obs = sim.run([1, 2, 4, 8])
        assert torch.equal(sim.state_tensor(), flat)
    assert all(4 * g.num == g.N ** 2 for g in obs)


FUSED_CASES = [
    (2048, 0.5, 0.0, 1), (2048, 0.7, 0.3, 2), (6144, 0.75, 0.25, 1),
    (8192, 0.875, 0.125, 1), (16384, 0.5, 0.5, 1), (8192, 0.95, 0.0, 2), (8192, 1.0, 0.0, 1),
]


@pytest.mark.parametrize("L,p,q,mode", FUSED_CASES)
def test_fused_equals_two_pass(sca, L, p, q, mode):
    """The fused one-launch-per-MCS kernel and the two-pass kernel give identical states and
    sums (the choice of kernel changes speed only)."""
    times = [1, 2, 5, 9]
    res = []
    for kernel in (sca.KERNEL_TWO_PASS, sca.KERNEL_FUSED):
        with sca.Sim(L, seed=31, p=p, q=q, rng=mode, kernel=kernel) as sim:
            assert sim.kernel_in_use() == kernel
            obs = sim.run(times)
            res.append(([(o.S1, o.S2, o.num) for o in obs], sim.get_state()))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_fused_against_oracle(sca):
    L, seed, p, q = 2048, 3, 0.625, 0.125
    times = [1, 2, 3, 6]
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=sca.KERNEL_FUSED) as sim:
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, times)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)


@pytest.mark.parametrize("L,shape", [(8192, (4, 12)), (8192, (4, 8)), (16384, (2, 6)),
                                     (4096, (1, 6)), (65536, (2, 6)), (65536, (4, 8))])
def test_fused_launch_shapes_agree(sca, L, shape):
    """Every launch shape of the fused kernel (words per thread, shared-memory ring depth)
    gives the same state and sums as the two-pass kernel."""
    times = [1, 2, 3]
    res = []
    for kernel, sh in ((sca.KERNEL_TWO_PASS, None), (sca.KERNEL_FUSED, shape)):
        with sca.Sim(L, seed=17, p=0.75, q=0.25, kernel=kernel) as sim:
            if sh:
                sim.set_fused_shape(*sh)
            obs = sim.run(times)
            res.append(([(o.S1, o.S2, o.num) for o in obs], sim.state_tensor().clone()))
    assert res[0][0] == res[1][0]
    import torch
    assert torch.equal(res[0][1], res[1][1])


@pytest.mark.parametrize("L,p,q,mode,k", [
    (128, 0.75, 0.25, 1, 4), (192, 0.875, 0.125, 1, 2), (320, 0.7, 0.3, 2, 4),
    (1024, 0.5, 0.0, 1, 8), (4096, 0.75, 0.25, 1, 4), (8192, 0.95, 0.05, 2, 2),
    (2048, 1.0, 0.0, 1, 16), (640, 0.5, 0.5, 1, 1),
])
def test_temporal_blocking_equals_two_pass(sca, L, p, q, mode, k):
    """Several MCS per launch in shared memory (with recomputed halos) give the same states and
    sums as the two-pass kernel, also when the run length is not a multiple of k."""
    times = sorted({1, 3, k + 1, 2 * k + 3})
    res = []
    for kernel in (sca.KERNEL_TWO_PASS, sca.KERNEL_TBLOCK):
        with sca.Sim(L, seed=23, p=p, q=q, rng=mode) as sim:
            if kernel == sca.KERNEL_TBLOCK:
                sim.set_temporal_block(k)
            sim.set_kernel(kernel)
            assert sim.kernel_in_use() == kernel
            obs = sim.run(times)
            res.append(([(o.S1, o.S2, o.num) for o in obs], sim.get_state()))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_temporal_blocking_against_oracle(sca):
    L, seed, p, q = 256, 4, 0.625, 0.375
    times = [2, 4, 9]
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=sca.KERNEL_TBLOCK) as sim:
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, times)
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)


@pytest.mark.parametrize("kernel", [0, 4])
def test_many_observation_times(sca, kernel):
    """More observation times than one result block holds (records are returned 64 at a time),
    an observation of the initial state and a repeated time, all exact against the oracle."""
    L, seed, p, q = 128, 13, 0.75, 0.25
    times = list(range(0, 150)) + [150, 150]
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        if kernel:
            sim.set_kernel(kernel)
        obs = sim.run(times)
        words = sim.get_state()
    words_o, ora = oracle_run_obs(L, seed, p, q, times)
    assert [g.t for g in obs] == times
    assert_obs_equal(obs, ora)
    assert np.array_equal(words, words_o)
