"""Register-wavefront temporal blocking (kernel 4) vs the two-pass kernel and the CPU oracle.

Several MCS per launch with each warp streaming a band of rows through registers; tiles
recompute halo words and rows.  Integer work: states and sums must be identical to the
two-pass kernel's and the oracle's.  Cases span one-word rows (W = 1), odd word counts, column
tiles that wrap around the lattice, two-row bands, uneven bands, run lengths that are not a
multiple of the MCS per launch (so shorter launches of 1..k-1 MCS), and the full-size
L = 65536 lattice.
"""
import numpy as np
import pytest

import oracle as o

pytestmark = pytest.mark.gpu


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


def _run(sca, kernel, L, p, q, times, k=None, bands=None, seed=23):
    with sca.Sim(L, seed=seed, p=p, q=q) as sim:
        sim.set_kernel(kernel)
        if k is not None:
            sim.set_temporal_block(k)
        if bands is not None:
            sim.set_wave_bands(bands)
        assert sim.kernel_in_use() == kernel
        obs = sim.run(times)
        return [(g.S1, g.S2, g.num) for g in obs], sim.get_state()


WAVE_CASES = [
    (64, 0.75, 0.25, 4, 0), (128, 1.0, 0.0, 8, 0), (192, 0.875, 0.125, 4, 0),
    (320, 0.5, 0.5, 8, 7), (2048, 0.75, 0.25, 8, 0), (1984, 0.625, 0.0, 2, 992),
    (4096, 1.0, 0.0, 8, 0), (4096, 0.5, 0.0, 1, 0), (8192, 0.9375, 0.0625, 8, 3),
    (6144, 1.0, 1.0, 4, 0), (3968, 0.75, 0.25, 2, 5),
    # four words per lane with the draw count fixed at compile time (1..3 draws, q = 0 or not),
    # p = 1 with dyadic q, and p = 0 (run-time draw loop)
    (2048, 0.875, 0.125, 2, 0), (1024, 0.625, 0.0, 2, 3), (512, 0.5, 0.5, 1, 0),
    (768, 0.75, 0.0, 2, 0), (1280, 1.0, 0.25, 2, 0), (1536, 0.0, 0.5, 2, 0),
    # the same at 4 MCS per launch
    (2048, 0.875, 0.125, 4, 0), (1024, 0.625, 0.0, 4, 3), (512, 0.5, 0.5, 4, 0), (768, 0.75, 0.0, 4, 0),
    (1280, 1.0, 0.25, 4, 0), (2560, 0.5, 0.0, 4, 0),
]


@pytest.mark.parametrize("L,p,q,k,bands", WAVE_CASES)
def test_wave_equals_two_pass(sca, L, p, q, k, bands):
    times = sorted({1, 3, k + 1, 2 * k + 3, 20})
    ref = _run(sca, sca.KERNEL_TWO_PASS, L, p, q, times)
    got = _run(sca, sca.KERNEL_WAVE, L, p, q, times, k=k, bands=bands)
    assert ref[0] == got[0]
    assert np.array_equal(ref[1], got[1])


@pytest.mark.parametrize("L,p,q,times", [(256, 0.625, 0.375, [2, 4, 9]),
                                         (320, 0.75, 0.0, [1, 8, 17]),
                                         (448, 1.0, 0.5, [5, 13])])
def test_wave_against_oracle(sca, L, p, q, times):
    seed = 4
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=sca.KERNEL_WAVE) as sim:
        obs = sim.run(times)
        words = sim.get_state()
    bx, by = o.init_flat(L)
    t = 0
    for tt, g in zip(times, obs):
        o.run(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe(bx, by)
        assert g.status == 0
        assert (g.S1, g.S2, g.num, g.N) == (r["S1"], r["S2"], r["num"], r["N"])
    assert np.array_equal(words, o.pack(bx, by))


@pytest.mark.parametrize("p,q", [(0.75, 0.25), (0.5, 0.0)])
def test_wave_full_size_equals_fused(sca, p, q):
    """L = 65536 (1 GiB of packed slopes), the automatic band count: identical device states
    and sums to the fused kernel after runs of 1, 3, 8 and 11 MCS."""
    import torch
    times = [1, 3, 8, 11]
    res = []
    for kernel in (sca.KERNEL_FUSED, sca.KERNEL_WAVE):
        with sca.Sim(65536, seed=9, p=p, q=q, kernel=kernel) as sim:
            obs = sim.run(times)
            res.append(([(g.S1, g.S2, g.num) for g in obs], sim.state_tensor().clone()))
    assert res[0][0] == res[1][0]
    assert torch.equal(res[0][1], res[1][1])


def test_wave_full_size_p1_closed_form(sca):
    """L = 65536, p = 1, q = 0: flat again after every MCS, num = N^2 / 4."""
    import torch
    with sca.Sim(65536, seed=1, p=1.0, q=0.0, kernel=sca.KERNEL_WAVE) as sim:
        flat = sim.state_tensor().clone()
        obs = sim.run([1, 2, 8, 24])
        assert torch.equal(sim.state_tensor(), flat)
    assert all(4 * g.num == g.N ** 2 for g in obs)


@pytest.mark.parametrize("L,p,q,k", [(256, 0.7, 0.3, 2), (320, 0.9, 0.05, 1), (4096, 0.55, 0.45, 2),
                                     (2048, 0.3, 0.0, 2), (1984, 1.0, 0.6, 1)])
def test_wave_uniform_equals_two_pass(sca, L, p, q, k):
    """Per-site uniform draws (non-dyadic p, q) in the wavefront kernel."""
    times = sorted({1, 3, k + 1, 2 * k + 3, 12})
    res = []
    for kernel in (sca.KERNEL_TWO_PASS, sca.KERNEL_WAVE):
        with sca.Sim(L, seed=19, p=p, q=q, rng=sca.RNG_UNIFORM32) as sim:
            sim.set_kernel(kernel)
            if kernel == sca.KERNEL_WAVE:
                sim.set_temporal_block(k)
            obs = sim.run(times)
            res.append(([(g.S1, g.S2, g.num) for g in obs], sim.get_state()))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_wave_rejects_what_it_cannot_run(sca):
    with sca.Sim(256, seed=1, p=0.75, q=0.25) as sim:
        sim.set_kernel(sca.KERNEL_WAVE)
        with pytest.raises(sca.ScaError):
            sim.set_temporal_block(12)
        with pytest.raises(sca.ScaError):
            sim.set_wave_bands(-1)
        with pytest.raises(sca.ScaError):
            sim.set_wave_bands(129)


def test_wave_resumes_from_a_set_state(sca):
    """A surface loaded with set_state (evolved by the oracle) passes the surface check and
    kernel 4 continues it exactly as the oracle does."""
    L, seed, p, q = 512, 6, 0.75, 0.25
    bx, by = o.init_flat(L)
    o.run(bx, by, seed, p, q, t0=0, n_mcs=5)
    start = o.pack(bx, by)
    o.run(bx, by, seed, p, q, t0=5, n_mcs=7)
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=sca.KERNEL_WAVE) as sim:
        sim.set_state(start, t=5)
        sim.step(7)
        assert np.array_equal(sim.get_state(), o.pack(bx, by))


def test_wave_refuses_a_state_that_is_not_a_surface(sca):
    """One flipped slope bit breaks two plaquettes: kernel 4 reports SCA_ESTATE instead of
    evolving it, while the slope-based kernels still accept the words as they are."""
    L = 256
    bx, by = o.init_flat(L)
    words = o.pack(bx, by)
    words[5] ^= 1 << 7
    with sca.Sim(L, seed=1, p=0.75, q=0.25, kernel=sca.KERNEL_WAVE) as sim:
        sim.set_state(words)
        with pytest.raises(sca.ScaError) as ei:
            sim.step(1)
        assert ei.value.code == sca.ESTATE
        sim.set_kernel(sca.KERNEL_TWO_PASS)
        sim.step(1)
        sim.reset()                       # a reset state is a surface again
        sim.set_kernel(sca.KERNEL_WAVE)
        sim.step(2)


def test_wave_largest_lattice_p1_closed_form(sca):
    """L = 131072 (the largest lattice, 4 GiB of packed slopes), automatic kernel choice: the
    height-bit kernel keeps the state flat under p = 1 and the exact W^2 is 1/4 at every time."""
    import torch
    L = 131072
    with sca.Sim(L, seed=3, p=1.0, q=0.0) as sim:
        assert sim.kernel_in_use() == sca.KERNEL_WAVE
        flat = sim.state_tensor().clone()
        obs = sim.run([1, 3, 20])
        assert torch.equal(sim.state_tensor(), flat)
        del flat
    assert all(4 * g.num == g.N ** 2 and g.status == 0 for g in obs)


# p, q in {0, 1} from a flat surface is a fixed point of every MCS (p = 1), so the cases below
# start from rough surfaces made by a dyadic rule: the oracle's at small L, the two-pass
# kernel's at large L.  16 MCS per launch is the default for L >= 16384 and is forced below it.
def _rough_gpu(sca, L, mcs, seed=31):
    with sca.Sim(L, seed=seed, p=0.625, q=0.375, kernel=sca.KERNEL_TWO_PASS) as sim:
        sim.step(mcs)
        return sim.get_state()


def _run_from(sca, L, p, q, words, times, kernel, k=None, bands=None):
    with sca.Sim(L, seed=5, p=p, q=q) as sim:
        sim.set_state(words, t=0)
        sim.set_kernel(kernel)
        if k is not None:
            sim.set_temporal_block(k)
        if bands is not None:
            sim.set_wave_bands(bands)
        assert sim.kernel_in_use() == kernel
        obs = sim.run(times)
        return [(g.S1, g.S2, g.num) for g in obs], sim.get_state()


@pytest.mark.parametrize("L,p,q,times,k", [(256, 1.0, 0.0, [48], 16), (320, 0.0, 1.0, [33, 80], 16),
                                           (448, 1.0, 1.0, [16, 64, 65], 16), (1024, 1.0, 0.0, [7, 71, 200], 16),
                                           (512, 1.0, 0.0, [9, 40], 8)])
def test_wave01_rough_against_oracle(sca, L, p, q, times, k):
    bx, by = o.init_flat(L)
    o.run(bx, by, 31, 0.625, 0.375, t0=0, n_mcs=6)
    got = _run_from(sca, L, p, q, o.pack(bx, by), times, sca.KERNEL_WAVE, k=k)
    t = 0
    for tt, g in zip(times, got[0]):
        o.run(bx, by, 5, p, q, t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe(bx, by)
        assert g == (r["S1"], r["S2"], r["num"])
    assert np.array_equal(got[1], o.pack(bx, by))


@pytest.mark.parametrize("L,p,q,times,k,bands", [
    (4096, 1.0, 0.0, [40, 200], 16, None), (8192, 0.0, 1.0, [64, 96], 16, None),
    (6144, 1.0, 1.0, [35, 99], 16, None), (16384, 1.0, 0.0, [32, 160], None, None),
    (4096, 1.0, 0.0, [80], 16, 31), (2048, 1.0, 0.0, [96], 16, 2), (1984, 1.0, 0.0, [64], 16, None),
    # bands of 32 rows, under 2K + 2: every launch writes its whole state
    (2048, 1.0, 0.0, [48], 16, 64),
    (8192, 1.0, 0.0, [24, 88], 8, 5),
    # four words per lane (1 and 2 MCS per launch): several tiles, uneven bands
    (8192, 1.0, 0.0, [10, 31], 2, None), (4096, 0.0, 1.0, [9], 1, 7), (6144, 1.0, 1.0, [5, 12], 2, 3)])
def test_wave01_rough_equals_two_pass(sca, L, p, q, times, k, bands):
    words = _rough_gpu(sca, L, 5)
    got = _run_from(sca, L, p, q, words, times, sca.KERNEL_WAVE, k=k, bands=bands)
    ref = _run_from(sca, L, p, q, words, times, sca.KERNEL_TWO_PASS)
    assert got[0] == ref[0]
    assert np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("L,times", [(65536, [50, 178]), (131072, [3, 40])])
def test_wave01_rough_full_size(sca, L, times):
    """The benchmark's lattice and the largest one, from a rough surface: the automatic choice
    (16 MCS per launch and the shorter launches up to each observation time) equals the two-pass
    kernel, device states and exact sums."""
    import torch
    words = _rough_gpu(sca, L, 3 if L == 65536 else 2)
    res = []
    for kernel in (sca.KERNEL_WAVE, sca.KERNEL_TWO_PASS):
        with sca.Sim(L, seed=5, p=1.0, q=0.0, kernel=kernel) as sim:
            sim.set_state(words, t=0)
            assert sim.kernel_in_use() == kernel
            obs = sim.run(times)
            res.append(([(g.S1, g.S2, g.num) for g in obs], sim.state_tensor().clone()))
    assert res[0][0] == res[1][0]
    assert torch.equal(res[0][1], res[1][1])


def _band_bits(w4, L, rows):
    """(bx, by) bytes of the given lattice rows from their canonical words w4[s][d][i][j]
    (restating the packed layout: site k of sublattice s in row y is x = 2k + ((s + y) & 1))."""
    bx = np.zeros((len(rows), L), np.uint8)
    by = np.zeros((len(rows), L), np.uint8)
    k = np.arange(L // 2)
    for i, y in enumerate(rows):
        for s in (0, 1):
            x = 2 * k + ((s + y) & 1)
            bx[i, x] = (w4[s, 0, i, k >> 5] >> (k & 31)) & 1
            by[i, x] = (w4[s, 1, i, k >> 5] >> (k & 31)) & 1
    return bx, by


def _device_rows(sim, L, rows):
    """Canonical words of the given rows, all four planes, copied from the device state."""
    import torch
    st = sim.state_tensor().view(2, 2, L, L // 64)
    idx = torch.tensor(rows, dtype=torch.long, device=st.device)
    return st.index_select(2, idx).cpu().numpy().view(np.uint32)


# windows: inside a band, across the periodic boundary in y, and across the boundary between
# the launch plan's tall bands and its second tier of shorter ones (rows 58984 and 117966)
@pytest.mark.parametrize("L,times,nrows,y_firsts", [(65536, [32, 40], 320, (1000, 65536 - 150, 58984 - 160)),
                                                     (131072, [32, 33], 256, (131072 - 90, 117966 - 128))])
def test_headline_kernel_rough_band_against_oracle(sca, L, times, nrows, y_firsts):
    """The benchmark's kernel (height bits, two 16-MCS launches, the first leaving the sx- planes
    to the second except on the rows the second starts its bands from, then the shorter launch
    up to the last time) at the benchmark's lattice and at the largest one, checked against the
    oracle
    itself on bands of rows, one of them wrapping around the periodic boundary in y.  Start: a
    rough surface, 3 MCS of p = 5/8, q = 3/8 (seed 31) from flat, made on the GPU by the two-pass
    kernel and by the band oracle from its own flat band (their common rows are compared too);
    then p = 1, q = 0.  After n MCS in all, a band of the oracle holds the full lattice's rows
    [2n, nrows - 2n) exactly (each half-step widens the dependence by one row either way)."""
    n_rough, seed_rough = 3, 31
    words = _rough_gpu(sca, L, n_rough, seed=seed_rough)
    with sca.Sim(L, seed=5, p=1.0, q=0.0) as sim:
        sim.set_state(words, t=0)
        del words
        assert sim.kernel_in_use() == sca.KERNEL_WAVE
        bands = {y0: [(y0 + i) % L for i in range(nrows)] for y0 in y_firsts}
        start = {y0: _device_rows(sim, L, rows) for y0, rows in bands.items()}
        obs = sim.run(times)
        assert all(g.status == 0 for g in obs)
        final = {y0: _device_rows(sim, L, rows) for y0, rows in bands.items()}
    for y0, rows in bands.items():
        gx, gy = o.init_flat_band(L, y0, nrows)
        o.run_band(L, y0, gx, gy, seed_rough, 0.625, 0.375, t0=0, n_mcs=n_rough)
        m = 2 * n_rough
        bx, by = _band_bits(start[y0], L, rows)
        assert np.array_equal(bx[m:nrows - m], gx[m:nrows - m])
        assert np.array_equal(by[m:nrows - m], gy[m:nrows - m])
        o.run_band(L, y0, gx, gy, 5, 1.0, 0.0, t0=0, n_mcs=times[-1])
        m = 2 * (n_rough + times[-1])
        assert nrows - 2 * m >= 100
        bx, by = _band_bits(final[y0], L, rows)
        assert np.array_equal(bx[m:nrows - m], gx[m:nrows - m])
        assert np.array_equal(by[m:nrows - m], gy[m:nrows - m])
        # the rough start and the result differ inside the compared rows: the kernel did work
        assert not np.array_equal(bx[m:nrows - m], _band_bits(start[y0], L, rows)[0][m:nrows - m])
