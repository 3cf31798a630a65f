"""X x Y lattices (X != Y) on the GPU vs the CPU oracle: bit-exact canonical words and exact
roughness sums.

The paper names the lateral sizes X and Y (Sec. II.B) and runs a wide system X = 2^17 (Sec.
III).  The library takes X = sca_params.L sites per row and Y = sca_params.Ly rows; the two-pass
kernel (1) and the height-bit wavefront kernel (4) run them, the automatic choice picks one of
the two.  Shapes cover wide and tall lattices, a row count below the wavefront's halo (bands
that stream some rows twice), odd word counts, every draw mode, and the {0, 1} rules from rough
surfaces (a flat surface is a fixed point of p = 1) at 16 MCS per launch.
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


def _oracle(X, Y, seed, p, q, times, start=None, t0=0, mode=None):
    if start is None:
        bx, by = o.init_flat_rect(X, Y)
    else:
        bx, by = o.unpack_rect(X, Y, start)
    res, t = [], t0
    for tt in times:
        o.run_rect(bx, by, seed, p, q, mode=mode, t0=t, n_mcs=tt - t)
        t = tt
        res.append(o.observe_rect(bx, by))
    return o.pack_rect(bx, by), res


def _gpu(sca, X, Y, seed, p, q, times, kernel, start=None, k=None, bands=None):
    with sca.Sim(X, seed=seed, p=p, q=q, Ly=Y) as sim:
        if start is not None:
            sim.set_state(start, t=0)
        sim.set_kernel(kernel)
        if k is not None:
            sim.set_temporal_block(k)
        if bands is not None:
            sim.set_wave_bands(bands)
        if kernel != sca.KERNEL_AUTO:
            assert sim.kernel_in_use() == kernel
        obs = sim.run(times)
        return obs, sim.get_state(), sim.kernel_in_use()


def _same(obs, ora):
    assert len(obs) == len(ora)
    for g, r in zip(obs, ora):
        assert g.status == 0
        assert (g.S1, g.S2, g.num, g.N) == (r["S1"], r["S2"], r["num"], r["N"]), (g, r)


CASES = [
    # X,     Y,    p,      q,     times
    (64, 128, 0.75, 0.25, [1, 2, 5]),
    (128, 64, 0.5, 0.0, [1, 3, 8]),
    (192, 66, 0.7, 0.3, [1, 4]),             # per-site uniforms, 3 words per row
    (256, 2, 0.625, 0.375, [1, 2, 7]),       # two rows
    (2048, 6, 0.875, 0.125, [2, 9]),
    (64, 2048, 0.5, 0.5, [1, 6]),            # tall and narrow
    (131072, 16, 0.5, 0.0, [1, 3]),          # the paper's wide system, X = 2^17, a few rows
    (320, 96, 0.9, 0.05, [3, 5]),            # per-site uniforms
    (131072, 16, 0.7, 0.3, [1, 2]),          # per-site uniforms on 2048-word rows, few rows
    (65536, 8, 0.6, 0.4, [1]),               # per-site uniforms, 512-thread row teams
]


@pytest.mark.parametrize("X,Y,p,q,times", CASES)
@pytest.mark.parametrize("kernel", [1, 4, 0])
def test_rect_parity_vs_oracle(sca, X, Y, p, q, times, kernel):
    words_o, ora = _oracle(X, Y, 9, p, q, times)
    obs, words, _ = _gpu(sca, X, Y, 9, p, q, times, kernel)
    _same(obs, ora)
    assert np.array_equal(words, words_o)


@pytest.mark.parametrize("X,Y,p,q,times,k,bands", [
    (1024, 96, 1.0, 0.0, [16, 40], 16, None),    # a band of 96 rows with 66 halo rows (wraps)
    (256, 512, 0.0, 1.0, [16, 33], 16, 3),
    (4096, 34, 1.0, 1.0, [8, 24], 8, None),
    (2048, 256, 1.0, 0.0, [2, 5], 2, 5),         # four words per lane, uneven bands
    (131072, 40, 1.0, 0.0, [16, 20], 16, None),
])
def test_rect_wave01_rough_against_oracle(sca, X, Y, p, q, times, k, bands):
    """The height-bit kernel at up to 16 MCS per launch from a rough X x Y surface (made by the
    oracle: 6 MCS of p = 5/8, q = 3/8) against the oracle."""
    bx, by = o.init_flat_rect(X, Y)
    o.run_rect(bx, by, 31, 0.625, 0.375, t0=0, n_mcs=6)
    start = o.pack_rect(bx, by)
    obs, words, kern = _gpu(sca, X, Y, 5, p, q, times, sca.KERNEL_WAVE, start=start, k=k, bands=bands)
    words_o, ora = _oracle(X, Y, 5, p, q, times, start=start)
    _same(obs, ora)
    assert np.array_equal(words, words_o)
    assert not np.array_equal(words, start)


def test_rect_wide_lattice_default_choice(sca):
    """X = 2^17, Y = 64, p = 1/2 with the automatic choice, against the oracle."""
    X, Y, times = 131072, 64, [1, 4]
    words_o, ora = _oracle(X, Y, 3, 0.5, 0.0, times)
    obs, words, kern = _gpu(sca, X, Y, 3, 0.5, 0.0, times, sca.KERNEL_AUTO)
    assert kern in (sca.KERNEL_TWO_PASS, sca.KERNEL_WAVE)
    _same(obs, ora)
    assert np.array_equal(words, words_o)


def test_rect_tall_two_tier_plan_equals_two_pass(sca):
    """A tall lattice (X = 10240, Y = 2^17: six column tiles, the last one ragged) from a rough
    surface at 16 MCS per launch, where the wavefront's launch plan has a second tier of
    shorter bands: the device state and exact sums equal those of the two-pass kernel."""
    import torch
    X, Y, times = 10240, 131072, [48, 96]
    with sca.Sim(X, seed=31, p=0.625, q=0.375, Ly=Y, kernel=sca.KERNEL_TWO_PASS) as sim:
        sim.step(3)
        words = sim.get_state()
    res = []
    for kernel in (sca.KERNEL_WAVE, sca.KERNEL_TWO_PASS):
        with sca.Sim(X, seed=5, p=1.0, q=0.0, Ly=Y, kernel=kernel) as sim:
            sim.set_state(words, t=0)
            if kernel == sca.KERNEL_WAVE:
                sim.set_temporal_block(16)
            assert sim.kernel_in_use() == kernel
            obs = sim.run(times)
            res.append(([(g.S1, g.S2, g.num) for g in obs], sim.state_tensor().clone()))
    assert res[0][0] == res[1][0]
    assert torch.equal(res[0][1], res[1][1])


def test_rect_refusals_and_state_check(sca):
    """Kernels 2 and 3 refuse X != Y; a loaded state with one flipped slope is not a surface:
    the wavefront kernel refuses it, the two-pass kernel runs it, and the observation reports
    SCA_ESTATE."""
    X, Y = 2048, 64
    with sca.Sim(X, seed=1, p=0.5, q=0.0, Ly=Y) as sim:
        for k in (sca.KERNEL_FUSED, sca.KERNEL_TBLOCK):
            with pytest.raises(sca.ScaError) as e:
                sim.set_kernel(k)
            assert e.value.code == sca.EINVAL
        w = sim.get_state()
        assert w.size == sca.words_count(X, Y)
        w[3 * (X // 64) + 1] ^= 1 << 5
        sim.set_state(w, t=0)
        assert sim.observe().status == sca.ESTATE
        sim.set_kernel(sca.KERNEL_WAVE)
        with pytest.raises(sca.ScaError) as e:
            sim.step(1)
        assert e.value.code == sca.ESTATE
        sim.set_kernel(sca.KERNEL_TWO_PASS)
        sim.step(1)
    with pytest.raises(sca.ScaError):
        with sca.Server(budget_bytes=1 << 30, max_active=1, max_L=512) as srv:
            prm = sca.sca_params(L=256, rng=0, seed=1, p=0.5, q=0.0, Ly=128)
            import ctypes as C
            tk = C.c_uint64()
            sca.check(sca.load().sca_server_submit(srv._h, C.byref(prm), 10, None, 0, C.byref(tk)),
                      "sca_server_submit")
