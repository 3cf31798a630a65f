"""Batched ensemble (one persistent, graph-captured launch over many lattices of uneven size)
vs the CPU oracle, vs single-lattice runs, and across launch shapes.  Exact equality of the
canonical words and of S1, S2, num for every lattice."""
import numpy as np
import pytest

import oracle as o
from paper_1606_00310_gb300 import workloads

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


MIX = [
    dict(L=128, p=0.75, q=0.25, seed=1), dict(L=192, p=1.0, q=0.0, seed=2),
    dict(L=256, p=0.875, q=0.125, seed=3), dict(L=320, p=0.7, q=0.3, seed=4),
    dict(L=512, p=0.5, q=0.5, seed=5), dict(L=640, p=0.625, q=0.0, seed=6),
    dict(L=1024, p=0.875, q=0.125, seed=7), dict(L=2048, p=0.75, q=0.25, seed=8),
    dict(L=128, p=0.95, q=0.05, seed=9), dict(L=1024, p=1.0, q=0.0, seed=10),
    dict(L=256, p=0.75, q=0.25, seed=11), dict(L=1536, p=0.5, q=0.0, seed=12),
]
TIMES = [1, 2, 3, 5, 8]


def oracle_lattice(d, times):
    bx, by = o.init_flat(d["L"])
    res, t = [], 0
    for tt in times:
        o.run(bx, by, d["seed"], d["p"], d["q"], t0=t, n_mcs=tt - t)
        t = tt
        res.append(o.observe(bx, by))
    return o.pack(bx, by), res


def test_batch_matches_oracle(sca):
    with sca.Batch(MIX) as b:
        obs, ens = b.run(TIMES)
        words = [b.get_state(i) for i in range(len(MIX))]
        shape = b.shape()
    assert shape["units"] >= 1
    for i, d in enumerate(MIX):
        w_o, ora = oracle_lattice(d, TIMES)
        for g, r in zip(obs[i], ora):
            assert g.status == 0
            assert (g.S1, g.S2, g.num, g.N) == (r["S1"], r["S2"], r["num"], r["N"]), (d, g, r)
        assert np.array_equal(words[i], w_o), d
    for k in range(len(TIMES)):
        assert ens[k] == pytest.approx(sum(obs[i][k].w2 for i in range(len(MIX))) / len(MIX),
                                       rel=1e-14)


def test_batch_alone_vs_in_the_mix(sca):
    """Each lattice's result is the same alone (a single-lattice simulation), in this batch,
    and in a batch of different composition and order."""
    sub = [MIX[7], MIX[0], MIX[3]]
    with sca.Batch(MIX) as b1, sca.Batch(sub) as b2:
        o1, _ = b1.run(TIMES)
        o2, _ = b2.run(TIMES)
        w1 = [b1.get_state(i) for i in (7, 0, 3)]
        w2 = [b2.get_state(i) for i in range(3)]
    for k, i in enumerate((7, 0, 3)):
        d = MIX[i]
        with sca.Sim(d["L"], seed=d["seed"], p=d["p"], q=d["q"]) as sim:
            so = sim.run(TIMES)
            sw = sim.get_state()
        assert [(x.S1, x.S2, x.num) for x in o1[i]] == [(x.S1, x.S2, x.num) for x in so]
        assert [(x.S1, x.S2, x.num) for x in o2[k]] == [(x.S1, x.S2, x.num) for x in so]
        assert np.array_equal(w1[k], sw) and np.array_equal(w2[k], sw)


@pytest.mark.parametrize("shape", [(8, 256), (8, 384), (16, 256), (4, 512), (6, 512), (5, 384),
                                   (3, 256)])
def test_batch_launch_shapes_agree(sca, shape):
    ref = None
    lat = [d for d in MIX if d["L"] <= 1024 or shape[0] >= 6]
    with sca.Batch(lat) as b:
        try:
            b.set_shape(*shape)
        except sca.ScaError:
            pytest.skip("shape %s not available on this GPU" % (shape,))
        got, _ = b.run(TIMES)
    with sca.Batch(lat) as b:
        ref, _ = b.run(TIMES)
    assert [[(x.S1, x.S2, x.num) for x in row] for row in got] == \
        [[(x.S1, x.S2, x.num) for x in row] for row in ref]


def test_batch_tune_and_repeat(sca):
    """The autotuner changes speed only; a repeated run of the captured graph after a reset
    reproduces the first run."""
    with sca.Batch(MIX) as b:
        first, _ = b.run(TIMES)
        b.reset()
        c, t = b.tune(8)
        assert b.t == 0 and c in (4, 5, 6, 8, 16) and t in (256, 384, 512)
        second, _ = b.run(TIMES)
        b.reset()
        third, _ = b.run(TIMES)
    key = lambda rows: [[(x.S1, x.S2, x.num) for x in row] for row in rows]  # noqa: E731
    assert key(first) == key(second) == key(third)


def test_ensemble_config_sample(sca):
    """The 4096-lattice ensemble (L uniform in {128..2048}, half (1, 0), half (7/8, 1/8),
    seed = index), 4096 MCS with W^2 at 2^0..2^12: every p = 1 lattice follows the closed form
    (num = N^2/4, state back to flat), and a stratified sample of small lattices equals the
    oracle at every observation time."""
    ens = workloads.ensemble()
    times = workloads.log_times(4096)
    with sca.Batch(ens) as b:
        obs, w2 = b.run(times)
        sample = []
        for L in (128, 256, 512):
            for kind in (1.0, 0.875):
                idx = [i for i, d in enumerate(ens) if d["L"] == L and d["p"] == kind]
                sample += idx[:2 if L < 512 else 1]
        words = {i: b.get_state(i) for i in sample}
        flat128 = None
        for i, d in enumerate(ens):
            if d["p"] == 1.0:
                assert all(4 * x.num == x.N ** 2 for x in obs[i]), i
        p1 = [i for i, d in enumerate(ens) if d["p"] == 1.0 and d["L"] == 2048][:2]
        for i in p1:
            bx, by = o.init_flat(2048)
            assert np.array_equal(b.get_state(i), o.pack(bx, by))
    for i in sample:
        w_o, ora = oracle_lattice(ens[i], times)
        assert [(x.S1, x.S2, x.num) for x in obs[i]] == [(r["S1"], r["S2"], r["num"]) for r in ora], i
        assert np.array_equal(words[i], w_o), i
    assert len(w2) == len(times) and all(np.isfinite(w2))
    del flat128


# Streaming engine (lane groups holding whole rows, bands streamed through registers): every
# power-of-two size the batch takes, every {0, 1} rule, dyadic rules with 1..4 draws, q = 0
# and not, p = 1 with dyadic q, p = 0; two runs in a row so the second starts mid-way.
STREAM_MIX = [
    dict(L=128, p=1.0, q=0.0, seed=21), dict(L=128, p=0.0, q=1.0, seed=22),
    dict(L=256, p=1.0, q=1.0, seed=23), dict(L=512, p=0.5, q=0.0, seed=24),
    dict(L=1024, p=0.75, q=0.25, seed=25), dict(L=2048, p=0.875, q=0.125, seed=26),
    dict(L=128, p=0.9375, q=0.0625, seed=27), dict(L=256, p=1.0, q=0.25, seed=28),
    dict(L=512, p=0.0, q=0.5, seed=29), dict(L=2048, p=1.0, q=0.0, seed=30),
    dict(L=256, p=0.625, q=0.375, seed=31), dict(L=1024, p=0.5, q=0.5, seed=32),
    dict(L=128, p=0.75, q=0.25, seed=33), dict(L=128, p=0.75, q=0.25, seed=34),
]


def _run_engine(sca, lattices, engine, runs):
    with sca.Batch(lattices) as b:
        b.set_engine(engine)
        assert b.engine() == engine
        out = []
        for times in runs:
            obs, ens = b.run(times)
            out.append(([[(x.S1, x.S2, x.num, x.status) for x in obs[i]] for i in range(len(lattices))], ens))
        words = [b.get_state(i) for i in range(len(lattices))]
    return out, words


def test_streaming_engine_equals_cluster_engine(sca):
    runs = [[1, 2, 5, 9, 16], [17, 25, 40]]
    a, wa = _run_engine(sca, STREAM_MIX, 1, runs)
    b, wb = _run_engine(sca, STREAM_MIX, 2, runs)
    for (oa, ea), (ob, eb) in zip(a, b):
        assert oa == ob
        assert ea == eb
    for x, y in zip(wa, wb):
        assert np.array_equal(x, y)


def test_streaming_engine_matches_oracle(sca):
    sub = [STREAM_MIX[i] for i in (1, 3, 4, 7, 10)]
    times = [1, 3, 8, 11]
    out, words = _run_engine(sca, sub, 2, [times])
    for i, d in enumerate(sub):
        w_o, ora = oracle_lattice(d, times)
        assert [(r["S1"], r["S2"], r["num"], 0) for r in ora] == out[0][0][i], d
        assert np.array_equal(words[i], w_o), d


def test_engine_choice(sca):
    """Per-site uniform draws and row lengths that are not a power of two keep the cluster
    engine; asking for the streaming engine there is refused."""
    with sca.Batch([dict(L=256, p=0.7, q=0.3, seed=1), dict(L=128, p=1.0, q=0.0, seed=2)]) as b:
        assert b.engine() == 1
        with pytest.raises(sca.ScaError):
            b.set_engine(2)
    with sca.Batch([dict(L=192, p=1.0, q=0.0, seed=1)]) as b:
        assert b.engine() == 1
    with sca.Batch([dict(L=256, p=0.75, q=0.25, seed=1), dict(L=512, p=1.0, q=0.0, seed=2)]) as b:
        assert b.engine() == 2
        with pytest.raises(sca.ScaError):
            b.set_engine(3)


# {0, 1} rules from a flat surface are fixed points of every MCS, so the engines' {0, 1} paths
# are checked from rough surfaces loaded with sca_batch_set_state (made by dyadic runs: the
# oracle's for the small lattices, the two-pass kernel's for the large ones).
ROUGH_MIX = [
    dict(L=128, p=1.0, q=0.0, seed=41), dict(L=128, p=0.0, q=1.0, seed=42),
    dict(L=256, p=1.0, q=1.0, seed=43), dict(L=512, p=1.0, q=0.0, seed=44),
    dict(L=1024, p=1.0, q=0.0, seed=45), dict(L=2048, p=1.0, q=0.0, seed=46),
    dict(L=256, p=0.75, q=0.25, seed=47), dict(L=2048, p=0.875, q=0.125, seed=48),
]


def _rough_words(sca, L, i):
    if L <= 256:
        bx, by = o.init_flat(L)
        o.run(bx, by, 100 + i, 0.625, 0.375, t0=0, n_mcs=5)
        return o.pack(bx, by)
    with sca.Sim(L, seed=100 + i, p=0.625, q=0.375, kernel=sca.KERNEL_TWO_PASS) as sim:
        sim.step(5)
        return sim.get_state()


@pytest.mark.parametrize("engine", [1, 2])
def test_batch_from_rough_surfaces(sca, engine):
    """Both engines, every {0, 1} rule and two dyadic ones, from rough surfaces: identical to a
    single-lattice simulation (two-pass kernel) from the same surface, and to the oracle for
    the small lattices."""
    starts = [_rough_words(sca, d["L"], i) for i, d in enumerate(ROUGH_MIX)]
    times = [3, 16, 37]
    with sca.Batch(ROUGH_MIX) as b:
        b.set_engine(engine)
        for i, w in enumerate(starts):
            b.set_state(i, w)
        obs, _ = b.run(times)
        words = [b.get_state(i) for i in range(len(ROUGH_MIX))]
    for i, d in enumerate(ROUGH_MIX):
        with sca.Sim(d["L"], seed=d["seed"], p=d["p"], q=d["q"], kernel=sca.KERNEL_TWO_PASS) as sim:
            sim.set_state(starts[i], t=0)
            ref = sim.run(times)
            ref_words = sim.get_state()
        assert [(g.S1, g.S2, g.num) for g in obs[i]] == [(g.S1, g.S2, g.num) for g in ref], d
        assert np.array_equal(words[i], ref_words), d
        if d["L"] <= 256:
            bx, by = o.unpack(d["L"], starts[i])
            t = 0
            for tt, g in zip(times, obs[i]):
                o.run(bx, by, d["seed"], d["p"], d["q"], t0=t, n_mcs=tt - t)
                t = tt
                r = o.observe(bx, by)
                assert (g.S1, g.S2, g.num) == (r["S1"], r["S2"], r["num"]), d
            assert np.array_equal(words[i], o.pack(bx, by)), d


def test_batch_set_state_refuses_a_non_surface(sca):
    with sca.Batch([dict(L=128, p=1.0, q=0.0, seed=1), dict(L=256, p=0.75, q=0.25, seed=2)]) as b:
        bx, by = o.init_flat(128)
        w = o.pack(bx, by)
        w[5] ^= 1 << 7
        with pytest.raises(sca.ScaError) as ei:
            b.set_state(0, w)
        assert ei.value.code == sca.ESTATE
        flat = o.pack(*o.init_flat(128))
        assert np.array_equal(b.get_state(0), flat)
        import ctypes
        assert sca.load().sca_batch_set_state(b._h, 2, flat.ctypes.data_as(ctypes.c_void_p), flat.size) == sca.EINVAL
        short = flat[:10].copy()
        assert sca.load().sca_batch_set_state(b._h, 0, short.ctypes.data_as(ctypes.c_void_p), short.size) == sca.EINVAL
