"""Degenerate inputs through the C ABI on the GPU: zero MCS, empty and repeated observation
lists, an observation at t = 0, the smallest lattices, and the refusals of empty work by the
batch and the server.

An observation at t = 0 is the flat surface h = (x + y) & 1 (Sec. I.A), W^2 = 1/4 exactly; the
sums at later times are the oracle's.
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


@pytest.mark.parametrize("kernel", [0, 1, 4])
def test_zero_mcs_empty_and_repeated_runs(sca, kernel):
    L, seed, p, q = 256, 7, 0.75, 0.25
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=kernel) as sim:
        flat = sim.get_state()
        sim.step(0)
        assert sim.t == 0 and np.array_equal(sim.get_state(), flat)
        assert sim.run([]) == []
        assert sim.t == 0 and np.array_equal(sim.get_state(), flat)
        obs = sim.run([0, 0, 3, 3, 3, 5])
        words = sim.get_state()
    assert [g.t for g in obs] == [0, 0, 3, 3, 3, 5]
    N = L * L
    for g in obs[:2]:                      # the flat surface: S1 = N/2, S2 = N/2, W^2 = 1/4
        assert (g.status, g.S1, g.S2, g.num) == (0, N // 2, N // 2, N * N // 4)
    bx, by = o.init_flat(L)
    assert np.array_equal(o.pack(bx, by), flat)
    o.run(bx, by, seed, p, q, t0=0, n_mcs=3)
    r3 = o.observe(bx, by)
    for g in obs[2:5]:
        assert (g.status, g.S1, g.S2, g.num) == (0, r3["S1"], r3["S2"], r3["num"])
    o.run(bx, by, seed, p, q, t0=3, n_mcs=2)
    r5 = o.observe(bx, by)
    assert (obs[5].S1, obs[5].S2, obs[5].num) == (r5["S1"], r5["S2"], r5["num"])
    assert np.array_equal(words, o.pack(bx, by))


@pytest.mark.parametrize("X,Y,kernel", [(64, 64, 0), (64, 64, 1), (64, 64, 4), (64, 2, 0), (64, 2, 4),
                                        (128, 4, 1)])
def test_smallest_lattices(sca, X, Y, kernel):
    """One 64-site word per sublattice row, down to two rows (the smallest the layout holds)."""
    seed, p, q, times = 3, 0.625, 0.375, [1, 2, 7]
    with sca.Sim(X, seed=seed, p=p, q=q, Ly=Y, kernel=kernel) as sim:
        obs = sim.run(times)
        words = sim.get_state()
    bx, by = o.init_flat_rect(X, Y)
    t = 0
    for g, tt in zip(obs, times):
        o.run_rect(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe_rect(bx, by)
        assert (g.status, g.S1, g.S2, g.num) == (0, r["S1"], r["S2"], r["num"]), tt
    assert np.array_equal(words, o.pack_rect(bx, by))


def test_sizes_outside_the_layout_are_refused(sca):
    for L, Ly in ((32, None), (96, None), (131072 + 64, None), (64, 3), (64, 131074)):
        with pytest.raises(sca.ScaError):
            sca.Sim(L, Ly=Ly)


def test_batch_and_server_refuse_empty_work(sca):
    with sca.Batch([dict(L=128, p=1.0, q=0.0, seed=1)]) as b:
        with pytest.raises(sca.ScaError):
            b.run([])
        with pytest.raises(sca.ScaError):
            b.run([0])                        # times must lie after the current MCS
        obs, _ = b.run([1, 2])
        assert [g.t for g in obs[0]] == [1, 2]
    with sca.Server(budget_bytes=1 << 30, max_active=2) as srv:
        with pytest.raises(sca.ScaError):
            srv.submit(256, 0.7, 0.3, 1, 0)   # zero MCS
