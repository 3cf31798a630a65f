"""Random-sequential dynamics on the local 4 x 4 encoding (sca_params.dynamics = 1, the paper's
non-vectorized comparison, Sec. II.A and Sec. III) on the GPU against the oracle: canonical
words and exact roughness sums after each run, on square and X x Y lattices, two rows of words
(Y = 8), every rule kind."""
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


@pytest.mark.parametrize("X,Y,p,q,times", [
    (64, 64, 0.75, 0.25, [1, 3, 7]), (128, 64, 1.0, 0.0, [2, 5]), (64, 8, 0.5, 0.5, [1, 4, 9]),
    (256, 256, 0.7, 0.3, [1, 6]), (64, 1024, 0.9, 0.05, [3]), (192, 40, 1.0, 1.0, [2, 7]),
    (4096, 4096, 0.5, 0.0, [1, 3]),
])
def test_random_sequential_against_oracle(sca, X, Y, p, q, times):
    bx, by = o.init_flat_rect(X, Y)
    with sca.Sim(X, seed=19, p=p, q=q, Ly=Y, dynamics=sca.DYN_RANDOM_SEQUENTIAL) as sim:
        assert sim.kernel_in_use() == sca.KERNEL_RANDOM_SEQUENTIAL
        obs = sim.run(times)
        words = sim.get_state()
    t = 0
    for g, tt in zip(obs, times):
        o.rs_run(bx, by, 19, p, q, t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe_rect(bx, by)
        assert g.status == 0 and (g.S1, g.S2, g.num, g.N) == (r["S1"], r["S2"], r["num"], r["N"]), tt
    assert np.array_equal(words, o.pack_rect(bx, by))
    assert not np.array_equal(words, o.pack_rect(*o.init_flat_rect(X, Y)))


def test_random_sequential_resume_and_refusals(sca):
    """A run split in two with a host round trip of the state equals one run; sizes the local
    words cannot tile, origin tracking, batches and servers refuse the dynamics."""
    import ctypes as C
    L = 512
    with sca.Sim(L, seed=2, p=0.6, q=0.2, dynamics=sca.DYN_RANDOM_SEQUENTIAL) as a:
        a.step(9)
        ref = a.get_state()
    with sca.Sim(L, seed=2, p=0.6, q=0.2, dynamics=sca.DYN_RANDOM_SEQUENTIAL) as b:
        b.step(4)
        w = b.get_state()
        b.set_state(w, t=4)
        b.step(5)
        assert np.array_equal(b.get_state(), ref)
        with pytest.raises(sca.ScaError) as e:
            b.track_origin(True)
        assert e.value.code == sca.EINVAL
    with pytest.raises(sca.ScaError) as e:
        sca.Sim(64, seed=1, p=0.5, q=0.0, Ly=12, dynamics=sca.DYN_RANDOM_SEQUENTIAL)
    assert e.value.code == sca.EINVAL
    prm = sca.sca_params(L=256, rng=0, seed=1, p=0.5, q=0.0, Ly=0, dynamics=1)
    with sca.Server(budget_bytes=1 << 30, max_active=1, max_L=512) as srv:
        tk = C.c_uint64()
        assert sca.load().sca_server_submit(srv._h, C.byref(prm), 10, None, 0, C.byref(tk)) == sca.EINVAL
    h = C.c_void_p()
    assert sca.load().sca_batch_init(C.byref(prm), 1, None, C.byref(h)) == sca.EINVAL
