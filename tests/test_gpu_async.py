"""Asynchronous host I/O and runs (sca_set_state_async, sca_get_state_async, sca_run_async,
sca_wait): pipelined over two simulations on two streams they give exactly the synchronous
results, the surface check still guards the height-bit kernel, and misuse is refused."""
import numpy as np
import pytest

import oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_00310_gb300 import build
    build.build()
    import paper_1606_00310_gb300.sca as mod
    mod.load()
    return mod, torch


def _pinned(torch, n):
    return torch.empty(n, dtype=torch.int32, pin_memory=True)


@pytest.mark.parametrize("L,p,q", [(4096, 1.0, 0.0), (2048, 0.75, 0.25), (1024, 0.7, 0.3)])
def test_pipelined_pair_equals_synchronous(env, L, p, q):
    sca, torch = env
    n = sca.words_count(L)
    times = [1, 3, 8, 17]
    # four different starting states: the oracle's flat surface advanced 0..3 MCS
    starts = []
    for k in range(4):
        bx, by = o.init_flat(L)
        if k:
            o.run(bx, by, 11, 0.625, 0.375, t0=0, n_mcs=k)
        starts.append(o.pack(bx, by).view(np.int32))
    ref = []
    with sca.Sim(L, seed=5, p=p, q=q) as sim:
        for w in starts:
            sim.set_state(w.view(np.uint32), t=0)
            ref.append(([(g.S1, g.S2, g.num) for g in sim.run(times)], sim.get_state()))
    ins = [_pinned(torch, n) for _ in range(4)]
    for i, w in enumerate(starts):
        ins[i].numpy()[:] = w
    outs = [_pinned(torch, n) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims = [sca.Sim(L, seed=5, p=p, q=q, stream=streams[i]) for i in range(2)]
    got = []
    try:
        pending = None
        for i in range(4):
            s = sims[i % 2]
            s.set_state_ptr_async(ins[i].data_ptr(), n, 0)
            s.run_async(times)
            s.get_state_ptr_async(outs[i % 2].data_ptr(), n)
            if pending is not None:
                j, sj = pending
                obs = sj.wait()
                got.append(([(g.S1, g.S2, g.num) for g in obs], outs[j % 2].numpy().view(np.uint32).copy()))
            pending = (i, s)
        j, sj = pending
        obs = sj.wait()
        got.append(([(g.S1, g.S2, g.num) for g in obs], outs[j % 2].numpy().view(np.uint32).copy()))
    finally:
        for s in sims:
            s.close()
    for (ro, rw), (go, gw) in zip(ref, got):
        assert ro == go
        assert np.array_equal(rw, gw)


def test_async_load_of_a_non_surface_is_caught(env):
    """The surface check of an asynchronous load is collected before the next kernel choice:
    forcing the height-bit kernel on a broken state fails with SCA_ESTATE."""
    sca, torch = env
    L = 256
    bx, by = o.init_flat(L)
    words = o.pack(bx, by)
    words[9] ^= 1 << 3
    n = sca.words_count(L)
    buf = _pinned(torch, n)
    buf.numpy()[:] = words.view(np.int32)
    with sca.Sim(L, seed=1, p=0.75, q=0.25, kernel=sca.KERNEL_WAVE) as sim:
        sim.set_state_ptr_async(buf.data_ptr(), n, 0)
        with pytest.raises(sca.ScaError) as ei:
            sim.run_async([2])
        assert ei.value.code == sca.ESTATE
        assert sim.wait() == []
        sim.set_kernel(sca.KERNEL_TWO_PASS)
        sim.set_state_ptr_async(buf.data_ptr(), n, 0)
        sim.run_async([2])
        assert len(sim.wait()) == 1


def test_async_misuse_is_refused(env):
    sca, torch = env
    import ctypes as C
    with sca.Sim(128, seed=1, p=1.0, q=0.0) as sim:
        lib = sca.load()
        times = (C.c_uint64 * 65)(*range(1, 66))
        assert lib.sca_run_async(sim._h, times, 65) == sca.EINVAL
        sim.run_async([1, 2])
        out = (sca.sca_obs * 3)()
        assert lib.sca_wait(sim._h, C.cast(out, C.c_void_p), 3) == sca.EINVAL
        assert len(sim.wait()) == 2
        back = (C.c_uint64 * 1)(1)
        assert lib.sca_run_async(sim._h, back, 1) == sca.EINVAL   # time before the current MCS
