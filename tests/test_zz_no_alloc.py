"""sca_observe_noalloc: the roughness observation for callers that cannot let the library
allocate device memory (their host application owns every byte of GPU memory, or cudaMalloc is
off limits where they run).  It must give exactly what sca_observe gives for the same words,
call after call, although all calls share one fixed scratch array on the device.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It also passes when run alone in a fresh process.
"""
import ctypes as C

import pytest

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


def _state_ptr(sim):
    import paper_1606_00310_gb300.sca as mod
    p = C.c_void_p()
    mod.check(mod.load().sca_state_device(sim._h, C.byref(p)), "sca_state_device")
    return p.value


def _same(a, b):
    return (a.t, a.N, a.S1, a.S2, a.num, a.status) == (b.t, b.N, b.S1, b.S2, b.num, b.status) \
        and a.w2 == b.w2


def test_noalloc_matches_observe_on_consecutive_calls(sca):
    """Two lattices of different sizes, observed one after the other through the new entry
    point, each against the allocating sca_observe on the same device words."""
    import torch
    cases = [(4096, 0.75, 0.25, 7, 5), (1024, 0.6, 0.3, 2, 9), (4096, 0.5, 0.0, 3, 2)]
    for L, p, q, seed, n in cases:
        with sca.Sim(L, seed=seed, p=p, q=q) as sim:
            sim.step(n)
            ref = sim.observe()
            torch.cuda.synchronize()
            got1 = sca.observe_noalloc(_state_ptr(sim), L, t=sim.t)
            got2 = sca.observe_noalloc(_state_ptr(sim), L, t=sim.t, stream=sim.stream)
            assert ref.status == 0
            assert _same(got1, ref), (got1, ref)
            assert _same(got2, ref), (got2, ref)


def test_noalloc_at_the_size_limit_and_beyond(sca):
    """L = 65536 is the largest size the fixed scratch holds (closed form p = 1: num = N^2/4);
    a larger L is refused on the host before any device work."""
    import torch
    with sca.Sim(65536, seed=1, p=1.0, q=0.0) as sim:
        sim.step(2)
        ref = sim.observe()
        torch.cuda.synchronize()
        got = sca.observe_noalloc(_state_ptr(sim), 65536, t=2)
        assert _same(got, ref)
        assert 4 * got.num == got.N ** 2
    o = sca.sca_obs()
    rc = sca.load().sca_observe_noalloc(C.c_void_p(16), 131072, 0, None, C.byref(o))
    assert rc == sca.EINVAL
    assert b"65536" in sca.load().sca_last_error()
