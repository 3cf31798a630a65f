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
    """L = 131072, the library's largest lattice, fits the fixed scratch (closed form p = 1:
    num = N^2/4); a larger L is refused on the host before any device work."""
    import torch
    with sca.Sim(131072, seed=1, p=1.0, q=0.0) as sim:
        sim.step(2)
        ref = sim.observe()
        torch.cuda.synchronize()
        got = sca.observe_noalloc(_state_ptr(sim), 131072, t=2)
        assert _same(got, ref)
        assert 4 * got.num == got.N ** 2
    o = sca.sca_obs()
    rc = sca.load().sca_observe_noalloc(C.c_void_p(16), 262144, 0, None, C.byref(o))
    assert rc == sca.EINVAL
    assert b"131072" in sca.load().sca_last_error()


def test_noalloc_reports_a_state_that_does_not_close(sca):
    """Words whose slopes do not close around the torus (one slope bit flipped in a rough
    surface): the entry point returns SCA_ESTATE with the same record as sca_observe."""
    import torch
    L = 1024
    with sca.Sim(L, seed=4, p=0.75, q=0.25) as sim:
        sim.step(3)
        words = sim.get_state()
        words[5 * (L // 64) + 3] ^= 1 << 7         # sublattice 0, sx-, row 5, word 3
        sim.set_state(words, t=3)
        ref = sim.observe()
        torch.cuda.synchronize()
        assert ref.status == sca.ESTATE
        got = sca.observe_noalloc(_state_ptr(sim), L, t=3)
        assert _same(got, ref), (got, ref)


def test_noalloc_leaves_nothing_for_the_next_call(sca):
    """A call that fills many chunk records (L = 65536, about four chunks per SM) followed by
    calls that fill few (L = 64 and 128, one chunk each): every result equals sca_observe's,
    so nothing the large call left in the shared array reaches the small ones."""
    import torch
    sims = [sca.Sim(65536, seed=2, p=0.5, q=0.0), sca.Sim(64, seed=3, p=0.75, q=0.25),
            sca.Sim(128, seed=5, p=0.6, q=0.3)]
    try:
        for sim, n in zip(sims, (2, 40, 25)):
            sim.step(n)
        refs = [sim.observe() for sim in sims]
        torch.cuda.synchronize()
        for _ in range(2):
            for sim, ref in zip(sims, refs):
                got = sca.observe_noalloc(_state_ptr(sim), sim.L, t=sim.t)
                assert ref.status == 0 and _same(got, ref), (sim.L, got, ref)
    finally:
        for sim in sims:
            sim.close()
