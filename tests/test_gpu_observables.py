"""Physics observables through the GPU path (paper Sec. I.A, Sec. I, Sec. IV).

* Two-time height correlation C(t, s) (sca_correlate): exact sums against the oracle on square
  and X x Y lattices for several (s, t) pairs; C(t, t) equals the roughness numerator; at the
  benchmark's size the p = 1 flat surface gives C = 1/4 between any two times; a reference
  state that does not close is reported with SCA_ESTATE.
* Edwards-Wilkinson growth for p = q (Sec. I.A): at L = 4096 the roughness grows
  logarithmically (about equal increments per factor of t) where q = 0 (KPZ) grows as a power.
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


@pytest.mark.parametrize("X,Y,p,q,s_times,t_times", [
    (256, 256, 0.75, 0.25, [1, 6], [9, 30]),
    (512, 512, 0.5, 0.0, [3], [4, 20]),
    (192, 66, 0.7, 0.3, [2], [5, 11]),          # per-site uniforms, 3 words per row
    (64, 130, 0.625, 0.375, [1, 4], [4, 12]),
    (8192, 34, 0.5, 0.5, [2], [7]),
])
def test_correlation_against_oracle(sca, X, Y, p, q, s_times, t_times):
    seed = 11
    bx, by = o.init_flat_rect(X, Y)
    states, t = {}, 0
    for tt in sorted(set(s_times + t_times)):
        o.run_rect(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
        t = tt
        states[tt] = (bx.copy(), by.copy())
    with sca.Sim(X, seed=seed, p=p, q=q, Ly=Y) as sim:
        snaps = {}
        for tt in sorted(set(s_times + t_times)):
            sim.step(tt - sim.t)
            snaps[tt] = sim.snapshot()
            for s in s_times:
                if s <= tt:
                    g = sim.correlate(snaps[s])
                    r = o.corr(states[tt], states[s])
                    assert g.status == 0
                    assert (g.t, g.N, g.Sa, g.Sb, g.Sab, g.cnum) == (tt, r["N"], r["Sa"], r["Sb"], r["Sab"],
                                                                    r["cnum"]), (tt, s)
                    assert g.c == pytest.approx(r["cnum"] / r["N"] ** 2, rel=1e-12, abs=1e-15)


def test_equal_times_give_the_roughness(sca):
    with sca.Sim(4096, seed=2, p=0.75, q=0.25) as sim:
        for n in (1, 10, 50):
            sim.step(n)
            w = sim.observe()
            g = sim.correlate(sim.snapshot())
            assert (g.cnum, g.Sa, g.Sb, g.Sab) == (w.num, w.S1, w.S1, w.S2)


def test_large_lattice_flat_closed_form(sca):
    """L = 65536, p = 1, q = 0: the state is the flat one after every MCS, so C(t, s) = 1/4 for
    every pair of times (cnum = N^2/4)."""
    with sca.Sim(65536, seed=1, p=1.0, q=0.0) as sim:
        sim.step(1)
        ref = sim.snapshot()
        sim.step(16)
        g = sim.correlate(ref)
        del ref
    assert g.status == 0 and 4 * g.cnum == g.N ** 2 and g.t == 17


def test_reference_that_does_not_close(sca):
    import torch
    with sca.Sim(1024, seed=2, p=0.5, q=0.0) as sim:
        sim.step(3)
        ref = sim.snapshot()
        ref[7 * 16 + 2] ^= 1 << 3
        torch.cuda.synchronize()
        g = sim.correlate(ref)
        assert g.status == sca.ESTATE


def test_edwards_wilkinson_log_growth(sca):
    """p = q = 1/2 (Edwards-Wilkinson, Sec. I.A): at L = 4096, W^2 rises by about the same
    amount per factor of 4 in t (logarithmic growth), while q = 0 (KPZ) rises by ever larger
    amounts (a power law)."""
    times = [4 ** k for k in range(1, 7)]          # 4 .. 4096
    ew = np.zeros(len(times))
    kpz = np.zeros(len(times))
    for seed in (1, 2, 3, 4):
        with sca.Sim(4096, seed=seed, p=0.5, q=0.5) as sim:
            ew += [x.w2 for x in sim.run(times)]
        with sca.Sim(4096, seed=seed, p=0.5, q=0.0) as sim:
            kpz += [x.w2 for x in sim.run(times)]
    inc = np.diff(ew)
    assert np.all(inc > 0)
    assert inc[1:].max() / inc[1:].min() < 1.4, inc
    kinc = np.diff(kpz)
    assert kinc[-1] / kinc[1] > 3.0, kinc
