"""Physics observables through the GPU path (paper Sec. I.A, Sec. I, Sec. IV).

* Two-time height correlation C(t, s) (sca_correlate): exact sums against the oracle on square
  and X x Y lattices for several (s, t) pairs; C(t, t) equals the roughness numerator; at the
  benchmark's size the p = 1 flat surface gives C = 1/4 between any two times; a reference
  state that does not close is reported with SCA_ESTATE.
* Edwards-Wilkinson growth for p = q (Sec. I.A): at L = 4096 the roughness grows
  logarithmically (about equal increments per factor of t) where q = 0 (KPZ) grows as a power.
* A run's observations on the wavefront kernel with repeated times (no launch between two
  observations) and gaps of several launches: exact sums at every time and the final state
  against the oracle, and against the two-pass kernel from a rough surface at larger sizes.
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


# ------------------------------------------------------------------------- origin height
def _oracle_h00(X, Y, seed, p, q, times, start=None):
    if start is None:
        bx, by = o.init_flat_rect(X, Y)
    else:
        bx, by = o.unpack_rect(X, Y, start)
    out, h00, t = [], 0, 0
    for tt in times:
        h00 += o.run_rect_counted(bx, by, seed, p, q, t0=t, n_mcs=tt - t)[0]
        t = tt
        out.append((h00, o.observe_rect(bx, by)["S1"]))
    return out


@pytest.mark.parametrize("X,Y,p,q,kernel,k", [
    (256, 256, 0.75, 0.25, 1, None),             # two-pass, one tracker launch per MCS
    (2048, 2048, 0.5, 0.0, 2, None),             # fused
    (512, 512, 0.7, 0.3, 3, 32),                 # shared-memory blocking, 32 MCS capped to 16
    (1024, 1024, 0.625, 0.375, 4, 4),            # height bits, dyadic
    (192, 66, 0.6, 0.35, 4, 2),                  # height bits, per-site uniforms, X x Y
    (128, 6, 0.875, 0.125, 0, None),             # few rows: the patch wraps the lattice
    (4096, 4096, 0.5, 0.5, 0, None),
])
def test_origin_height_against_oracle(sca, X, Y, p, q, kernel, k):
    times = [1, 5, 18, 40]
    with sca.Sim(X, seed=13, p=p, q=q, Ly=Y) as sim:
        sim.set_kernel(kernel)
        if k is not None:
            sim.set_temporal_block(k)
        sim.track_origin(True)
        obs = sim.run(times)
    ref = _oracle_h00(X, Y, 13, p, q, times)
    assert [(g.h00, g.S1) for g in obs] == ref
    assert any(h != 0 for h, _ in ref)


def test_origin_height_rough_p1_wavefront(sca):
    """p = 1 from a rough surface at 16 MCS per launch (the benchmark's kernel): against the
    oracle, and the absolute mean height identity N h00 + S1 = N/2 + (all height changes)."""
    L = 2048
    bx, by = o.init_flat(L)
    o.run(bx, by, 31, 0.625, 0.375, t0=0, n_mcs=4)
    start = o.pack(bx, by)
    times = [16, 33, 64]
    with sca.Sim(L, seed=5, p=1.0, q=0.0, kernel=sca.KERNEL_WAVE) as sim:
        sim.set_state(start, t=0)
        sim.set_temporal_block(16)
        sim.track_origin(True)
        obs = sim.run(times)
    assert [(g.h00, g.S1) for g in obs] == _oracle_h00(L, L, 5, 1.0, 0.0, times, start=start)


def test_origin_height_closed_form_large(sca):
    """L = 65536, p = 1 from flat: every site deposits once per MCS, so h00 = 2t and the
    absolute mean height h00 + S1/N = 2t + 1/2."""
    with sca.Sim(65536, seed=1, p=1.0, q=0.0) as sim:
        sim.track_origin(True)
        obs = sim.run([1, 16, 40])
    for g in obs:
        assert g.h00 == 2 * g.t and 2 * g.S1 == g.N


def test_origin_tracking_needs_a_surface(sca):
    with sca.Sim(512, seed=1, p=0.5, q=0.0) as sim:
        w = sim.get_state()
        w[9] ^= 1
        sim.set_state(w, t=0)
        sim.set_kernel(sca.KERNEL_TWO_PASS)
        sim.track_origin(True)
        with pytest.raises(sca.ScaError) as e:
            sim.step(1)
        assert e.value.code == sca.ESTATE
        sim.track_origin(False)
        sim.step(1)


@pytest.mark.parametrize("L,p,q,times,k", [
    (1024, 0.75, 0.25, [1, 1, 2, 6, 6, 7, 23, 24, 40], 4),
    (1024, 1.0, 1.0, [3, 3, 16, 17, 49, 49, 80], 16),
    (768, 0.7, 0.3, [1, 3, 3, 8, 13], 2),
])
def test_run_observations_against_oracle(sca, L, p, q, times, k):
    """Every observation of a run equals the oracle's sums at its time, including a repeated
    time (no launch between two observations) and gaps of several launches; the final state
    too."""
    seed = 17
    with sca.Sim(L, seed=seed, p=p, q=q, kernel=sca.KERNEL_WAVE) as sim:
        sim.set_temporal_block(k)
        assert sim.kernel_in_use() == sca.KERNEL_WAVE
        obs = sim.run(times)
        words = sim.get_state()
    bx, by = o.init_flat(L)
    t = 0
    for g, tt in zip(obs, times):
        o.run(bx, by, seed, p, q, t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe(bx, by)
        assert (g.t, g.status, g.S1, g.S2, g.num) == (tt, 0, r["S1"], r["S2"], r["num"]), tt
    assert np.array_equal(words, o.pack(bx, by))


@pytest.mark.parametrize("L,p,q,times", [(8192, 1.0, 0.0, [16, 16, 17, 49, 50, 130]),
                                         (16384, 0.5, 0.0, [4, 8, 8, 9, 28, 60])])
def test_run_observations_large(sca, L, p, q, times):
    """From a rough surface (3 MCS of p = 5/8, q = 3/8) at larger sizes: the run's observations
    and final state on the wavefront kernel equal those of the two-pass kernel."""
    import torch
    with sca.Sim(L, seed=31, p=0.625, q=0.375, kernel=sca.KERNEL_TWO_PASS) as sim:
        sim.step(3)
        words = sim.get_state()
    res = []
    for kernel in (sca.KERNEL_WAVE, sca.KERNEL_TWO_PASS):
        with sca.Sim(L, seed=5, p=p, q=q, kernel=kernel) as sim:
            sim.set_state(words, t=0)
            assert sim.kernel_in_use() == kernel
            obs = sim.run(times)
            res.append(([(g.t, g.status, g.S1, g.S2, g.num) for g in obs], sim.state_tensor().clone()))
    assert res[0][0] == res[1][0]
    assert torch.equal(res[0][1], res[1][1])
