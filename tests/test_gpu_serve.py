"""Serving loop (continuous batching): each request's result is the same alone and in the mix
(tolerance: zero, integer results), admission respects slots and the memory budget, and
cancellation, timeouts and bad requests are reported through status codes."""
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


REQS = [
    dict(L=256, p=0.7, q=0.3, seed=1, n=200), dict(L=320, p=0.875, q=0.125, seed=2, n=150),
    dict(L=512, p=0.6180339887, q=0.3819660113, seed=3, n=300), dict(L=1024, p=0.5, q=0.0, seed=4, n=130),
    dict(L=2048, p=0.9, q=0.1, seed=5, n=140), dict(L=4096, p=0.75, q=0.25, seed=6, n=70),
    dict(L=640, p=0.55, q=0.45, seed=7, n=257), dict(L=256, p=1.0, q=0.0, seed=8, n=129),
    dict(L=2112, p=0.8, q=0.2, seed=9, n=65), dict(L=768, p=0.95, q=0.05, seed=10, n=400),
]


def key(obs):
    return [(x.t, x.S1, x.S2, x.num) for x in obs]


def test_alone_and_in_the_mix_are_identical(sca):
    with sca.Server(budget_bytes=8 << 30, max_active=6, max_L=4096) as srv:
        tickets = [srv.submit(r["L"], r["p"], r["q"], r["seed"], r["n"]) for r in REQS]
        mixed = []
        for tk in tickets:
            rc, obs, info = srv.wait(tk, timeout_ms=120000)
            assert rc == sca.OK, (rc, info.status)
            assert info.done_s >= info.admit_s >= info.submit_s > 0
            mixed.append(obs)
        st = srv.stats()
        assert st["completed"] == len(REQS) and st["failed"] == 0
    for r, obs in zip(REQS, mixed):
        times = [x.t for x in obs]
        assert times[-1] == r["n"]
        with sca.Sim(r["L"], seed=r["seed"], p=r["p"], q=r["q"]) as sim:
            alone = sim.run(times)
        assert key(obs) == key(alone), r


def test_served_result_matches_oracle(sca):
    r = dict(L=256, p=0.7, q=0.3, seed=11, n=140)
    with sca.Server(budget_bytes=1 << 30, max_active=2, max_L=512) as srv:
        rc, obs, _ = srv.wait(srv.submit(r["L"], r["p"], r["q"], r["seed"], r["n"]), 60000)
    assert rc == sca.OK
    bx, by = o.init_flat(r["L"])
    t = 0
    for x in obs:
        o.run(bx, by, r["seed"], r["p"], r["q"], t0=t, n_mcs=x.t - t)
        t = x.t
        ref = o.observe(bx, by)
        assert (x.S1, x.S2, x.num) == (ref["S1"], ref["S2"], ref["num"])


def _max_overlap(infos):
    ev = []
    for i in infos:
        ev.append((i.admit_s, 1))
        ev.append((i.done_s, -1))
    ev.sort(key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def test_admission_respects_slots_and_budget(sca):
    need = sca.workspace_bytes(1024) + 256
    # budget for three 1024 lattices, six slots: memory binds
    with sca.Server(budget_bytes=3 * need + 1000, max_active=6, max_L=2048) as srv:
        tks = [srv.submit(1024, 0.7, 0.3, s, 200) for s in range(8)]
        infos = [srv.wait(tk, 120000)[2] for tk in tks]
        assert all(i.status == sca.OK for i in infos)
        assert _max_overlap(infos) <= 3
        with pytest.raises(sca.ScaError) as e:
            srv.submit(2048, 0.5, 0.0, 1, 10)           # its state alone exceeds the budget
        assert e.value.code == sca.EBUDGET
    # two slots, ample memory: slots bind
    with sca.Server(budget_bytes=8 << 30, max_active=2, max_L=2048) as srv:
        tks = [srv.submit(512, 0.6, 0.2, s, 300) for s in range(6)]
        infos = [srv.wait(tk, 120000)[2] for tk in tks]
        assert all(i.status == sca.OK for i in infos)
        assert _max_overlap(infos) <= 2
        order = sorted(range(6), key=lambda k: infos[k].admit_s)
        assert order == list(range(6))                    # admitted in arrival order


def test_cancel_timeout_and_bad_requests(sca):
    with sca.Server(budget_bytes=4 << 30, max_active=2, max_L=4096) as srv:
        long_tk = srv.submit(4096, 0.7, 0.3, 1, 10 ** 7)
        rc, _, info = srv.wait(long_tk, timeout_ms=50)
        assert rc == sca.ETIMEOUT and info.status == sca.EBUSY
        srv.cancel(long_tk)
        rc, obs, info = srv.wait(long_tk, timeout_ms=60000)
        assert rc == sca.ECANCELED and obs is None
        queued = [srv.submit(2048, 0.7, 0.3, s, 10 ** 6) for s in range(4)]
        for tk in queued:
            srv.cancel(tk)
        assert all(srv.wait(tk, 60000)[0] == sca.ECANCELED for tk in queued)
        ok = srv.submit(256, 0.7, 0.3, 5, 100)
        assert srv.wait(ok, 60000)[0] == sca.OK
        srv.release(ok)
        with pytest.raises(sca.ScaError) as e:
            srv.poll(ok)
        assert e.value.code == sca.ENOTFOUND
        for bad in [dict(L=100), dict(L=8192), dict(L=256, p=1.5)]:
            args = dict(L=256, p=0.5, q=0.0)
            args.update(bad)
            with pytest.raises(sca.ScaError) as e:
                srv.submit(args["L"], args["p"], args["q"], 1, 10)
            assert e.value.code == sca.EINVAL
        st = srv.stats()
        assert st["cancelled"] >= 5 and st["failed"] == 0


def test_request_stream_sample_against_oracle(sca):
    """Requests drawn from the serving workload (non-dyadic p, q = 1 - p, 512-8192 MCS): three
    small ones and one with L = 1152 (a row length that is not a power of two), served while
    larger ones from the same stream run beside them, equal the oracle at every observation
    time, and their final states (returned through sca_server_submit_state) equal the
    oracle's final words."""
    from paper_1606_00310_gb300 import workloads
    stream = workloads.request_stream(n=2000)
    small = [r for r in stream if r["L"] <= 384 and r["mcs"] <= 2000][:3]
    mid = [r for r in stream if r["id"] == 1017]
    assert mid[0]["L"] == 1152 and mid[0]["mcs"] == 563
    sample = small + mid
    big = [r for r in stream if r["L"] >= 2048][:4]
    assert len(small) == 3
    finals = [np.zeros(sca.words_count(r["L"]), np.uint32) for r in sample]
    with sca.Server(budget_bytes=16 << 30, max_active=8, max_L=8192) as srv:
        tk_big = [srv.submit(r["L"], r["p"], r["q"], r["seed"], r["mcs"]) for r in big]
        tk_s = [srv.submit(r["L"], r["p"], r["q"], r["seed"], r["mcs"], final_words=f)
                for r, f in zip(sample, finals)]
        results = [srv.wait(tk, 300000) for tk in tk_s]
        for tk in tk_big:
            srv.cancel(tk)
    for r, (rc, obs, _), fw in zip(sample, results, finals):
        assert rc == sca.OK
        bx, by = o.init_flat(r["L"])
        t = 0
        for x in obs:
            o.run(bx, by, r["seed"], r["p"], r["q"], mode=o.UNIFORM32, t0=t, n_mcs=x.t - t)
            t = x.t
            ref = o.observe(bx, by)
            assert (x.S1, x.S2, x.num) == (ref["S1"], ref["S2"], ref["num"]), (r, x.t)
        assert t == r["mcs"]
        assert np.array_equal(fw, o.pack(bx, by)), r


def test_submit_state_refuses_a_short_buffer(sca):
    with sca.Server(budget_bytes=1 << 30, max_active=1, max_L=512) as srv:
        with pytest.raises(sca.ScaError) as e:
            srv.submit(256, 0.5, 0.0, 1, 10, final_words=np.zeros(sca.words_count(256) - 1, np.uint32))
        assert e.value.code == sca.EINVAL


def test_served_kernels_agree(sca):
    """Requests whose lattice runs with temporal blocking (dyadic, small L), the two-pass kernel
    (per-site uniforms, which the server runs on it at every size) and the fused kernel (dyadic,
    L = 32768) all equal a single simulation with the kernel fixed to two-pass."""
    reqs = [dict(L=512, p=0.75, q=0.25, seed=3, n=200), dict(L=1024, p=0.7, q=0.3, seed=4, n=130),
            dict(L=4096, p=0.6, q=0.4, seed=5, n=66), dict(L=32768, p=0.5, q=0.0, seed=6, n=66)]
    with sca.Server(budget_bytes=8 << 30, max_active=4, max_L=32768) as srv:
        tks = [srv.submit(r["L"], r["p"], r["q"], r["seed"], r["n"]) for r in reqs]
        res = [srv.wait(tk, 300000) for tk in tks]
    for r, (rc, obs, _) in zip(reqs, res):
        assert rc == sca.OK
        with sca.Sim(r["L"], seed=r["seed"], p=r["p"], q=r["q"], kernel=sca.KERNEL_TWO_PASS) as sim:
            ref = sim.run([x.t for x in obs])
        assert key(obs) == key(ref), r
