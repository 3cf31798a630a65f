"""Failure detection without a GPU fault: a device-side wait that cannot complete gives up after
its limit, the host reads the error status, and the CUDA context stays usable."""
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


def test_bounded_wait_reports_timeout_and_context_survives(sca):
    lib = sca.load()
    for limit_us in (2000, 20000):
        assert lib.sca_selftest_wait_timeout(limit_us) == sca.ETIMEOUT
        assert b"gave up" in lib.sca_last_error()
    assert lib.sca_selftest_wait_timeout(0) == sca.EINVAL
    with sca.Sim(256, seed=1, p=1.0, q=0.0) as sim:      # the context still works
        obs = sim.run([1, 2])
        assert all(4 * o.num == o.N ** 2 for o in obs)
