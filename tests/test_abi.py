"""The C-ABI library builds, loads without a GPU, exports every symbol include/sca.h declares,
and rejects bad arguments on the host before touching the device (CPU only; no compute)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00310_gb300 import build
    build.build()
    import paper_1606_00310_gb300.sca as sca
    return sca.load()


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(sca_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_functions():
    assert {"sca_init", "sca_step", "sca_observe", "sca_free"} <= set(header_functions())


def test_every_declared_symbol_is_exported(lib):
    import paper_1606_00310_gb300.sca as sca
    for name in header_functions():
        assert hasattr(lib, name), name
        assert name in sca.SIGNATURES, "binding lacks " + name


def test_struct_sizes_match_header(lib):
    import paper_1606_00310_gb300.sca as sca
    assert C.sizeof(sca.sca_obs) == 72
    assert C.sizeof(sca.sca_params) == 32


def test_workspace_bytes(lib):
    import paper_1606_00310_gb300.sca as sca
    assert sca.workspace_bytes(63) == 0
    assert sca.workspace_bytes(0) == 0
    assert sca.workspace_bytes(131072 + 64) == 0
    L = 65536
    state = L * L // 4
    assert 2 * state <= sca.workspace_bytes(L) <= 2 * state + (8 << 20)
    assert sca.workspace_bytes(64) >= 2 * 64 * 64 // 4


@pytest.mark.parametrize("L,p,q,rng", [(100, 0.5, 0.0, 0), (64, 1.5, 0.0, 0), (64, 0.5, -0.1, 0),
                                       (64, 0.3, 0.0, 1), (64, 0.5, 0.0, 7)])
def test_init_rejects_bad_parameters_on_host(lib, L, p, q, rng):
    import paper_1606_00310_gb300.sca as sca
    prm = sca.sca_params(L=L, rng=rng, seed=1, p=p, q=q)
    h = C.c_void_p()
    rc = lib.sca_init(C.byref(prm), None, None, 0, C.byref(h))
    assert rc == sca.EINVAL
    assert not h.value
    assert lib.sca_last_error()


def test_strerror_names_every_status(lib):
    for code in range(0, -10, -1):
        assert lib.sca_strerror(code) not in (None, b"unknown status")


def test_null_handles_are_refused_on_host(lib):
    """Every entry point that takes a simulation, batch or server handle refuses NULL with
    SCA_EINVAL before touching a device."""
    import paper_1606_00310_gb300.sca as sca
    buf = (C.c_uint32 * 16)()
    assert lib.sca_batch_set_state(None, 0, buf, 16) == sca.EINVAL
    assert lib.sca_batch_get_state(None, 0, buf, 16) == sca.EINVAL
    assert lib.sca_batch_reset(None) == sca.EINVAL
    assert lib.sca_set_wave_bands(None, 0) == sca.EINVAL
    assert lib.sca_set_temporal_block(None, 0) == sca.EINVAL
    assert lib.sca_set_kernel(None, 0) == sca.EINVAL
    assert lib.sca_step(None, 1) == sca.EINVAL
