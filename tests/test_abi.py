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


def _c_layout(struct, fields):
    """sizeof and field offsets of a header struct, as the C compiler lays it out."""
    import subprocess
    import tempfile
    prog = "#include <stddef.h>\n#include <stdio.h>\n#include \"sca.h\"\nint main(void){printf(\"%%zu\", sizeof(%s));" % struct
    for f in fields:
        prog += 'printf(" %%zu", offsetof(%s, %s));' % (struct, f)
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), src, "-o", exe])
        return [int(v) for v in subprocess.check_output([exe]).split()]


def test_struct_layouts_match_header(lib):
    """The binding's ctypes structures have the header's size and field offsets."""
    import paper_1606_00310_gb300.sca as sca
    for cls, name in ((sca.sca_params, "sca_params"), (sca.sca_obs, "sca_obs"),
                      (sca.sca_request_info, "sca_request_info"),
                      (sca.sca_server_stats, "sca_server_stats")):
        fields = [f for f, _ in cls._fields_]
        got = _c_layout(name, fields)
        assert got[0] == C.sizeof(cls), name
        assert got[1:] == [getattr(cls, f).offset for f in fields], name


def test_workspace_bytes(lib):
    import paper_1606_00310_gb300.sca as sca
    assert sca.workspace_bytes(63) == 0
    assert sca.workspace_bytes(0) == 0
    assert sca.workspace_bytes(131072 + 64) == 0
    L = 65536
    state = L * L // 4
    assert 2 * state <= sca.workspace_bytes(L) <= 2 * state + (8 << 20)
    assert sca.workspace_bytes(64) >= 2 * 64 * 64 // 4


def test_workspace_bytes_xy(lib):
    import paper_1606_00310_gb300.sca as sca
    assert sca.workspace_bytes(4096, 4096) == sca.workspace_bytes(4096)
    for X, Y in ((64, 0), (64, 3), (64, 131074), (100, 64), (131136, 2)):
        assert sca.workspace_bytes(X, Y) == 0, (X, Y)
    X, Y = 131072, 64
    state = X * Y // 4
    assert 2 * state <= sca.workspace_bytes(X, Y) <= 2 * state + (1 << 20)
    assert sca.workspace_bytes(64, 131072) >= 2 * 64 * 131072 // 4


@pytest.mark.parametrize("L,Ly", [(64, 3), (64, 131074), (128, 1)])
def test_init_rejects_bad_row_counts_on_host(lib, L, Ly):
    import paper_1606_00310_gb300.sca as sca
    prm = sca.sca_params(L=L, rng=0, seed=1, p=0.5, q=0.0, Ly=Ly)
    h = C.c_void_p()
    assert lib.sca_init(C.byref(prm), None, None, 0, C.byref(h)) == sca.EINVAL
    assert not h.value


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
