"""Python binding of libsca (include/sca.h): argument marshalling only.

Every step of the dynamics and every observable runs in the library's CUDA kernels.  PyTorch
supplies device memory (the workspace tensor handed to ``sca_init``) and the stream.  There is
no fallback: if the compiled library is missing or fails to load, construction raises.
"""
import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsca.so")

OK, EINVAL, ENOMEM, ECUDA, EBUDGET, ETIMEOUT, EBUSY, ESTATE, ENOTFOUND, ECANCELED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
RNG_AUTO, RNG_DYADIC, RNG_UNIFORM32 = 0, 1, 2
KERNEL_AUTO, KERNEL_TWO_PASS, KERNEL_FUSED, KERNEL_TBLOCK, KERNEL_WAVE = 0, 1, 2, 3, 4
KERNEL_RANDOM_SEQUENTIAL = 5          # reported by kernel_in_use() for DYN_RANDOM_SEQUENTIAL
DYN_SCA, DYN_RANDOM_SEQUENTIAL = 0, 1


class sca_params(C.Structure):
    _fields_ = [("L", C.c_uint32), ("rng", C.c_uint32), ("seed", C.c_uint64),
                ("p", C.c_double), ("q", C.c_double), ("Ly", C.c_uint32), ("dynamics", C.c_uint32)]


class sca_obs(C.Structure):
    _fields_ = [("t", C.c_uint64), ("N", C.c_uint64), ("S1", C.c_int64),
                ("S2_lo", C.c_uint64), ("S2_hi", C.c_uint64),
                ("num_lo", C.c_uint64), ("num_hi", C.c_uint64),
                ("w2", C.c_double), ("status", C.c_int32), ("reserved", C.c_int32),
                ("h00", C.c_int64)]


OBS_RECORD_BYTES = C.sizeof(sca_obs)


class sca_corr(C.Structure):
    _fields_ = [("t", C.c_uint64), ("N", C.c_uint64), ("Sa", C.c_int64), ("Sb", C.c_int64),
                ("Sab_lo", C.c_uint64), ("Sab_hi", C.c_int64), ("cnum_lo", C.c_uint64),
                ("cnum_hi", C.c_int64), ("c", C.c_double), ("status", C.c_int32),
                ("reserved", C.c_int32)]


class sca_request_info(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("n_mcs", C.c_uint64), ("n_obs", C.c_uint32),
                ("status", C.c_int32), ("L", C.c_uint32), ("reserved", C.c_uint32),
                ("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double)]


class sca_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("failed", C.c_uint64), ("active", C.c_uint32),
                ("pending", C.c_uint32), ("bytes_in_use", C.c_uint64),
                ("budget_bytes", C.c_uint64), ("updates_done", C.c_uint64)]


# Every symbol include/sca.h declares, with its ctypes signature.
SIGNATURES = {
    "sca_workspace_bytes": (C.c_size_t, [C.c_uint32]),
    "sca_workspace_bytes_xy": (C.c_size_t, [C.c_uint32, C.c_uint32]),
    "sca_init": (C.c_int, [C.POINTER(sca_params), C.c_void_p, C.c_void_p, C.c_size_t,
                           C.POINTER(C.c_void_p)]),
    "sca_reset": (C.c_int, [C.c_void_p]),
    "sca_step": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sca_observe": (C.c_int, [C.c_void_p, C.POINTER(sca_obs)]),
    "sca_run": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.c_uint32, C.POINTER(sca_obs)]),
    "sca_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sca_correlate": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(sca_corr)]),
    "sca_track_origin": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint64]),
    "sca_state_device": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "sca_time": (C.c_uint64, [C.c_void_p]),
    "sca_set_kernel": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_get_kernel": (C.c_int, [C.c_void_p]),
    "sca_set_fused_shape": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "sca_set_temporal_block": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_set_wave_bands": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_measure_logic_rate": (C.c_int, [C.POINTER(C.c_double)]),
    "sca_measure_mul_rate": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sca_batch_set_engine": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_batch_get_engine": (C.c_int, [C.c_void_p]),
    "sca_set_state_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint64]),
    "sca_get_state_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sca_run_async": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.c_uint32]),
    "sca_wait": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32]),
    "sca_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "sca_timing_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "sca_free": (None, [C.c_void_p]),
    "sca_batch_init": (C.c_int, [C.POINTER(sca_params), C.c_uint32, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "sca_batch_set_shape": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "sca_batch_get_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sca_batch_tune": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sca_batch_run": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.c_uint32, C.c_void_p,
                                C.c_void_p]),
    "sca_batch_get_state": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t]),
    "sca_batch_set_state": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t]),
    "sca_batch_unit_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32]),
    "sca_batch_reset": (C.c_int, [C.c_void_p]),
    "sca_batch_time": (C.c_uint64, [C.c_void_p]),
    "sca_batch_free": (None, [C.c_void_p]),
    "sca_server_create": (C.c_int, [C.c_size_t, C.c_uint32, C.c_uint32, C.POINTER(C.c_void_p)]),
    "sca_server_submit": (C.c_int, [C.c_void_p, C.POINTER(sca_params), C.c_uint64, C.c_void_p,
                                    C.c_uint32, C.POINTER(C.c_uint64)]),
    "sca_server_submit_state": (C.c_int, [C.c_void_p, C.POINTER(sca_params), C.c_uint64, C.c_void_p,
                                          C.c_uint32, C.c_void_p, C.c_size_t, C.POINTER(C.c_uint64)]),
    "sca_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32, C.c_void_p]),
    "sca_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_uint32,
                                  C.c_void_p]),
    "sca_server_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sca_server_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sca_server_get_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sca_server_destroy": (None, [C.c_void_p]),
    "sca_observe_noalloc": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p,
                                      C.POINTER(sca_obs)]),
    "sca_strerror": (C.c_char_p, [C.c_int]),
    "sca_last_error": (C.c_char_p, []),
    "sca_kernel_launches": (C.c_uint64, []),
    "sca_selftest_wait_timeout": (C.c_int, [C.c_uint32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsca.so and attach signatures.  Raises if it is missing: no fallback exists."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsca.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ScaError(RuntimeError):
    def __init__(self, code, where, detail=None):
        lib = load()
        msg = "%s: %s (%s)" % (where, lib.sca_strerror(code).decode(),
                               detail if detail is not None else lib.sca_last_error().decode())
        super().__init__(msg)
        self.code = code


def check(code, where):
    if code != OK:
        raise ScaError(code, where)


def workspace_bytes(L: int, Ly: int = None) -> int:
    """Device bytes of one simulation of L x L sites, or of L sites per row and Ly rows."""
    if Ly is None:
        return int(load().sca_workspace_bytes(L))
    return int(load().sca_workspace_bytes_xy(L, Ly))


def measure_logic_rate() -> float:
    """Measured 32-bit three-input logic instructions per second of the current GPU."""
    r = C.c_double()
    check(load().sca_measure_logic_rate(C.byref(r)), "sca_measure_logic_rate")
    return float(r.value)


def measure_mul_rate():
    """(32x32->64 multiply-adds per second, Philox4x32-10 calls per second) on this GPU."""
    m = C.c_double()
    p = C.c_double()
    check(load().sca_measure_mul_rate(C.byref(m), C.byref(p)), "sca_measure_mul_rate")
    return float(m.value), float(p.value)


def kernel_launches() -> int:
    return int(load().sca_kernel_launches())


@dataclass
class Obs:
    t: int
    N: int
    S1: int
    S2: int
    num: int
    w2: float
    status: int
    h00: int = 0          # absolute height of the origin (while tracked; see Sim.track_origin)

    @staticmethod
    def from_c(o: sca_obs) -> "Obs":
        return Obs(t=int(o.t), N=int(o.N), S1=int(o.S1),
                   S2=int(o.S2_lo) | (int(o.S2_hi) << 64),
                   num=int(o.num_lo) | (int(o.num_hi) << 64), w2=float(o.w2),
                   status=int(o.status), h00=int(o.h00))


@dataclass
class Corr:
    """Two-time height correlation: C = cnum / N^2 (cnum = N Sab - Sa Sb, exact)."""
    t: int
    N: int
    Sa: int
    Sb: int
    Sab: int
    cnum: int
    c: float
    status: int

    @staticmethod
    def from_c(o: sca_corr) -> "Corr":
        return Corr(o.t, o.N, o.Sa, o.Sb, (o.Sab_hi << 64) | o.Sab_lo, (o.cnum_hi << 64) | o.cnum_lo,
                    o.c, o.status)


def observe_noalloc(words_dev_ptr: int, L: int, t: int = 0, stream=None) -> Obs:
    """Exact roughness of caller-owned device words without any library allocation (the
    scratch is a fixed device array shared by all calls; serialise overlapping calls)."""
    o = sca_obs()
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = load().sca_observe_noalloc(C.c_void_p(words_dev_ptr), int(L), int(t), st, C.byref(o))
    if rc not in (OK, ESTATE):
        check(rc, "sca_observe_noalloc")
    return Obs.from_c(o)


def words_count(L: int, Ly: int = None) -> int:
    """Canonical words of an L x L lattice, or of L sites per row and Ly rows."""
    return 4 * (L if Ly is None else Ly) * (L // 64)


class Sim:
    """One L x L lattice on the current CUDA device, flat at MCS 0; with Ly, a lattice of L
    sites per row and Ly rows.

    ``workspace`` may be a caller-owned uint8 CUDA tensor of at least workspace_bytes(L, Ly);
    otherwise one is allocated with PyTorch.  ``stream`` is a torch.cuda.Stream (default: a new
    stream of the current device); all of the simulation's kernels run on it."""

    def __init__(self, L, seed=1, p=1.0, q=0.0, rng=RNG_AUTO, stream=None, workspace=None,
                 kernel=KERNEL_AUTO, Ly=None, dynamics=DYN_SCA):
        import torch
        lib = load()
        self.L = int(L)
        self.Ly = self.L if Ly is None else int(Ly)
        nbytes = workspace_bytes(self.L, self.Ly)
        if nbytes == 0:
            raise ScaError(EINVAL, "L=%d Ly=%d" % (self.L, self.Ly),
                           "L must be a multiple of 64 in [64, 131072] and Ly even in [2, 131072]")
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if workspace.numel() * workspace.element_size() < nbytes or not workspace.is_cuda:
            raise ValueError("workspace must be a CUDA tensor of at least %d bytes" % nbytes)
        self.workspace = workspace
        if stream is None:
            stream = torch.cuda.Stream()
            stream.wait_stream(torch.cuda.current_stream())   # workspace allocation order
        self.stream = stream
        prm = sca_params(L=self.L, rng=rng, seed=seed, p=p, q=q,
                         Ly=0 if self.Ly == self.L else self.Ly, dynamics=int(dynamics))
        h = C.c_void_p()
        check(lib.sca_init(C.byref(prm), C.c_void_p(self.stream.cuda_stream),
                           C.c_void_p(workspace.data_ptr()), nbytes, C.byref(h)), "sca_init")
        self._h = h
        self.params = dict(L=self.L, Ly=self.Ly, seed=seed, p=p, q=q, rng=rng, dynamics=int(dynamics))
        if kernel != KERNEL_AUTO:
            self.set_kernel(kernel)

    # -- dynamics
    def reset(self):
        check(load().sca_reset(self._h), "sca_reset")

    def step(self, n_mcs: int):
        check(load().sca_step(self._h, int(n_mcs)), "sca_step")

    def set_kernel(self, kernel: int):
        check(load().sca_set_kernel(self._h, int(kernel)), "sca_set_kernel")

    def set_temporal_block(self, mcs_per_launch: int):
        check(load().sca_set_temporal_block(self._h, int(mcs_per_launch)), "sca_set_temporal_block")

    def set_wave_bands(self, bands: int):
        check(load().sca_set_wave_bands(self._h, int(bands)), "sca_set_wave_bands")

    def set_fused_shape(self, words_per_thread: int, ring: int):
        check(load().sca_set_fused_shape(self._h, int(words_per_thread), int(ring)),
              "sca_set_fused_shape")

    def kernel_in_use(self) -> int:
        return int(load().sca_get_kernel(self._h))

    @property
    def t(self) -> int:
        return int(load().sca_time(self._h))

    # -- observables
    def observe(self) -> Obs:
        o = sca_obs()
        rc = load().sca_observe(self._h, C.byref(o))
        if rc not in (OK, ESTATE):
            check(rc, "sca_observe")
        return Obs.from_c(o)

    def run(self, times):
        times = [int(x) for x in times]
        n = len(times)
        arr = (C.c_uint64 * n)(*times)
        out = (sca_obs * n)()
        rc = load().sca_run(self._h, arr, n, out)
        if rc not in (OK, ESTATE):
            check(rc, "sca_run")
        return [Obs.from_c(o) for o in out]

    def track_origin(self, enable: bool = True):
        """Carry the origin's absolute height through the updates (observations report h00)."""
        check(load().sca_track_origin(self._h, 1 if enable else 0), "sca_track_origin")

    def snapshot(self):
        """A device copy (int32 CUDA tensor) of the current canonical words, the reference state
        of a later correlate()."""
        return self.state_tensor().clone()

    def correlate(self, ref) -> "Corr":
        """Two-time height correlation of the current state with ``ref``, a CUDA tensor holding
        canonical words of this lattice (e.g. from snapshot())."""
        import torch
        n = words_count(self.L, self.Ly)
        if not ref.is_cuda or ref.numel() * ref.element_size() != 4 * n or not ref.is_contiguous():
            raise ValueError("ref must be a contiguous CUDA tensor of %d words" % n)
        self.stream.wait_stream(torch.cuda.current_stream())
        o = sca_corr()
        rc = load().sca_correlate(self._h, C.c_void_p(ref.data_ptr()), C.byref(o))
        if rc not in (OK, ESTATE):
            check(rc, "sca_correlate")
        return Corr.from_c(o)

    # -- kernel timing (CUDA events around update launches on this simulation's stream)
    def timing(self, enable: bool):
        check(load().sca_timing(self._h, 1 if enable else 0), "sca_timing")

    def timing_read(self):
        ms = C.c_double()
        n = C.c_uint64()
        check(load().sca_timing_read(self._h, C.byref(ms), C.byref(n)), "sca_timing_read")
        return float(ms.value), int(n.value)

    # -- state
    def get_state(self, out: np.ndarray = None) -> np.ndarray:
        n = words_count(self.L, self.Ly)
        if out is None:
            out = np.empty(n, dtype=np.uint32)
        assert out.dtype == np.uint32 and out.size >= n and out.flags.c_contiguous
        check(load().sca_get_state(self._h, out.ctypes.data_as(C.c_void_p), n), "sca_get_state")
        return out

    def set_state(self, words: np.ndarray, t: int = 0):
        words = np.ascontiguousarray(words, dtype=np.uint32)
        check(load().sca_set_state(self._h, words.ctypes.data_as(C.c_void_p), words.size, int(t)),
              "sca_set_state")

    def set_state_ptr(self, host_ptr: int, n_words: int, t: int = 0):
        """Set the state from a host pointer (e.g. a pinned torch CPU tensor's data_ptr())."""
        check(load().sca_set_state(self._h, C.c_void_p(host_ptr), int(n_words), int(t)),
              "sca_set_state")

    def get_state_ptr(self, host_ptr: int, n_words: int):
        check(load().sca_get_state(self._h, C.c_void_p(host_ptr), int(n_words)), "sca_get_state")

    # -- asynchronous host I/O and runs (enqueue only; collect with wait())
    def set_state_ptr_async(self, host_ptr: int, n_words: int, t: int = 0):
        check(load().sca_set_state_async(self._h, C.c_void_p(host_ptr), int(n_words), int(t)),
              "sca_set_state_async")

    def get_state_ptr_async(self, host_ptr: int, n_words: int):
        check(load().sca_get_state_async(self._h, C.c_void_p(host_ptr), int(n_words)),
              "sca_get_state_async")

    def run_async(self, times):
        times = [int(x) for x in times]
        n = len(times)
        arr = (C.c_uint64 * n)(*times)
        check(load().sca_run_async(self._h, arr, n), "sca_run_async")
        self._async_n = n

    def wait(self):
        """Synchronise and return the last run_async's observations."""
        n = getattr(self, "_async_n", 0)
        out = (sca_obs * max(n, 1))()
        rc = load().sca_wait(self._h, C.cast(out, C.c_void_p), n)
        self._async_n = 0
        if rc not in (OK, ESTATE):
            check(rc, "sca_wait")
        return [Obs.from_c(out[i]) for i in range(n)]

    def state_tensor(self):
        """The current canonical words as a uint32-viewed slice of the workspace tensor."""
        import torch
        p = C.c_void_p()
        check(load().sca_state_device(self._h, C.byref(p)), "sca_state_device")
        off = p.value - self.workspace.data_ptr()
        n = words_count(self.L, self.Ly)
        torch.cuda.current_stream().wait_stream(self.stream)
        return self.workspace[off:off + 4 * n].view(torch.int32)

    def close(self):
        if getattr(self, "_h", None):
            load().sca_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """An ensemble of independent lattices advanced by one persistent, graph-captured launch.

    ``lattices``: iterable of dicts with keys L, p, q, seed and optional rng."""

    def __init__(self, lattices, stream=None):
        import torch
        lib = load()
        lat = list(lattices)
        self.Ls = [int(d["L"]) for d in lat]
        arr = (sca_params * len(lat))()
        for i, d in enumerate(lat):
            arr[i] = sca_params(L=int(d["L"]), rng=int(d.get("rng", RNG_AUTO)),
                                seed=int(d["seed"]), p=float(d["p"]), q=float(d["q"]))
        if stream is None:
            stream = torch.cuda.Stream()
        self.stream = stream
        h = C.c_void_p()
        check(lib.sca_batch_init(arr, len(lat), C.c_void_p(stream.cuda_stream), C.byref(h)),
              "sca_batch_init")
        self._h = h
        self.count = len(lat)

    def set_shape(self, cluster: int, threads: int):
        check(load().sca_batch_set_shape(self._h, int(cluster), int(threads)), "sca_batch_set_shape")

    def set_engine(self, engine: int):
        check(load().sca_batch_set_engine(self._h, int(engine)), "sca_batch_set_engine")

    def engine(self) -> int:
        return int(load().sca_batch_get_engine(self._h))

    def tune(self, probe_mcs: int = 32):
        c, t = C.c_int(), C.c_int()
        check(load().sca_batch_tune(self._h, int(probe_mcs), C.byref(c), C.byref(t)),
              "sca_batch_tune")
        return c.value, t.value

    def shape(self):
        c, t, n, u = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(load().sca_batch_get_shape(self._h, C.byref(c), C.byref(t), C.byref(n), C.byref(u)),
              "sca_batch_get_shape")
        return {"cluster": c.value, "threads": t.value, "clusters": n.value, "units": u.value}

    def run(self, times, want_obs=True):
        """Returns (obs[lattice][k], ensemble_w2[k])."""
        times = [int(x) for x in times]
        n = len(times)
        arr = (C.c_uint64 * n)(*times)
        out = (sca_obs * (self.count * n))() if want_obs else None
        ens = (C.c_double * n)()
        rc = load().sca_batch_run(self._h, arr, n, C.cast(out, C.c_void_p) if want_obs else None,
                                  C.cast(ens, C.c_void_p))
        if rc not in (OK, ESTATE):
            check(rc, "sca_batch_run")
        obs = None
        if want_obs:
            obs = [[Obs.from_c(out[i * n + k]) for k in range(n)] for i in range(self.count)]
        return obs, list(ens)

    def unit_times(self):
        """(start_ns, end_ns, first_lattice) per work unit of the last run."""
        u = self.shape()["units"]
        st = np.zeros(u, np.uint64)
        en = np.zeros(u, np.uint64)
        fl = np.zeros(u, np.int32)
        check(load().sca_batch_unit_times(self._h, st.ctypes.data_as(C.c_void_p),
                                          en.ctypes.data_as(C.c_void_p),
                                          fl.ctypes.data_as(C.c_void_p), u), "sca_batch_unit_times")
        return st, en, fl

    def get_state(self, index: int) -> np.ndarray:
        n = words_count(self.Ls[index])
        out = np.empty(n, dtype=np.uint32)
        check(load().sca_batch_get_state(self._h, int(index), out.ctypes.data_as(C.c_void_p), n),
              "sca_batch_get_state")
        return out

    def set_state(self, index: int, words: np.ndarray):
        """Lattice `index` from canonical words (a surface); the batch time is unchanged."""
        w = np.ascontiguousarray(words, dtype=np.uint32)
        check(load().sca_batch_set_state(self._h, int(index), w.ctypes.data_as(C.c_void_p), w.size),
              "sca_batch_set_state")

    def reset(self):
        check(load().sca_batch_reset(self._h), "sca_batch_reset")

    @property
    def t(self) -> int:
        return int(load().sca_batch_time(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().sca_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server (native scheduler thread inside the library)."""

    def __init__(self, budget_bytes: int, max_active: int = 64, max_L: int = 8192):
        lib = load()
        h = C.c_void_p()
        check(lib.sca_server_create(int(budget_bytes), int(max_active), int(max_L), C.byref(h)),
              "sca_server_create")
        self._h = h
        self._keep = {}         # final-state buffers of requests not yet released

    def submit(self, L, p, q, seed, n_mcs, times=None, rng=RNG_AUTO, final_words=None) -> int:
        """Queue a request; with final_words (a C-contiguous uint32 array of 4 * L * L/64 words,
        kept alive here until the request is released) its final state comes back there."""
        prm = sca_params(L=int(L), rng=int(rng), seed=int(seed), p=float(p), q=float(q))
        tk = C.c_uint64()
        arr = (C.c_uint64 * len(times))(*[int(x) for x in times]) if times else None
        tptr = C.cast(arr, C.c_void_p) if times else None
        nt = len(times) if times else 0
        if final_words is not None:
            if final_words.dtype != np.uint32 or not final_words.flags["C_CONTIGUOUS"]:
                raise ValueError("final_words must be a C-contiguous uint32 array")
            rc = load().sca_server_submit_state(self._h, C.byref(prm), int(n_mcs), tptr, nt,
                                                final_words.ctypes.data, final_words.size, C.byref(tk))
        else:
            rc = load().sca_server_submit(self._h, C.byref(prm), int(n_mcs), tptr, nt, C.byref(tk))
        check(rc, "sca_server_submit")
        if final_words is not None:
            self._keep[int(tk.value)] = final_words
        return int(tk.value)

    def _result(self, fn, ticket, *extra):
        out = (sca_obs * 64)()
        info = sca_request_info()
        rc = fn(self._h, int(ticket), *extra, C.cast(out, C.c_void_p), 64, C.byref(info))
        if rc in (ENOTFOUND, EINVAL):
            raise ScaError(rc, "request %d" % ticket)
        obs = [Obs.from_c(out[i]) for i in range(info.n_obs)] if rc in (OK, ESTATE) else None
        return rc, obs, info

    def poll(self, ticket):
        """(status, observations or None, info)."""
        return self._result(load().sca_server_poll, ticket)

    def wait(self, ticket, timeout_ms: int = -1):
        return self._result(load().sca_server_wait, ticket, int(timeout_ms))

    def cancel(self, ticket):
        check(load().sca_server_cancel(self._h, int(ticket)), "sca_server_cancel")

    def release(self, ticket):
        check(load().sca_server_release(self._h, int(ticket)), "sca_server_release")
        self._keep.pop(int(ticket), None)

    def stats(self) -> dict:
        st = sca_server_stats()
        check(load().sca_server_get_stats(self._h, C.byref(st)), "sca_server_get_stats")
        return {k: getattr(st, k) for k, _ in sca_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().sca_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
