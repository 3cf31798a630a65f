#!/usr/bin/env python3
"""Benchmark of the bit-vectorized octahedron-model SCA on one GB300 (or N independent replicas).

Workload (one "step"): an L = 65536 periodic lattice (4.3 G sites, 1 GiB of packed slopes),
flat start, p = 1, q = 0, 1024 Monte-Carlo steps with the exact roughness W^2 observed at
MCS 1, 2, 4, ..., 1024.  Metric: site updates per second (L^2 attempts per MCS).  The state
(1 GiB, read and written at least once per update launch, i.e. every MCS or every 16 MCS
depending on the kernel) is far larger than L2, so no flush is needed between steps.

Arms:
  default          the CUDA library through its C ABI, state resident in HBM;
  --impl reference the CPU oracle (test infrastructure, deliberately slow) on a bounded sample
                   of the same workload, on the host's cores.

With torchrun (WORLD_SIZE > 1) every rank runs its own replica on its own GPU (the update has no
exchange between independent lattices); value = all ranks' updates / max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving run keeps one stream per active request; let up to 32 of them run concurrently
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "site updates/s"
UNIT = "updates/s"
WORKLOAD = "octahedron SCA L=65536 p=1 q=0 flat, 1024 MCS, exact W^2 at 2^0..2^10"
BYTES_PER_UPDATE = 0.5   # each slope bit read once and written once per MCS (roofline unit)
# Height-bit wavefront kernel, one of p, q equal to 1 and the other 0: per 32-site word and
# half-step, two 3-input logic ops fold the four neighbour comparisons, one applies the flip,
# one funnel shift aligns the offset x-neighbour: 4 ALU-pipe ops per 32 site updates.
WAVE_ALU_OPS_PER_UPDATE = 4.0 / 32.0
# Paths that draw random numbers are bound by issue slots shared by the Philox rounds and the
# logic of the update: time per update = (Philox calls per update) / (measured Philox calls/s)
# + (logic ops per update outside Philox) / (measured logic ops/s), counts read off the source:
# - p = 1/2 on the height-bit kernel (four words per lane): one Philox call per lane, half-step
#   and 128 sites; the update takes 5 logic ops per 32-site word (two three-input ops folding
#   the four neighbour comparisons, one combining them with the draw, the flip, the funnel
#   shift of the offset neighbour);
# - per-site uniforms on the two-pass kernel: one call per 4 sites; per site two threshold
#   compares with their bit packing (about 5 ops), plus the word's mask and its four XORs
#   (about 12 ops per 32 sites).
P_HALF_CALLS_PER_UPDATE = 1.0 / 128.0
P_HALF_OPS_PER_UPDATE = 5.0 / 32.0
UNIFORM_CALLS_PER_UPDATE = 1.0 / 4.0
UNIFORM_OPS_PER_UPDATE = 5.0 + 12.0 / 32.0


def issue_bound(calls_per_update, ops_per_update, philox_rate, logic_rate):
    """Updates per second if the GPU did nothing but the path's Philox calls and logic ops at
    their measured rates, one after the other."""
    return 1.0 / (calls_per_update / philox_rate + ops_per_update / logic_rate)
ALU_LANES_PER_SM = 64    # 32-bit logic / shift results per clock per SM (4 SMSPs x 16 lanes)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=65536)
    ap.add_argument("--p", type=float, default=1.0)
    ap.add_argument("--q", type=float, default=0.0)
    ap.add_argument("--mcs", type=int, default=1024)
    ap.add_argument("--kernel", type=int, default=0,
                    help="0 auto, 1 two-pass, 2 fused, 3 shared-memory temporal blocking, "
                         "4 register wavefront on height bits")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the p=1/2 context line")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble line")
    ap.add_argument("--only", default="", choices=["", "batch", "serve"],
                    help="run only the batched ensemble (--batch-count/--batch-mcs) or the "
                         "serving stream (--serve-requests)")
    ap.add_argument("--batch-engine", type=int, default=0, choices=[0, 1, 2],
                    help="with --only batch: 0 automatic, 1 clusters, 2 streaming")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=96)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving line")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-mcs", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="seconds of oracle work per reference-arm step (default: about a "
                         "minute in total, 2 to 20 s per step)")
    return ap.parse_args()


def obs_times(mcs):
    t, out = 1, []
    while t < mcs:
        out.append(t)
        t *= 2
    out.append(mcs)
    return out


def config(a, world):
    return {"workload": WORKLOAD if (a.L, a.p, a.q, a.mcs) == (65536, 1.0, 0.0, 1024) else
            "octahedron SCA L=%d p=%g q=%g flat, %d MCS, exact W^2 at log times"
            % (a.L, a.p, a.q, a.mcs),
            "L": a.L, "p": a.p, "q": a.q, "mcs_per_step": a.mcs,
            "observations": len(obs_times(a.mcs)),
            "state_bytes": a.L * a.L // 4,
            "l2_policy": "state (%.2f GiB) exceeds L2 (129 MB); no flush needed"
                         % (a.L * a.L / 4 / 2 ** 30),
            "parallelism": "replicas x%d" % world}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
               "reasons": sorted(reasons), "samples": len(sm), "sm_mhz_min": min(sm)}
        if pw:
            out["power_w_median"] = statistics.median(pw)
        return out


# ----------------------------------------------------------------------------- roofline inputs
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def alu_peak_tops(n_sm):
    """Logic-op peak of the whole GPU in Tops/s: SMs x ALU lanes x maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return n_sm * ALU_LANES_PER_SM * mhz * 1e6 / 1e12, mhz


KERNEL_SOURCES = {
    "k_fused_mcs": ("sca_update.cu", "sca_fused.cu", "sca_rng.cuh", "sca_internal.h"),
    "k_half_step": ("sca_update.cu", "sca_fused.cu", "sca_rng.cuh", "sca_internal.h"),
    "k_wave": ("sca_wave.cuh", "sca_wave.cu", "sca_rng.cuh", "sca_internal.h"),
}


def kernel_source_hash(kernel_name="k_fused_mcs"):
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kernel_name]:
        with open(os.path.join(ROOT, "paper_1606_00310_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel_name, L):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel_name)
    if not e or e.get("src_sha256") != kernel_source_hash(kernel_name):
        return None
    return float(e["bytes_per_launch_at_L"][str(L)]) if str(L) in e.get(
        "bytes_per_launch_at_L", {}) else None


# ----------------------------------------------------------------------------- replicas
def aggregate_replicas(local_updates, local_seconds, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank's updates summed, divided by
    the slowest rank's time (max over ranks).  Returns (updates_per_s, max_seconds)."""
    if dist is None:
        return local_updates / local_seconds, local_seconds
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


# ----------------------------------------------------------------------------- oracle arm
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the architecture."""
    import platform
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        name = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return "%s (%s)" % (name or "unknown", platform.machine())


def oracle_sample(L, p, q, seconds, seed=1, threads=0):
    """Time the CPU oracle on a band of rows of the same lattice (full width L), enough MCS
    for about `seconds` of work, on all host cores (or `threads`).  Returns (updates_per_s,
    cores, description)."""
    import oracle as o
    all_cores = o.threads()
    cores = o.threads(threads) if threads else all_cores
    nrows = 16
    gx, gy = o.init_flat_band(L, 0, nrows)
    t0 = time.perf_counter()
    o.run_band(L, 0, gx, gy, seed, p, q, t0=0, n_mcs=1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-6)))
    gx, gy = o.init_flat_band(L, 0, nrows)
    t0 = time.perf_counter()
    o.run_band(L, 0, gx, gy, seed, p, q, t0=0, n_mcs=n)
    dt = time.perf_counter() - t0
    updates = (nrows - 1) * L * n
    desc = ("oracle (scalar, one site at a time) on a %d-row band of the L=%d lattice, "
            "p=%g q=%g, %d MCS = %.3g site updates in %.1f s" % (nrows, L, p, q, n, updates, dt))
    if threads:
        o.threads(all_cores)
    return updates / dt, cores, desc


def bitvec_sample(L, p, q, seconds):
    """Time the bit-vectorized CPU implementation (w = 64, all host cores; the paper's CPU
    design, Sec. II.B) on the full L x L lattice from flat, enough MCS for about `seconds`.
    Returns (updates_per_s, cores, description)."""
    import cpu_bitvec as bv
    import oracle as o
    mode = o.rng_mode(p, q)
    w = bv.flat_words(L)
    t0 = time.perf_counter()
    bv.run(w, L, 1, p, q, mode, t0=0, n_mcs=1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    bv.run(w, L, 1, p, q, mode, t0=1, n_mcs=n)
    dt = time.perf_counter() - t0
    desc = ("bit-vectorized CPU implementation (64-bit words, OpenMP over rows), full L=%d lattice "
            "from flat, p=%g q=%g, %d MCS = %.3g site updates in %.1f s" % (L, p, q, n, float(L) * L * n, dt))
    return float(L) * L * n / dt, bv.threads(), desc


def run_reference(a, rank, world):
    if rank != 0:
        return
    per_step = a.ref_seconds
    if per_step is None:
        per_step = max(2.0, min(20.0, 60.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        oracle_sample(a.L, a.p, a.q, per_step / 4)
    rates, descs, cores = [], [], 1
    t0 = time.perf_counter()
    for _ in range(a.steps):
        r, cores, d = oracle_sample(a.L, a.p, a.q, per_step)
        rates.append(r)
        descs.append(d)
    wall = time.perf_counter() - t0
    value = statistics.mean(rates)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * wall / max(1, a.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (flat initial surface, seeded Philox)", "impl": "reference",
            "config": config(a, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": descs[-1], "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def run_batch_only(a):
    """The batched ensemble alone (first --batch-count lattices of the ensemble list,
    --batch-mcs MCS), one timed run after one warm-up; prints one JSON line."""
    import torch
    import paper_1606_00310_gb300.sca as sca
    from paper_1606_00310_gb300 import build, workloads
    build.build()
    sca.load()
    ens = workloads.ensemble()[: a.batch_count]
    times = workloads.log_times(a.batch_mcs)
    stream = torch.cuda.Stream()
    with sca.Batch(ens, stream=stream) as b:
        if a.batch_engine:
            b.set_engine(a.batch_engine)
        b.run(times, want_obs=False)
        b.reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, w2 = b.run(times, want_obs=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        shape = b.shape()
        engine = b.engine()
    sites = sum(d["L"] ** 2 for d in ens)
    print(json.dumps({"metric": METRIC, "value": sites * a.batch_mcs / (ms / 1000.0), "unit": UNIT,
                      "workload": "batched ensemble, first %d lattices, %d MCS" % (len(ens), a.batch_mcs),
                      "ms": ms, "engine": engine, "cluster_shape": shape,
                      "ensemble_w2_final": w2[-1]}), flush=True)


def run_serving(n_requests, slots, rate_per_s=200.0):
    """Serving: a Poisson stream (200 requests/s) of simulations with L log-uniform in
    [256, 8192], p ~ U(0.5, 1), q = 1 - p (per-site uniforms), 512-8192 MCS, each observed at
    1, 2, 4, ..., n; submitted at their arrival times to the library's continuous-batching
    server under a 120 GB budget.  Latency = finish - arrival."""
    import paper_1606_00310_gb300.sca as sca
    from paper_1606_00310_gb300 import workloads
    reqs = workloads.request_stream(n=n_requests, rate_per_s=rate_per_s)
    with sca.Server(budget_bytes=120 * 10 ** 9, max_active=slots, max_L=8192) as srv:
        warm = srv.submit(8192, 0.7, 0.3, 10 ** 6, 64)      # first-use set-up off the clock
        srv.wait(warm)
        srv.release(warm)
        t_start = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = t_start + r["arrival_s"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(r["L"], r["p"], r["q"], r["seed"], r["mcs"]))
        infos = []
        for tk in tickets:
            rc, _, info = srv.wait(tk)
            if rc != sca.OK:
                raise RuntimeError("request %d failed: %d" % (tk, rc))
            infos.append(info)
        st = srv.stats()
    lat = np.array([i.done_s - i.submit_s for i in infos])
    queue = np.array([i.admit_s - i.submit_s for i in infos])
    span = max(i.done_s for i in infos) - min(i.submit_s for i in infos)
    updates = sum(r["L"] ** 2 * r["mcs"] for r in reqs)
    offered = updates / max(reqs[-1]["arrival_s"], 1e-9)
    return {"workload": "%d requests, Poisson %g/s, L log-uniform [256,8192] (x64), "
                        "p~U(0.5,1), q=1-p (per-site uniform), MCS U[512,8192], 120 GB budget, "
                        "%d slots" % (len(reqs), rate_per_s, slots),
            "value": updates / span, "unit": UNIT, "span_s": span,
            "offered_updates_per_s": offered,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_queue_s": float(np.percentile(queue, 50)),
            "p99_queue_s": float(np.percentile(queue, 99)),
            "completed": int(st["completed"]), "max_bytes_budget": int(st["budget_bytes"])}


def run_batched(sca, torch, stream, dev, L_single, peak):
    """Batched ensemble: 4096 lattices, L uniform in {128..2048}, half (1, 0), half (7/8, 1/8),
    4096 MCS with W^2 at 2^0..2^12, one persistent graph-captured launch per run.  Compared
    with the single-lattice rate at a similar total site count (one L=65536 lattice, 4.3 G
    sites vs 4.6 G), weighted by the same 50/50 mix of rules."""
    from paper_1606_00310_gb300 import workloads
    ens = workloads.ensemble()
    times = workloads.log_times(4096)
    sites = sum(d["L"] ** 2 for d in ens)
    with sca.Batch(ens, stream=stream) as b:
        c, t = b.tune(16)
        obs, _ = b.run(times, want_obs=True)  # warm-up (captures the graph); per-class W^2
        b.reset()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, w2 = b.run(times, want_obs=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        shape = b.shape()
        engine = b.engine()
    rate = sites * 4096 / (ms / 1000.0)
    # ensemble-averaged W^2 at the last time per class (lattice size and rule), from the
    # warm-up run (the timed run repeats it exactly: the same seeds and counters)
    per_class = {}
    for d, o in zip(ens, obs):
        per_class.setdefault("L=%d (%g,%g)" % (d["L"], d["p"], d["q"]), []).append(o[-1].w2)
    class_w2 = {k: float(np.mean(v)) for k, v in sorted(per_class.items())}
    # single-lattice rates for the same two rules at L = 65536
    single = {}
    for p, q in ((1.0, 0.0), (0.875, 0.125)):
        s = sca.Sim(L_single, seed=1, p=p, q=q, stream=stream)
        s.step(2)
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s.step(32)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        single[(p, q)] = L_single * L_single * 32 / (f0.elapsed_time(f1) / 1000.0)
        s.close()
    mix = 2.0 / (1.0 / single[(1.0, 0.0)] + 1.0 / single[(0.875, 0.125)])
    return {"workload": "4096 lattices, L uniform in {128,256,512,1024,2048}, 2048 x (1,0) + "
                        "2048 x (7/8,1/8), seeds 0-4095, 4096 MCS, W^2 at 2^0..2^12",
            "sites": sites, "value": rate, "unit": UNIT, "ms": ms,
            "single_lattice_rate_same_mix": mix,
            "single_lattice_rates": {"p=1,q=0": single[(1.0, 0.0)],
                                     "p=7/8,q=1/8": single[(0.875, 0.125)]},
            "ratio_to_single": rate / mix,
            "engine": {1: "clusters (shared memory)", 2: "streaming (register wavefront)"}.get(engine, engine),
            "cluster_shape": shape, "tuned": [c, t],
            "ensemble_w2_final": w2[-1], "class_w2_final": class_w2}


def run_ours(a, rank, world, local_rank):
    import torch
    import paper_1606_00310_gb300.sca as sca
    from paper_1606_00310_gb300 import build

    if rank == 0 or not os.path.exists(sca.LIB_PATH):
        build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.set_device(local_rank)
    sca.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    times = obs_times(a.mcs)
    L = a.L
    updates_per_step = L * L * a.mcs
    sim = sca.Sim(L, seed=1 + rank, p=a.p, q=a.q, stream=stream, kernel=a.kernel)

    def step():
        sim.reset()
        obs = sim.run(times)
        assert obs[-1].t == a.mcs and all(o.status == 0 for o in obs)
        return obs

    def sync_all():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    # measured logic-instruction rate (roofline context for the height-bit kernel), outside
    # the timed region
    try:
        logic_rate = sca.measure_logic_rate()
    except Exception:
        logic_rate = None
    try:
        mul_rate, philox_rate = sca.measure_mul_rate()
    except Exception:
        mul_rate = philox_rate = None
    for _ in range(a.warmup):
        step()
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = vis[local_rank] if len(vis) > local_rank and vis[local_rank].isdigit() else local_rank
    clocks = ClockSampler(gpu_index)
    sync_all()
    launches0 = sca.kernel_launches()
    sim.timing(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        obs = step()
    ev1.record(stream)
    sync_all()
    launches = sca.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    upd_ms, upd_launches = sim.timing_read()
    sim.timing(False)
    clk = clocks.stop()
    value, secs = aggregate_replicas(updates_per_step * a.steps, ms / 1000.0, dist, dev)
    ms = secs * 1000.0

    # roofline of the dominant (update) kernel, timed live over the same region
    kern = sim.kernel_in_use()
    peak, peak_src = peaks()
    upd_total = updates_per_step * a.steps
    upd_s = upd_ms / 1000.0
    avg_launch_s = upd_s / max(1, upd_launches)
    one_rule = {a.p, a.q} == {0.0, 1.0}
    if kern == sca.KERNEL_WAVE and one_rule:
        # ALU-bound: algorithmic logic ops over the measured launch time
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        apeak, mhz = alu_peak_tops(n_sm)
        achieved = WAVE_ALU_OPS_PER_UPDATE * upd_total / upd_s / 1e12
        state_bytes = L * L / 4.0           # canonical words: two slope bits per site
        traffic = recorded_traffic("k_wave", L)
        roof = {"bound": "alu", "achieved": achieved, "peak": apeak, "unit": "Tops/s",
                "frac": achieved / apeak, "traffic": traffic,
                "kernel": "k_wave",
                "peak_source": "derived: %d SMs x %d logic lanes/clk x %.0f MHz (max SM clock)"
                               % (n_sm, ALU_LANES_PER_SM, mhz),
                "alg_ops_per_update": WAVE_ALU_OPS_PER_UPDATE,
                "peak_measured": logic_rate / 1e12 if logic_rate else None,
                "frac_of_measured": achieved / (logic_rate / 1e12) if logic_rate else None,
                "peak_measured_source": "sca_measure_logic_rate: independent LOP3 chains on "
                                        "every SM, CUDA events",
                "one_pass_hbm_roofline_updates_per_s": peak * 1e9 / BYTES_PER_UPDATE,
                "x_one_pass_hbm_roofline": (upd_total / upd_s) / (peak * 1e9 / BYTES_PER_UPDATE),
                "avg_launch_ms": avg_launch_s * 1e3, "launches": upd_launches,
                "mcs_per_launch_avg": a.mcs * a.steps / max(1, upd_launches),
                # the canonical state (L^2/4 bytes) read and written once per launch
                "hbm_GBs_state_once_per_launch": 2 * state_bytes * upd_launches / upd_s / 1e9,
                # DRAM bytes per launch from the ncu capture over the live average launch time
                "dram_GBs_measured": traffic / avg_launch_s / 1e9 if traffic else None,
                "hbm_peak_GBs": peak,
                "update_share_of_step": upd_ms / ms if ms > 0 else None,
                "updates_per_s_kernel_only": upd_total / upd_s}
    else:
        kname = {sca.KERNEL_FUSED: "k_fused_mcs", sca.KERNEL_WAVE: "k_wave",
                 sca.KERNEL_TBLOCK: "k_tblock"}.get(kern, "k_half_step")
        # bytes: the state read and written once per launch (one sublattice per two-pass
        # launch; one MCS per fused launch; several per temporal-blocking launch)
        alg_bytes = BYTES_PER_UPDATE * (L * L // 2 if kern == sca.KERNEL_TWO_PASS else L * L)
        achieved = alg_bytes / avg_launch_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(kname, L),
                "kernel": kname, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else peak_src,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                "update_share_of_step": upd_ms / ms if ms > 0 else None,
                "updates_per_s_kernel_only": upd_total / upd_s}

    # end-to-end through the C ABI with host buffers: pinned flat words in, state + W^2 out
    e2e = None
    if not a.no_e2e:
        n_words = sca.words_count(L)
        host_in = torch.empty(n_words, dtype=torch.int32, pin_memory=True)
        host_out = torch.empty(n_words, dtype=torch.int32, pin_memory=True)
        flat = sca.Sim(L, seed=1, p=1.0, q=0.0, stream=stream)   # flat words from the library
        flat.get_state_ptr(host_in.data_ptr(), n_words)
        flat.close()
        del flat

        def e2e_step():
            sim.set_state_ptr(host_in.data_ptr(), n_words, 0)
            obs = sim.run(times)
            sim.get_state_ptr(host_out.data_ptr(), n_words)
            return obs

        # one simulation, synchronous calls: copies and updates in sequence (context)
        e2e_step()
        sync_all()
        clk_seq = ClockSampler(gpu_index)
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        sync_all()
        seq_s = time.perf_counter() - t0
        clk_seq = clk_seq.stop()
        seq_value, seq_s = aggregate_replicas(updates_per_step * a.steps, seq_s, dist, dev)

        # two simulations on two streams, asynchronous calls: step i's host copies overlap
        # step i-1's updates on the other simulation; every copy is inside the timed region.
        # The updates of step i wait for those of step i-1 (an event between the streams), so
        # the two simulations' kernels never share the SMs: each launch keeps its one full wave.
        stream2 = torch.cuda.Stream(device=dev)
        sim2 = sca.Sim(L, seed=1 + rank, p=a.p, q=a.q, stream=stream2, kernel=a.kernel)
        host_out2 = torch.empty(n_words, dtype=torch.int32, pin_memory=True)
        sims, outs, streams = [sim, sim2], [host_out, host_out2], [stream, stream2]

        def pipelined(k):
            # events on each step's stream (before the copy in, after it and the surface check,
            # when the updates start, when they end, after the copy out) and the host time the
            # run call spends waiting for that check: where a step's time goes
            pending, updated, rec = None, None, []
            for i in range(k):
                s, st_ = sims[i % 2], streams[i % 2]
                ev = {x: torch.cuda.Event(enable_timing=True) for x in "abce"}
                ev["a"].record(st_)
                s.set_state_ptr_async(host_in.data_ptr(), n_words, 0)
                ev["b"].record(st_)
                if updated is not None:
                    st_.wait_event(updated)
                ev["c"].record(st_)
                h0 = time.perf_counter()
                s.run_async(times)
                ev["host_run_ms"] = 1e3 * (time.perf_counter() - h0)
                updated = torch.cuda.Event(enable_timing=True)
                updated.record(st_)
                ev["d"] = updated
                s.get_state_ptr_async(outs[i % 2].data_ptr(), n_words)
                ev["e"].record(st_)
                if pending is not None:
                    ob = pending.wait()
                    assert ob[-1].t == a.mcs and all(o_.status == 0 for o_ in ob)
                pending = s
                rec.append(ev)
            ob = pending.wait()
            assert ob[-1].t == a.mcs and all(o_.status == 0 for o_ in ob)
            return rec

        def step_profile(rec):
            torch.cuda.synchronize(dev)
            mean = lambda v: float(sum(v) / len(v)) if v else None
            return {"copy_in_and_check_ms": mean([r["a"].elapsed_time(r["b"]) for r in rec]),
                    "run_ms": mean([r["c"].elapsed_time(r["d"]) for r in rec]),
                    "copy_out_ms": mean([r["d"].elapsed_time(r["e"]) for r in rec]),
                    "gap_between_runs_ms": mean([rec[i - 1]["d"].elapsed_time(rec[i]["c"])
                                                 for i in range(1, len(rec))]),
                    "host_run_call_ms": mean([r["host_run_ms"] for r in rec])}

        pipelined(2)
        sync_all()
        sim.timing(True)
        sim2.timing(True)
        clk_e2e = ClockSampler(gpu_index)
        t0 = time.perf_counter()
        e2e_rec = pipelined(a.steps)
        sync_all()
        e2e_s = time.perf_counter() - t0
        e2e_steps = step_profile(e2e_rec)
        clk_e2e = clk_e2e.stop()
        # the updates' own device time inside the pipelined region (CUDA events around each
        # run's update launches): the difference to ms_per_step is what the copies did not hide
        e2e_upd_ms = sim.timing_read()[0] + sim2.timing_read()[0]
        sim.timing(False)
        sim2.timing(False)
        sim2.close()
        e2e_value, e2e_s = aggregate_replicas(updates_per_step * a.steps, e2e_s, dist, dev)

        # context, outside the timed regions: this host's pinned copy rate each way (one
        # 1 GiB copy after a warm one, CUDA events on the simulation's stream)
        def copy_GBs(dst, src):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
            torch.cuda.synchronize(dev)
            return 4 * n_words / (e0.elapsed_time(e1) / 1e3) / 1e9
        dev_buf = torch.empty(n_words, dtype=torch.int32, device=dev)
        h2d_GBs, d2h_GBs = copy_GBs(dev_buf, host_in), copy_GBs(host_out, dev_buf)
        del dev_buf
        obs_bytes = len(times) * sca.OBS_RECORD_BYTES
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 4 * n_words, "d2h_bytes_per_step": 4 * n_words + obs_bytes,
               "ms_per_step": 1000.0 * e2e_s / a.steps,
               "pipelined": "two simulations on two streams: sca_set_state_async (pinned 1 GiB "
                            "in), sca_run_async (after the other simulation's updates), "
                            "sca_get_state_async (1 GiB out), sca_wait",
               "sequential_value": seq_value,
               "sequential_ms_per_step": 1000.0 * seq_s / a.steps,
               "pinned_h2d_GBs": h2d_GBs, "pinned_d2h_GBs": d2h_GBs,
               "update_ms_per_step": e2e_upd_ms / a.steps, "step_profile": e2e_steps,
               "clocks": clk_e2e, "clocks_sequential": clk_seq}

    # context: the paper's own benchmark case p = 1/2, q = 0 (random bits every update)
    extra = None
    if not a.no_extra and rank == 0 and world == 1 and (a.p, a.q) == (1.0, 0.0):
        half = sca.Sim(L, seed=1, p=0.5, q=0.0, stream=stream, kernel=a.kernel)
        half.step(4)
        torch.cuda.synchronize(dev)
        half.timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n_half = 64
        e0.record(stream)
        half.step(n_half)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        hms = e0.elapsed_time(e1)
        h_upd_ms, h_launches = half.timing_read()
        h_kern = half.kernel_in_use()
        half.close()
        del half
        rate = L * L * n_half / (hms / 1000.0)
        bound = issue_bound(P_HALF_CALLS_PER_UPDATE, P_HALF_OPS_PER_UPDATE, philox_rate, logic_rate) \
            if philox_rate and logic_rate else None
        extra = {"workload": "L=65536 p=1/2 q=0 (paper Sec. III headline case), %d MCS" % n_half,
                 "value": rate, "unit": UNIT,
                 "roofline": {"bound": "issue: Philox calls + logic ops (measured rates)",
                              "achieved": rate, "peak": bound, "unit": UNIT,
                              "frac": rate / bound if bound else None,
                              "philox_calls_per_update": P_HALF_CALLS_PER_UPDATE,
                              "logic_ops_per_update": P_HALF_OPS_PER_UPDATE,
                              "philox_calls_per_s_measured": philox_rate,
                              "logic_ops_per_s_measured": logic_rate,
                              "wide_mul_per_s_measured": mul_rate},
                 "paper_titan_black_updates_per_s": 2.29e11,
                 "ratio_to_paper": rate / 2.29e11,
                 "kernel": h_kern, "launches": h_launches,
                 # the canonical state read and written once per launch, over the launch time
                 "hbm_frac_state_once_per_launch":
                     BYTES_PER_UPDATE * L * L * h_launches / (h_upd_ms / 1000.0) / 1e9 / peak}

    # context: non-dyadic p (per-site 32-bit uniforms, the paper's arbitrary-p case and the
    # serving workload's rule) at the benchmark's size
    uni = None
    if not a.no_extra and rank == 0 and world == 1 and (a.p, a.q) == (1.0, 0.0):
        us = sca.Sim(L, seed=1, p=0.7, q=0.3, stream=stream)
        us.step(2)
        torch.cuda.synchronize(dev)
        n_u = 8
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        us.step(n_u)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        u_rate = L * L * n_u / (e0.elapsed_time(e1) / 1000.0)
        u_kern = us.kernel_in_use()
        us.close()
        del us
        bound = issue_bound(UNIFORM_CALLS_PER_UPDATE, UNIFORM_OPS_PER_UPDATE, philox_rate, logic_rate) \
            if philox_rate and logic_rate else None
        uni = {"workload": "L=%d p=0.7 q=0.3 (per-site 32-bit uniforms), %d MCS" % (L, n_u),
               "value": u_rate, "unit": UNIT, "kernel": u_kern,
               "roofline": {"bound": "issue: Philox calls + logic ops (measured rates)",
                            "achieved": u_rate, "peak": bound, "unit": UNIT,
                            "frac": u_rate / bound if bound else None,
                            "philox_calls_per_update": UNIFORM_CALLS_PER_UPDATE,
                            "logic_ops_per_update": UNIFORM_OPS_PER_UPDATE,
                            "philox_calls_per_s_measured": philox_rate,
                            "logic_ops_per_s_measured": logic_rate,
                            "philox_only_bound": UNIFORM_CALLS_PER_UPDATE ** -1 * philox_rate
                            if philox_rate else None}}

    # context: the same rule and kernel from a rough surface (a flat surface is a fixed point of
    # p = 1; the kernel's work does not depend on the state, and this measures it)
    rough = None
    if not a.no_extra and rank == 0 and world == 1 and (a.p, a.q) == (1.0, 0.0):
        prep = sca.Sim(L, seed=7, p=0.625, q=0.375, stream=stream, kernel=sca.KERNEL_TWO_PASS)
        prep.step(3)
        words = prep.get_state()
        prep.close()
        del prep
        rs = sca.Sim(L, seed=1, p=1.0, q=0.0, stream=stream, kernel=a.kernel)
        rs.set_state(words, t=0)
        del words
        rs.step(16)
        torch.cuda.synchronize(dev)
        n_rough = 256
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs.step(n_rough)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        rms = e0.elapsed_time(e1)
        w2 = rs.observe().w2
        r_kern = rs.kernel_in_use()
        rs.close()
        del rs
        rough = {"workload": "L=%d p=1 q=0 from a rough surface (3 MCS of p=5/8 q=3/8), %d MCS of "
                             "updates only" % (L, n_rough),
                 "value": L * L * n_rough / (rms / 1000.0), "unit": UNIT, "kernel": r_kern,
                 "w2_after": w2}

    # context: the wide system L = 2^17 (4 GiB of packed slopes per buffer), the paper's case
    # p = 1/2 and the headline rule, updates only; the paper reports its wide system within 5 %
    # of L = 2^16
    wide = None
    if not a.no_extra and rank == 0 and world == 1 and (a.L, a.p, a.q) == (65536, 1.0, 0.0):
        wide = {"workload": "L=131072 flat start, updates only (CUDA events)", "unit": UNIT}
        for key, (wp, wq, n_w) in (("p_half", (0.5, 0.0, 32)), ("p1", (1.0, 0.0, 128))):
            ws = sca.Sim(131072, seed=1, p=wp, q=wq, stream=stream, kernel=a.kernel)
            ws.step(16)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ws.step(n_w)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            wide[key] = 131072.0 * 131072.0 * n_w / (e0.elapsed_time(e1) / 1000.0)
            wide[key + "_kernel"] = ws.kernel_in_use()
            ws.close()
            del ws
        if extra:
            wide["p_half_ratio_to_L65536"] = wide["p_half"] / extra["value"]

    batched = None
    if not a.no_batch and rank == 0 and world == 1 and (a.L, a.p, a.q) == (65536, 1.0, 0.0):
        batched = run_batched(sca, torch, stream, dev, L, peak)
    serving = serving_light = None
    if not a.no_serve and rank == 0 and world == 1 and (a.L, a.p, a.q) == (65536, 1.0, 0.0):
        serving = run_serving(a.serve_requests, a.serve_slots)
        # the same request mix at about three quarters of the sustained capacity (15/s instead
        # of 200/s): latency without the queue of the oversubscribed stream
        serving_light = run_serving(150, a.serve_slots, rate_per_s=15.0)

    cpu = cpu_bv = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        r, cores, desc = oracle_sample(L, a.p, a.q, a.cpu_seconds)
        r1, _, desc1 = oracle_sample(L, a.p, a.q, max(1.0, a.cpu_seconds / 3), threads=1)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "cpu_model": cpu_model(), "value_1_core": r1, "sample_1_core": desc1}
        # the like-for-like CPU baseline: the same bit-vectorized update on 64-bit words over
        # all cores (the paper's CPU implementation), the workload's rule and the paper's p = 1/2
        bv_rate, bv_cores, bv_desc = bitvec_sample(L, a.p, a.q, a.cpu_seconds)
        bv_half, _, bv_half_desc = bitvec_sample(L, 0.5, 0.0, a.cpu_seconds)
        cpu_bv = {"value": bv_rate, "unit": UNIT, "cores": bv_cores, "cpu_model": cpu_model(),
                  "kind": "bit-vectorized w=64 (paper Sec. II.B CPU implementation)",
                  "sample": bv_desc, "gpu_over_cpu": value / bv_rate,
                  "p_half": bv_half, "sample_p_half": bv_half_desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic (flat initial surface, seeded Philox)",
                "config": config(a, world), "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "w2_final": obs[-1].w2}
        if cpu_bv:
            if extra:
                cpu_bv["gpu_over_cpu_p_half"] = extra["value"] / cpu_bv["p_half"]
            line["cpu_baseline_bitvec"] = cpu_bv
        if extra:
            line["context_p_half"] = extra
        if uni:
            line["context_uniform"] = uni
        if rough:
            line["context_rough_p1"] = rough
        if wide:
            line["context_wide_L131072"] = wide
        if batched:
            line["batched"] = batched
        if serving:
            line["serving"] = serving
        if serving_light:
            line["serving_below_capacity"] = serving_light
        print(json.dumps(line), flush=True)
    sim.close()


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.only == "batch":
        run_batch_only(a)
        return
    if a.only == "serve":
        from paper_1606_00310_gb300 import build
        build.build()
        line = run_serving(a.serve_requests, a.serve_slots)
        line["metric"] = METRIC
        print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
