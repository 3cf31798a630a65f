"""Seeded synthetic workloads (inputs only; none of the model's arithmetic lives here).

Both the GPU path and the CPU oracle take their inputs from these generators, so a test can
run one workload on both sides.  Every list is a pure function of its seed.
"""
import numpy as np


def log_times(t_max: int):
    """MCS 1, 2, 4, ... up to t_max (t_max appended if it is not a power of two)."""
    out, t = [], 1
    while t < t_max:
        out.append(t)
        t *= 2
    out.append(t_max)
    return out


def log_spaced_times(t_max: int = 10_000, n: int = 40):
    """n distinct, roughly log-spaced times from 1 to t_max: t_i = max(t_{i-1}+1,
    round(t_max^(i/(n-1))))."""
    out = [1]
    for i in range(1, n):
        out.append(max(out[-1] + 1, int(round(t_max ** (i / (n - 1))))))
    return out


def ensemble(count: int = 4096, sizes=(128, 256, 512, 1024, 2048), seed: int = 0):
    """The batched ensemble: `count` lattices, L drawn uniformly from `sizes`, exactly half with
    (p, q) = (1, 0) and half with (7/8, 1/8) (assignment drawn by the same generator), lattice
    i seeded with i.  Returns a list of dicts (L, p, q, seed)."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(np.asarray(sizes), size=count)
    kind = np.zeros(count, dtype=np.int64)
    kind[rng.permutation(count)[: count // 2]] = 1
    out = []
    for i in range(count):
        p, q = (0.875, 0.125) if kind[i] else (1.0, 0.0)
        out.append({"L": int(Ls[i]), "p": p, "q": q, "seed": i})
    return out


def request_stream(n: int = 2000, rate_per_s: float = 200.0, seed: int = 0, l_min: int = 256,
                   l_max: int = 8192, mcs_min: int = 512, mcs_max: int = 8192):
    """Serving workload: Poisson arrivals (mean `rate_per_s`), L log-uniform in [l_min, l_max]
    rounded to a multiple of 64, p ~ U(0.5, 1), q = 1 - p (non-dyadic), MCS uniform integer in
    [mcs_min, mcs_max], seed = request index.  Returns a list of dicts sorted by arrival time."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    arrival = np.cumsum(gaps) - gaps[0]
    u = rng.uniform(np.log2(l_min), np.log2(l_max), size=n)
    Ls = np.clip(64 * np.round(2.0 ** u / 64), l_min, l_max).astype(np.int64)
    p = rng.uniform(0.5, 1.0, size=n)
    mcs = rng.integers(mcs_min, mcs_max + 1, size=n)
    return [{"id": i, "arrival_s": float(arrival[i]), "L": int(Ls[i]), "p": float(p[i]),
             "q": float(1.0 - p[i]), "mcs": int(mcs[i]), "seed": i} for i in range(n)]
