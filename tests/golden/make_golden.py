"""Write tests/golden/oracle_small.json from the CPU oracle alone.

The paper prints no trajectories or roughness values, so these fixtures are regression pins of
the oracle itself (they change only with a change to the oracle's arithmetic, which must then
name the paper passage that justifies it) and expected values for small GPU parity cases.
Each case: lattice size L, seed, (p, q), mode (1 = dyadic, 2 = per-site uniform), observation
times; stored: exact S1, S2, num at each time and the sha256 of the final canonical words.

The mid-size workload (L = 4096, 10^4 MCS, 40 log-spaced observation times, p = 3/4, q = 1/4,
seeds 1-4) takes the oracle about 25 minutes per seed on 8 host cores; it is written to its own
file, oracle_mid_size.json, one case at a time, so the GPU tests compare the full runs without
running the oracle at test time.

Run:  python tests/golden/make_golden.py            (small cases)
      python tests/golden/make_golden.py --mid-size  (the L = 4096 workload)
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o  # noqa: E402
from paper_1606_00310_gb300 import workloads  # noqa: E402  (seeded inputs only)

CASES = [
    # L=64, p=1, q=0, seed 1, 1000 MCS, roughness at 1, 2, 4, ..., 512 (the small lattice case)
    dict(name="L64_p1_q0_s1", L=64, seed=1, p=1.0, q=0.0, mode=1,
         times=[2 ** k for k in range(10)] + [1000]),
    dict(name="L64_p3/4_q1/4_s1", L=64, seed=1, p=0.75, q=0.25, mode=1,
         times=[1, 2, 4, 8, 16, 32, 64, 128, 200]),
    dict(name="L64_p3/4_q1/4_s4", L=64, seed=4, p=0.75, q=0.25, mode=1,
         times=[1, 2, 4, 8, 16, 32, 64, 128, 200]),
    dict(name="L128_p7/8_q1/8_s0", L=128, seed=0, p=0.875, q=0.125, mode=1,
         times=[1, 2, 4, 8, 16, 32, 64]),
    dict(name="L128_p0.7_q0.3_uniform_s5", L=128, seed=5, p=0.7, q=0.3, mode=2,
         times=[1, 2, 4, 8, 16, 32, 64, 100]),
    dict(name="L192_p1/2_q0_s2", L=192, seed=2, p=0.5, q=0.0, mode=1,
         times=[1, 2, 4, 8, 16, 32, 64]),
    dict(name="L320_p0.95_q0_uniform_s3", L=320, seed=3, p=0.95, q=0.0, mode=2,
         times=[1, 2, 4, 8, 16, 32]),
]


# L=4096, 16.8M sites, flat start, 10^4 MCS, exact W^2 at 40 log-spaced times, dyadic
# (3/4, 1/4), seeds 1-4 (the (1, 0) runs of this workload follow the p = 1 closed form)
MID_SIZE_CASES = [
    dict(name="L4096_p3/4_q1/4_s%d" % s, L=4096, seed=s, p=0.75, q=0.25, mode=1,
         times=workloads.log_spaced_times(10_000, 40))
    for s in (1, 4, 2, 3)
]


def run_case(c):
    bx, by = o.init_flat(c["L"])
    obs = []
    t = 0
    for tt in c["times"]:
        o.run(bx, by, c["seed"], c["p"], c["q"], mode=c["mode"], t0=t, n_mcs=tt - t)
        t = tt
        r = o.observe(bx, by)
        obs.append({"t": tt, "S1": r["S1"], "S2": str(r["S2"]), "num": str(r["num"])})
    words = o.pack(bx, by)
    return {**c, "obs": obs, "final_words_sha256": hashlib.sha256(words.tobytes()).hexdigest()}


SOURCE = "CPU oracle (oracle/sca_oracle.c); paper arXiv 1606.00310 Sec. I.A, II"


def write(name, cases):
    tmp = os.path.join(HERE, name + ".tmp")
    with open(tmp, "w") as f:
        json.dump({"source": SOURCE, "cases": cases}, f, indent=1)
    os.replace(tmp, os.path.join(HERE, name))


def main():
    if "--mid-size" in sys.argv:
        done = []
        for c in MID_SIZE_CASES:
            done.append(run_case(c))
            write("oracle_mid_size.json", done)
        return
    write("oracle_small.json", [run_case(c) for c in CASES])


if __name__ == "__main__":
    main()
