"""The oracle still reproduces its committed small-case fixtures (CPU only).

The fixtures were written by tests/golden/make_golden.py from the oracle alone; the p = 1 case
is also the closed form (slopes return to the flat pattern after every MCS, W^2 = 1/4).
"""
import hashlib
import json
import os

import pytest

import oracle as o

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))


@pytest.mark.parametrize("case", GOLDEN["cases"], ids=[c["name"] for c in GOLDEN["cases"]])
def test_oracle_reproduces_golden(case):
    bx, by = o.init_flat(case["L"])
    t = 0
    for ob in case["obs"]:
        o.run(bx, by, case["seed"], case["p"], case["q"], mode=case["mode"], t0=t,
              n_mcs=ob["t"] - t)
        t = ob["t"]
        r = o.observe(bx, by)
        assert (r["S1"], str(r["S2"]), str(r["num"])) == (ob["S1"], ob["S2"], ob["num"])
    assert hashlib.sha256(o.pack(bx, by).tobytes()).hexdigest() == case["final_words_sha256"]


def test_p1_golden_is_the_closed_form():
    case = next(c for c in GOLDEN["cases"] if c["name"] == "L64_p1_q0_s1")
    N = case["L"] ** 2
    assert all(int(ob["num"]) * 4 == N * N for ob in case["obs"])
    bx, by = o.init_flat(case["L"])
    assert hashlib.sha256(o.pack(bx, by).tobytes()).hexdigest() == case["final_words_sha256"]
