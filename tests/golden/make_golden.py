"""Writes tests/golden/oracle_regression.json: outputs of the oracle alone
(no CUDA path) on small fixed inputs, so that an unintended change to the
oracle's arithmetic shows up as a test failure.  The paper prints no worked
example of the step, so these values are the oracle's own; what pins the
oracle to the paper and the mathematics is tests/pins.py.  Regenerate only
together with a deliberate, justified change of the oracle:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import Oracle  # noqa: E402

CASES = [
    dict(n_poly=16, N=8, n_A=3, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=20.0, kappaN=50.0, seed=3),
    dict(n_poly=12, N=6, n_A=2, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=20.0, kappaN=50.0, seed=4, move=1),
    dict(n_poly=12, N=6, n_A=6, box=(2.0, 2.0, 1.5), grid=(4, 4, 3), chiN=0.0, kappaN=30.0, seed=5, wall_z=1),
]
STEPS = 3


def run_case(kw):
    o = Oracle(**kw)
    pos = o.init()
    res = o.run(pos, 0, STEPS, n_threads=1, acc_trace=True)
    counts = o.density(pos)
    return {"params": kw, "steps": STEPS, "accepted_per_step": [int(a) for a in res["acc"]],
            "positions": np.round(pos, 12).tolist(), "counts": counts.tolist()}


def philox_vectors():
    ctr = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]],
                   np.uint32)
    key = np.array([[0, 0], [5, 6], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]], np.uint32)
    out = Oracle.philox(ctr, key)
    return {"ctr": ctr.tolist(), "key": key.tolist(), "out": out.tolist()}


def main():
    data = {"philox4x32_10": philox_vectors(), "cases": [run_case(kw) for kw in CASES]}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(data, f)
    print("wrote", os.path.join(HERE, "oracle_regression.json"))


if __name__ == "__main__":
    main()
