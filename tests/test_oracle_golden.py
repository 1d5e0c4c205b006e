"""The oracle against its own stored outputs (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): Philox words bit for
bit, accept counts exactly, positions to 1e-9, counts exactly.  CPU only."""
import json
import os

import numpy as np

from oracle import Oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


def test_oracle_matches_stored_outputs():
    data = json.load(open(GOLDEN))
    p = data["philox4x32_10"]
    out = Oracle.philox(np.array(p["ctr"], np.uint32), np.array(p["key"], np.uint32))
    assert out.tolist() == p["out"]
    for case in data["cases"]:
        o = Oracle(**{k: (tuple(v) if isinstance(v, list) else v) for k, v in case["params"].items()})
        pos = o.init()
        res = o.run(pos, 0, case["steps"], n_threads=1, acc_trace=True)
        assert [int(a) for a in res["acc"]] == case["accepted_per_step"]
        assert np.abs(pos - np.array(case["positions"])).max() <= 1e-9
        assert o.density(pos).tolist() == case["counts"]
