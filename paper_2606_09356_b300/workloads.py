"""Synthetic workloads shaped like the paper's particle runs (no arithmetic of
the method lives here; both the CUDA path and the oracle take these as input).

The paper's own particle workload (a membrane-forming melt on a grid refined
to R_e/10, Sec. 4) needs continuum-supplied fields and is not available; these
AB diblock melts stand in for it at the same kind of SCMF densities.

* ``melt_512x32``  512 chains x 32, f_A = 0.5, box 4^3, grid 16^3, chiN 20,
  kappaN 50: the small case the oracle runs in full.
* ``melt_131072x32``  131,072 x 32 (4.19 M beads), box 16^3, grid 128^3, chiN 30:
  the single-GPU throughput workload.
* ``melt_1048576x64``  1,048,576 x 64, f_A = 0.3 (n_A = 19), box 32^3, grid 256^3,
  chiN 25 (67.1 M beads).
* ``batch64``  64 independent systems of uneven size (``batch64.json``,
  written by ``make_batch64``): N in {16, 32, 64}, chains log-uniform in
  [2048, 65536], cubic boxes 4-12 R_e rounded to 1/8 with grid 8L, chiN
  uniform in [10, 40], kappaN 50, f_A uniform in [0.3, 0.5].
"""
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
BATCH64_JSON = os.path.join(_HERE, "batch64.json")

WORKLOADS = {
    "melt_512x32": dict(n_poly=512, N=32, n_A=16, box=(4.0, 4.0, 4.0), grid=(16, 16, 16), chiN=20.0, kappaN=50.0,
                    seed=1, steps=100),
    "melt_131072x32": dict(n_poly=131072, N=32, n_A=16, box=(16.0, 16.0, 16.0), grid=(128, 128, 128), chiN=30.0,
                    kappaN=50.0, seed=1, steps=1000),
    "melt_1048576x64": dict(n_poly=1048576, N=64, n_A=19, box=(32.0, 32.0, 32.0), grid=(256, 256, 256), chiN=25.0,
                    kappaN=50.0, seed=1, steps=500),
}


def system_kwargs(name, **override):
    """Keyword arguments of ``soma.System`` / ``oracle.Oracle`` for a config."""
    c = dict(WORKLOADS[name])
    c.pop("steps")
    c.update(override)
    return c


def make_batch64(seed=1, n=64):
    """Draw the 64-system batch with numpy's MT19937 seeded by ``seed``."""
    rng = np.random.Generator(np.random.MT19937(seed))
    systems = []
    for s in range(n):
        N = int(rng.choice([16, 32, 64]))
        n_poly = int(round(np.exp(rng.uniform(np.log(2048), np.log(65536)))))
        L = round(float(rng.uniform(4.0, 12.0)) * 8) / 8.0
        g = int(round(8 * L))
        fA = float(rng.uniform(0.3, 0.5))
        systems.append(dict(n_poly=n_poly, N=N, n_A=int(np.floor(fA * N + 0.5)), box=(L, L, L), grid=(g, g, g),
                            chiN=float(rng.uniform(10.0, 40.0)), kappaN=50.0, seed=1, system_id=s, f_A=fA))
    return systems


def batch64():
    """The committed 64-system batch (list of dicts)."""
    with open(BATCH64_JSON) as f:
        return json.load(f)["systems"]


if __name__ == "__main__":
    with open(BATCH64_JSON, "w") as f:
        json.dump({"generator": "make_batch64(seed=1)", "steps": 1000, "systems": make_batch64()}, f, indent=1)
