"""Precision study: the FP32 + image form against the FP64-position form.

    python -m paper_2606_09356_b300.precision_study --steps 100000 --seeds 8

For each seed the melt_131072x32 system (131,072 AB diblocks, N = 32, box 16^3,
grid 128^3, chiN 30, kappaN 50) runs in both forms from its own GPU initial
configuration.  After a burn-in, <R_e^2>, <R_g^2>, the acceptance rate, the
non-bonded energy per chain and the composition structure factor at the
lowest q shells are averaged over samples taken every --every steps (FP64
reductions on the GPU).  The two forms follow the same Philox streams, so
they start on the same trajectory and separate only through last-bit
differences; their statistics must agree within the seed-to-seed spread.
Prints one JSON document.
"""
import argparse
import json
import time

import numpy as np

from . import build as _build
from . import soma, workloads


def shells(max_m2=4):
    m = [(x, y, z) for x in range(-2, 3) for y in range(-2, 3) for z in range(-2, 3)
         if 0 < x * x + y * y + z * z <= max_m2]
    m = np.array(m, np.int32)
    return m, (m ** 2).sum(1)


def run(precision, seed, steps, burn, every, m, m2):
    s = soma.System(**{**workloads.system_kwargs("melt_131072x32"), "seed": seed})
    with soma.Handle(s, precision=precision) as h:
        h.mc_steps(burn)
        h.sync()
        a0 = h.accepted()
        t0 = time.perf_counter()
        rows = []
        for _ in range(steps // every):
            h.mc_steps(every)
            o = h.observables()
            S = h.structure_factor(m)
            rows.append([o["Re2"], o["Rg2"], o["Enb"] / s.n_poly] +
                        [float(S[m2 == k].mean()) for k in sorted(set(m2.tolist()))])
        dt = time.perf_counter() - t0
        acc = (h.accepted() - a0) / (s.n_beads * (steps // every) * every)
    r = np.array(rows).mean(axis=0)
    return np.concatenate([[acc], r]), dt


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=100000)
    p.add_argument("--burn", type=int, default=2000)
    p.add_argument("--every", type=int, default=1000)
    p.add_argument("--seeds", type=int, default=8)
    a = p.parse_args()
    _build.build()
    m, m2 = shells()
    names = ["acc", "Re2", "Rg2", "Enb_per_chain"] + [f"S(|m|^2={k})" for k in sorted(set(m2.tolist()))]
    out = {"workload": "melt_131072x32", "steps": a.steps, "burn": a.burn, "every": a.every, "seeds": a.seeds,
           "observables": {}}
    res = {0: [], 1: []}
    secs = {0: 0.0, 1: 0.0}
    for seed in range(1, a.seeds + 1):
        for prec in (soma.SOMA_PREC_FP32, soma.SOMA_PREC_FP64):
            r, dt = run(prec, seed, a.steps, a.burn, a.every, m, m2)
            res[prec].append(r)
            secs[prec] += dt
    f32, f64 = np.array(res[0]), np.array(res[1])
    n = len(f32)
    for j, name in enumerate(names):
        m32, m64 = f32[:, j].mean(), f64[:, j].mean()
        se32 = f32[:, j].std(ddof=1) / np.sqrt(n) if n > 1 else float("nan")
        se64 = f64[:, j].std(ddof=1) / np.sqrt(n) if n > 1 else float("nan")
        se = float(np.hypot(se32, se64))
        out["observables"][name] = {"fp32": m32, "fp32_se": se32, "fp64": m64, "fp64_se": se64,
                                    "difference": m32 - m64, "difference_in_se": (m32 - m64) / se if se else None}
    out["gpu_seconds_sampling"] = {"fp32": secs[0], "fp64": secs[1]}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
