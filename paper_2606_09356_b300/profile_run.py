"""Run a workload for a fixed number of Monte Carlo steps (a driver for
profilers such as ncu; prints nothing but a one-line summary).

    python -m paper_2606_09356_b300.profile_run --workload melt_131072x32 --steps 20 [--move smart]
        [--walls] [--conversion] [--move-warps 12]

--workload batch64 steps the 64-system batch in one handle (the batch
kernel; uniform moves, periodic z).

--conversion switches on boundary-zone conversion (zones 2 R_e wide at the
bottom and top, per-step rates 0.05, 0.02, 0.03, 0.04, converted molecules
with half the A block); it is meant with --walls.
"""
import argparse
import time

from . import build as _build
from . import soma, workloads


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="melt_131072x32")
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--graph-steps", type=int, default=0)
    p.add_argument("--sort-interval", type=int, default=-1)
    p.add_argument("--hist-mode", type=int, default=0)
    p.add_argument("--ctas-per-sm", type=int, default=0)
    p.add_argument("--move", default="uniform", choices=["uniform", "smart"])
    p.add_argument("--walls", action="store_true")
    p.add_argument("--conversion", action="store_true")
    p.add_argument("--move-warps", type=int, default=0, help="consumer warps per CTA: 8, 12 or 24 (0: 8)")
    a = p.parse_args()
    _build.build()
    move = soma.SOMA_MOVE_SMART if a.move == "smart" else soma.SOMA_MOVE_UNIFORM
    if a.workload == "batch64":
        systems = [soma.System(**{k: v for k, v in d.items() if k != "f_A"}) for d in workloads.batch64()]
        n_beads = sum(x.n_beads for x in systems)
    else:
        kw = workloads.system_kwargs(a.workload)
        systems = soma.System(**{**kw, "move": move, "wall_z": 1 if a.walls else 0})
        n_beads = systems.n_beads
    with soma.Handle(systems, graph_steps=a.graph_steps, sort_interval=a.sort_interval, hist_mode=a.hist_mode,
                     ctas_per_sm=a.ctas_per_sm, move_warps=a.move_warps) as h:
        if a.conversion and a.workload != "batch64":
            h.set_conversion(kw["n_A"] // 2, 2.0, 2.0, (0.05, 0.02, 0.03, 0.04))
        t = time.perf_counter()
        h.mc_steps(a.steps)
        h.sync()
        dt = time.perf_counter() - t
        print(f"{a.workload}: {a.steps} steps, {a.steps * n_beads / dt:.3e} moves/s (wall, incl. launch)")


if __name__ == "__main__":
    main()
