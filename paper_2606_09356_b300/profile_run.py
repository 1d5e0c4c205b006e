"""Run a workload for a fixed number of Monte Carlo steps (a driver for
profilers such as ncu; prints nothing but a one-line summary).

    python -m paper_2606_09356_b300.profile_run --workload config1 --steps 20 [--move smart]
"""
import argparse
import time

from . import build as _build
from . import soma, workloads


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="config1")
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--graph-steps", type=int, default=0)
    p.add_argument("--sort-interval", type=int, default=-1)
    p.add_argument("--hist-mode", type=int, default=0)
    p.add_argument("--ctas-per-sm", type=int, default=0)
    p.add_argument("--move", default="uniform", choices=["uniform", "smart"])
    a = p.parse_args()
    _build.build()
    move = soma.SOMA_MOVE_SMART if a.move == "smart" else soma.SOMA_MOVE_UNIFORM
    s = soma.System(**{**workloads.system_kwargs(a.workload), "move": move})
    with soma.Handle(s, graph_steps=a.graph_steps, sort_interval=a.sort_interval, hist_mode=a.hist_mode,
                     ctas_per_sm=a.ctas_per_sm) as h:
        t = time.perf_counter()
        h.mc_steps(a.steps)
        h.sync()
        dt = time.perf_counter() - t
        print(f"{a.workload}: {a.steps} steps, {a.steps * s.n_beads / dt:.3e} moves/s (wall, incl. launch)")


if __name__ == "__main__":
    main()
