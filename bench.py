"""Throughput benchmark of the SCMF Monte Carlo step (bead moves per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload melt_131072x32]
                    [--impl reference] [--no-batched] [--no-e2e] [--no-cpu]
                    [--no-steady] [--no-smart] [--no-energy]

One JSON line on rank 0.  A step is one whole Monte Carlo step of every bead
(one move kernel: moves against the fields of the previous step's counts,
fused histogram, clearing of the next count buffer; plus the periodic chain
reorder when it falls due).  Inputs are resident in HBM; between timed steps
a 256 MiB buffer (twice the L2) is written so every step starts from a cold
L2; each step is bracketed by CUDA events on the library's stream and the
move and field kernels by the library's own per-kernel events.  The steps
are queued while a spin kernel holds the stream, so the event windows hold
GPU work only (no host launch latency).

Beside the headline the line carries: the move kernel's roofline fraction
(with the DRAM traffic of the committed ncu summary when it was taken from
the current kernel source), the CPU oracle on a bounded sample, the end to
end rate through the C ABI with host buffers, CUDA-graph steady state,
energy per step from NVML, the smart-move, umbrella and walls with
boundary-zone conversion variants of the same workload, and the 64-system
batch against its systems run one by one.

``--impl reference`` times the plain FP64 CPU oracle on the same workload
shape (a bounded sample of it) on the host cores instead.

With N > 1 (torchrun), every rank runs its own replica of the workload on
its own GPU (independent systems, no data-path collective): weak scaling.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bead MC moves/s on 1xB300 and % of HBM roofline; batched vs plain speedup"
UNIT = "moves/s"
FLUSH_BYTES = 256 << 20
SECOND_WORKLOAD = "melt_1048576x64"  # the other full-size melt the roofline target names


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("soma_move.cu", "soma_device.cuh", "soma_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2606_09356_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_value(workload, variant, key):
    """A per-launch figure of the move kernel (`key: value` line) from the
    committed ncu summary, if that summary was taken from the current kernel
    source."""
    path = os.path.join(ROOT, "profiles", f"k_move{variant}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != _kernel_source_hash():
        return None
    return float(t.group(1))


def _profiled_traffic(workload, variant=""):
    """DRAM bytes per launch of the move kernel (ncu dram__bytes_read.sum +
    dram__bytes_write.sum)."""
    return _profiled_value(workload, variant, "dram_bytes_per_launch")


def issue_roofline(workload, variant, move_ms, sm_max_mhz):
    """The move kernel against the SM issue ceiling: its warp instructions per
    launch (ncu smsp__inst_executed.sum of the same kernel source) over its
    average launch time, against 4 warp instructions per cycle per SM (one
    per scheduler) at the SM count and the maximum SM clock."""
    inst = _profiled_value(workload, variant, "warp_instructions_per_launch")
    if inst is None or not move_ms:
        return None
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz or 2032.0
    peak = n_sm * 4 * mhz * 1e6 / 1e9
    achieved = inst / (move_ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp instructions/s",
            "frac": achieved / peak, "warp_instructions": inst, "floor_ms": inst / (peak * 1e9) * 1e3,
            "peak_kind": f"{n_sm} SMs x 4 schedulers x {mhz:.0f} MHz"
                         + ("" if sm_max_mhz else " (nominal maximum clock)")}


class _Nvml:
    """Minimal ctypes binding of the NVML calls used for clock sampling
    (libnvidia-ml ships with the driver; the pynvml module may be absent)."""

    def __init__(self, index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")
        reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = reasons or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sm_clock(self, max_clock=False):
        v = self.ct.c_uint()
        fn = self.lib.nvmlDeviceGetMaxClockInfo if max_clock else self.lib.nvmlDeviceGetClockInfo
        if fn(self.h, self.ct.c_int(1), self.ct.byref(v)) != 0:  # NVML_CLOCK_SM = 1
            raise RuntimeError("clock query failed")
        return v.value

    def energy_mj(self):
        """Total energy the GPU has consumed since the driver loaded, in mJ."""
        v = self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.h, self.ct.byref(v)) != 0:
            raise RuntimeError("energy query failed")
        return v.value

    def reasons(self):
        v = self.ct.c_ulonglong()
        if self.reasons_fn(self.h, self.ct.byref(v)) != 0:
            raise RuntimeError("reason query failed")
        return v.value


class Clocks:
    """SM clock and clock-event (throttle) reasons sampled during the timed
    region: NVML polled every millisecond from a thread (the timed region of
    a default run lasts a few milliseconds)."""
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, index):
        self.index = index
        self.sm, self.reasons, self.max_mhz, self.error = [], set(), None, None

    def _poll(self):
        while not self._stop.is_set():
            try:
                self.sm.append(self._nvml.sm_clock())
                bits = self._nvml.reasons()
                for name, bit in self.REASONS:
                    if bits & bit:
                        self.reasons.add(name)
            except Exception as e:  # keep sampling; report the last error
                self.error = repr(e)
            self._stop.wait(0.001)

    def __enter__(self):
        import threading
        self._stop = threading.Event()
        self._thread = None
        try:
            self._nvml = _Nvml(self.index)
            self.max_mhz = self._nvml.sm_clock(max_clock=True)
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
        except Exception as e:
            self.error = repr(e)
        return self

    def __exit__(self, *a):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(2)

    def summary(self):
        out = {"sm_mhz": statistics.median(self.sm) if self.sm else None, "sm_max_mhz": self.max_mhz,
               "reasons": sorted(self.reasons), "samples": len(self.sm), "source": "NVML, 1 ms polling"}
        if self.error and not self.sm:
            out["error"] = self.error
        return out


def hold_stream(torch, stream, steps, per_step_s=1.5e-3, clock_hz=2.0e9):
    """Keep the stream busy (a bounded spin kernel, outside every timed
    window) while the host queues the timed steps, so the per-step CUDA-event
    windows measure the GPU's work and not the host's launch latency."""
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(min(2.0, (steps + 2) * per_step_s) * clock_hz))


def warm_up(torch, stream, flush, step, n):
    """n untimed iterations shaped exactly like the timed ones (L2 flush,
    event records, step), so that every first-use cost of the process (the
    flush kernel's first launch, the first timing events) is paid before
    timing starts."""
    for i in range(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(float(-1 - i))
            a.record(stream)
        step()
        with torch.cuda.stream(stream):
            b.record(stream)
    torch.cuda.synchronize()


def rank_system_kwargs(workload, rank):
    """Each rank runs its own replica of the workload: same shape, its own
    random stream (system_id = rank), no data exchanged between ranks."""
    from paper_2606_09356_b300 import workloads
    return {**workloads.system_kwargs(workload), "system_id": rank}


def aggregate(total_ms, moves_local, pg=None, device=None):
    """Whole-job throughput: moves of all ranks over the slowest rank's time.
    Returns (max_ms, total_moves, moves_per_s)."""
    if pg is None:
        return total_ms, moves_local, moves_local / (total_ms * 1e-3)
    import torch
    t = torch.tensor([float(total_ms), float(moves_local)], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    pg.all_reduce(mx, op=pg.ReduceOp.MAX)
    tot = t[1:].clone()
    pg.all_reduce(tot, op=pg.ReduceOp.SUM)
    max_ms, moves = float(mx.item()), float(tot.item())
    return max_ms, moves, moves / (max_ms * 1e-3)


def workload_desc(name, c):
    return (f"{name}: {c['n_poly']} AB diblocks N={c['N']} n_A={c['n_A']}, box {c['box'][0]:g}^3 R_e, "
            f"grid {c['grid'][0]}^3, chiN={c['chiN']:g}, kappaN={c['kappaN']:g}, FP32 positions + int16 image")


def algorithmic_bytes(n_b, n_c):
    """Bytes the method must move per step: positions read and written
    (24 B per bead-move) and per cell the counts written and read and the
    fields written and read (32 B)."""
    return 24 * n_b + 32 * n_c


def move_kernel_bytes(n_b, n_c):
    """Algorithmic bytes of one move-kernel launch.  The kernel performs the
    whole step (moves against the fields of the previous counts, re-binning,
    clearing of the next count buffer), so its share is the whole step's
    24 B per bead + 32 B per cell."""
    return algorithmic_bytes(n_b, n_c)


# ---------------------------------------------------------------------------
def cpu_baseline(name, budget_s=12.0, steps_cap=None):
    """The oracle as it stands, on the host cores, on a bounded sample of
    about budget_s seconds: the workload's system itself for as many steps as
    fit, or, where three of its steps take longer, a system of its shape (same
    Delta, density, N, chiN, kappaN) with the box shrunk to fit."""
    from oracle import Oracle
    from paper_2606_09356_b300 import workloads
    c = workloads.system_kwargs(name)
    cores = os.cpu_count() or 1
    # probe: rate on a small box of the same shape
    L0, g0 = c["box"][0], c["grid"][0]
    h = L0 / g0

    def make(L):
        g = int(round(L / h))
        L = g * h
        n_poly = max(1, int(round(c["n_poly"] * (L / L0) ** 3)))
        return Oracle(n_poly, c["N"], c["n_A"], (L, L, L), (g, g, g), c["chiN"], c["kappaN"], seed=c["seed"])

    probe = make(max(4.0, L0 / 4))
    X = probe.init()
    t = time.perf_counter()
    probe.run(X, 0, 2, n_threads=cores)
    rate = 2 * probe.n_b / (time.perf_counter() - t)
    steps = 3 if steps_cap is None else steps_cap
    target_beads = rate * budget_s / steps
    L = min(L0, max(4.0, L0 * (target_beads / (c["n_poly"] * c["N"])) ** (1 / 3)))
    o = make(L)
    if steps_cap is None:  # a full-size system done in under the budget: more steps of it
        steps = max(steps, min(60, int(rate * budget_s / o.n_b)))
    X = o.init()
    t = time.perf_counter()
    o.run(X, 0, steps, n_threads=cores)
    dt = time.perf_counter() - t
    sample = (f"{steps} full oracle steps (moves, re-binning, field rebuild) of a {o.n_b}-bead system of the "
              f"{name} shape (box {o.d.box[0]:g}^3, grid {o.d.grid[0]}^3, same N, density, chiN, kappaN)")
    return {"value": steps * o.n_b / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": dt}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import Oracle
    from paper_2606_09356_b300 import workloads
    c = workloads.system_kwargs(args.workload)
    cores = os.cpu_count() or 1
    # bounded sample: shrink the box (same shape) so the K + W steps fit in ~2 minutes
    probe = Oracle(max(1, c["n_poly"] // 64), c["N"], c["n_A"], tuple(b / 4 for b in c["box"]),
                   tuple(g // 4 for g in c["grid"]), c["chiN"], c["kappaN"], seed=c["seed"])
    X = probe.init()
    t = time.perf_counter()
    probe.run(X, 0, 1, n_threads=cores)
    rate = probe.n_b / (time.perf_counter() - t)
    total_steps = args.steps + args.warmup
    frac = min(1.0, rate * 120.0 / (total_steps * c["n_poly"] * c["N"]))
    L0, g0 = c["box"][0], c["grid"][0]
    g = max(8, int(round(g0 * frac ** (1 / 3))))
    L = L0 * g / g0
    n_poly = max(1, int(round(c["n_poly"] * (g / g0) ** 3)))
    o = Oracle(n_poly, c["N"], c["n_A"], (L, L, L), (g, g, g), c["chiN"], c["kappaN"], seed=c["seed"])
    X = o.init()
    o.run(X, 0, args.warmup, n_threads=cores)
    t = time.perf_counter()
    o.run(X, args.warmup, args.steps, n_threads=cores)
    dt = time.perf_counter() - t
    value = args.steps * o.n_b / dt
    sample = (f"full oracle steps of a {o.n_b}-bead system of the {args.workload} shape (box {L:g}^3, grid {g}^3, "
              f"same N, density, chiN, kappaN)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, c), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2606_09356_b300 import build as _build
    from paper_2606_09356_b300 import soma, workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    if rank == 0:
        _build.build()
    if pg:
        pg.barrier()
    soma.load_library()

    c = workloads.system_kwargs(args.workload)
    system = soma.System(**rank_system_kwargs(args.workload, rank))
    n_b, n_c = system.n_beads, system.n_cells
    hbm_peak, peak_kind = _peaks()

    # CPU baseline first (no GPU work in flight), rank 0 at N = 1 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.workload)

    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # the autotuner times trial steps with CUDA events; under a profiler those
    # timings are distorted (serialised, cache-flushed launches), so profiling
    # runs pass --no-autotune and get the default launch shape (8 consumer
    # warps, 3 CTAs per SM), which ties with the autotuner's pick on this
    # workload outside a profiler
    # kernel_timing = 0: no timing events of the library's own inside the step
    # windows; a step is one launch of the move kernel (the launch counts
    # below confirm it), so the window is that launch's duration
    h = soma.Handle(system, device=local, kernel_timing=0, graph_steps=0, autotune=0 if args.no_autotune else 1)
    sptr = stream.cuda_stream

    def one_step():
        h.mc_steps(1, stream=sptr)

    # warm-up (the first call runs the autotuner, which restores the state it tried on)
    warm_up(torch, stream, flush, one_step, args.warmup)
    h.kernel_times(reset=True)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with Clocks(local) as clk:
        hold_stream(torch, stream, args.steps)
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))          # evict the L2 between timed steps
                ev[i][0].record(stream)
            one_step()
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    kt = h.kernel_times(reset=True)
    info_after = h.info()
    total_ms, moves, value = aggregate(total_ms, args.steps * n_b, pg, device="cuda")
    sorts = kt["reorder"][1]
    # the library's own kernels in the timed region: move (+ bin / field where
    # used) per step, and three per chain reorder (keys, permute, copy back)
    launches = kt["move"][1] + kt["bin"][1] + kt["field"][1] + sorts * 3

    # dominant kernel: the move kernel, its average launch duration = the
    # step windows' mean when every step is exactly one move launch
    mv_n = kt["move"][1]
    one_launch = mv_n == args.steps and launches == args.steps
    move_avg = total_ms / args.steps if one_launch else None
    if move_avg is None:  # a reorder or a separate histogram launch inside a window:
        # time the move kernel alone with the library's events, same shape
        move_avg = move_kernel_ms(soma, torch, system, local, sptr, stream, flush, args.steps, args.warmup,
                                  info_after)
    achieved = move_kernel_bytes(n_b, n_c) / (move_avg * 1e-3) / 1e9
    traffic = _profiled_traffic(args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_move", "move_ms": move_avg,
                "timing": ("CUDA events around each step's single launch of the move kernel, on its stream"
                           if one_launch else "the library's CUDA events around each move launch, a separate "
                           "pass in the same launch shape"),
                "step_frac": algorithmic_bytes(n_b, n_c) * args.steps / (total_ms * 1e-3) / 1e9 / hbm_peak}

    # steady state without flushes: CUDA-graph replay of many steps (L2-warm)
    steady = None
    if not args.no_steady:
        hg = soma.Handle(soma.System(**{**c, "system_id": rank}), device=local)
        hg.mc_steps(args.warmup + 16, stream=sptr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_st = max(args.steps, 64)
        with torch.cuda.stream(stream):
            a.record(stream)
        hg.mc_steps(n_st, stream=sptr)
        with torch.cuda.stream(stream):
            b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        steady = {"value": n_st * n_b / (ms * 1e-3), "unit": UNIT, "steps": n_st,
                  "note": "CUDA-graph replay, no L2 flush between steps, reorder every "
                          f"{hg.info()['sort_interval']} steps"}
        hg.close()

    # energy per step (context: the paper reports energy per unit of work):
    # NVML's energy counter across about two seconds of CUDA-graph replays
    energy = None
    if not args.no_energy:
        energy = measure_energy(soma, torch, c, rank, local, sptr, stream, n_b)

    # end to end through the public API with pinned host buffers: the state
    # goes up once, every step's accepted count comes down (enqueued behind
    # its step, one synchronisation at the end), then the final counts
    e2e = None
    if not args.no_e2e:
        he = soma.Handle(soma.System(**rank_system_kwargs(args.workload, rank)), device=local, autotune=1,
                         graph_steps=0)
        he.mc_steps(args.warmup, stream=sptr)  # tuning and warm-up, untimed
        torch.cuda.synchronize()
        pos, img, step = he.get_state()
        pin_pos = torch.from_numpy(pos).pin_memory()
        pin_img = torch.from_numpy(img).pin_memory()
        dens = torch.empty((2, n_c), dtype=torch.int32).pin_memory()
        accs = torch.zeros(args.steps, dtype=torch.int64).pin_memory()
        acc_np = accs.numpy()
        # one untimed pass of the same calls (first-call costs: staging, pinned paths)
        he.set_state(pin_pos.numpy(), pin_img.numpy(), step)
        for i in range(min(3, args.steps)):
            he.mc_steps(1, stream=sptr)
            he.copy_accepted(acc_np[i:i + 1], stream=sptr)
        he.get_density(out=dens.numpy().view(np.uint32))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        he.set_state(pin_pos.numpy(), pin_img.numpy(), step)
        for i in range(args.steps):
            he.mc_steps(1, stream=sptr)
            he.copy_accepted(acc_np[i:i + 1], stream=sptr)  # the step's result, 8 bytes to the host
        he.get_density(out=dens.numpy().view(np.uint32))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = int(acc_np[-1]) == he.accepted() and bool(np.all(np.diff(acc_np) >= 0))
        he.close()
        h2d = (pos.nbytes + img.nbytes) / args.steps
        d2h = 8 + dens.numel() * 4 / args.steps
        e2e = {"value": args.steps * n_b * ws / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "results_consistent": ok,
               "note": "set_state from pinned host; per step soma_mc_steps + soma_copy_accepted to pinned "
                       "host (enqueued behind the step); then soma_get_density to pinned host; host wall clock"}

    # the bond-force-biased (smart) move on the same workload, timed like the
    # headline (L2 flushed between steps, CUDA events around each step)
    smart = umbrella = zones = None
    if not args.no_smart:
        kw = rank_system_kwargs(args.workload, rank)
        smart = bench_variant(soma, torch, args.workload, kw, local, sptr, stream, flush, args.steps, args.warmup,
                              hbm_peak, n_b, n_c, move=soma.SOMA_MOVE_SMART, sm_max_mhz=clk.max_mhz,
                              note="SOMA_MOVE_SMART, same workload, L2 flushed between timed steps")
        umbrella = bench_variant(soma, torch, args.workload, kw, local, sptr, stream, flush, args.steps,
                                 args.warmup, hbm_peak, n_b, n_c, umbrella=50.0,
                                 note="umbrella restraint (lambdaN = 50) toward a lamellar target: field "
                                      "array from the counts, then the move kernel, per step; L2 flushed")
        zones = bench_variant(soma, torch, args.workload, kw, local, sptr, stream, flush, args.steps,
                              args.warmup, hbm_peak, n_b, n_c, wall_z=1, sm_max_mhz=clk.max_mhz,
                              conversion=(kw["n_A"] // 2, 2.0, 2.0, (0.05, 0.02, 0.03, 0.04)),
                              note="walls in z and boundary-zone conversion (zones 2 R_e wide, per-step "
                                   "rates 0.02-0.05): each chain's conversion decided inside the move kernel, "
                                   "whose moves and counts use the new types; L2 flushed")

    # the second full-size melt (1,048,576 chains of 64, grid 256^3), timed like
    # the headline in the same run: the HBM-roofline target covers both
    second = None
    if not args.no_config2 and args.workload != SECOND_WORKLOAD:
        kw2 = rank_system_kwargs(SECOND_WORKLOAD, rank)
        s2 = soma.System(**kw2)
        second = bench_variant(soma, torch, SECOND_WORKLOAD, kw2, local, sptr, stream, flush, args.steps,
                               args.warmup, hbm_peak, s2.n_beads, s2.n_cells,
                               note="second melt workload, uniform moves, L2 flushed between timed steps "
                                    "(positions alone exceed the L2)")
        second = {"workload": workload_desc(SECOND_WORKLOAD, workloads.system_kwargs(SECOND_WORKLOAD)),
                  "n_beads": s2.n_beads, "n_cells": s2.n_cells, "steps": args.steps,
                  "algorithmic_bytes_per_step": algorithmic_bytes(s2.n_beads, s2.n_cells), **second}

    # batched replicas vs sequential plain runs of the same 64 systems
    batched = None
    if rank == 0 and not args.no_batched:
        batched = bench_batched(soma, workloads, torch, sptr, stream, hbm_peak, steps=args.batched_steps)
    h.close()

    if rank == 0:
        clk_summary = clk.summary()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, c), "n_beads": n_b, "n_cells": n_c,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "sort_interval": info_after["sort_interval"],
                       "tuned": {k: info_after[k] for k in ("ctas_per_sm", "hist_mode", "move_warps")},
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "step_ms_stats": {"median": float(statistics.median(step_ms)), "min": float(min(step_ms)),
                              "max": float(max(step_ms))},
            "issue_roofline": issue_roofline(args.workload, "", move_avg, clk_summary.get("sm_max_mhz")),
            "clocks": clk_summary, "steady_state": steady, "energy": energy, "smart_moves": smart, "umbrella": umbrella,
            "boundary_zones": zones,
            "config2": second,
            "batched": batched,
            "wall_s_timed": wall,
        }
        print(json.dumps(out))
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_partitioned(args):
    """One system split by chains over the ranks (one GPU each): every timed
    step is the rank's move kernel over its chains plus the all-reduce (sum)
    of the partial counts (NCCL between GPUs; a no-op at one rank).  Strong
    scaling: the whole system's moves over the slowest rank's time."""
    import torch

    from paper_2606_09356_b300 import build as _build
    from paper_2606_09356_b300 import partition, soma, workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    if rank == 0:
        _build.build()
    if pg:
        pg.barrier()
    soma.load_library()
    c = workloads.system_kwargs(args.partition_workload)
    system = soma.System(**c)
    begin, end = partition.chain_range(system.n_poly, rank, ws)
    hbm_peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()  # the steps and the all-reduces share it
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    h = soma.Handle(system, partition=(begin, end), device=local, kernel_timing=1, graph_steps=0)
    reduce = partition.all_reduce_sum() if pg else (lambda t: None)
    partition.exchange(h, reduce, stream)  # the exchange after creation

    def one_step():
        partition.step(h, reduce, stream)

    warm_up(torch, stream, flush, one_step, args.warmup)
    h.kernel_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
            one_step()
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    kt = h.kernel_times(reset=True)
    move_ms = kt["move"][0] / max(1, kt["move"][1])
    # whole-job moves: every rank's chains (their sum is the system)
    total_ms, moves, value = aggregate(total_ms, args.steps * (end - begin) * system.N, pg, device="cuda")
    h.close()
    if rank == 0:
        local_bytes = 24 * (end - begin) * system.N + 32 * system.n_cells
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload_desc(args.partition_workload, c), "n_beads": system.n_beads,
                          "n_cells": system.n_cells, "l2": "flushed between timed steps (256 MiB write)",
                          "parallelism": f"chain partition x{ws}, counts all-reduced every step"},
               "roofline": {"bound": "hbm", "kernel": "k_move", "move_ms": move_ms, "unit": "GB/s",
                            "achieved": local_bytes / (move_ms * 1e-3) / 1e9, "peak": hbm_peak,
                            "frac": local_bytes / (move_ms * 1e-3) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                            "traffic": None},
               "exchange_bytes_per_step": 8 * system.n_cells, "gpu_launches": kt["move"][1],
               "cpu_baseline": None, "e2e": None, "clocks": clk.summary()}
        print(json.dumps(out))
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def measure_energy(soma, torch, c, rank, local, sptr, stream, n_b, seconds=2.0):
    try:
        nv = _Nvml(local)
        nv.energy_mj()
    except Exception as e:
        return {"error": repr(e)}
    h = soma.Handle(soma.System(**{**c, "system_id": rank}), device=local)
    h.mc_steps(64, stream=sptr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.mc_steps(256, stream=sptr)
    torch.cuda.synchronize()
    per = (time.perf_counter() - t0) / 256
    n = max(256, int(seconds / per))
    e0, t0 = nv.energy_mj(), time.perf_counter()
    h.mc_steps(n, stream=sptr)
    torch.cuda.synchronize()
    e1, t1 = nv.energy_mj(), time.perf_counter()
    h.close()
    joules = (e1 - e0) * 1e-3
    return {"steps": n, "seconds": t1 - t0, "joules_per_step": joules / n, "moves_per_joule": n * n_b / joules
            if joules > 0 else None, "avg_power_w": joules / (t1 - t0),
            "note": "NVML total-energy counter over CUDA-graph replays (L2 warm), whole GPU board"}


def move_kernel_ms(soma, torch, system, device, sptr, stream, flush, steps, warmup, info):
    """Average move-kernel launch time by the library's CUDA events around
    each launch, in the given launch shape (ctas_per_sm, hist_mode), L2
    flushed before every step."""
    h = soma.Handle(system, device=device, kernel_timing=1, graph_steps=0, autotune=0,
                    ctas_per_sm=info["ctas_per_sm"], hist_mode=info["hist_mode"])
    warm_up(torch, stream, flush, lambda: h.mc_steps(1, stream=sptr), warmup)
    h.kernel_times(reset=True)
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        h.mc_steps(1, stream=sptr)
    torch.cuda.synchronize()
    ms, n = h.kernel_times(reset=True)["move"]
    h.close()
    return ms / max(1, n)


def bench_variant(soma, torch, workload, kw, device, sptr, stream, flush, steps, warmup, hbm_peak, n_b, n_c,
                  move=0, umbrella=0.0, wall_z=0, conversion=None, note="", sm_max_mhz=None):
    """The workload with another trial move, the umbrella restraint, or walls
    and boundary-zone conversion: moves/s over flushed steps and the move
    kernel's fraction of the HBM roofline (same algorithmic bytes per step as
    the headline)."""
    # one launch per step unless the umbrella's field pass precedes it: then
    # the library's events time the two kernels apart
    h = soma.Handle(soma.System(**{**kw, "move": move, "wall_z": wall_z}), device=device,
                    kernel_timing=1 if umbrella else 0, graph_steps=0, autotune=1)
    if conversion:
        h.set_conversion(*conversion)
    if umbrella:
        import numpy as np
        nx = kw["grid"][0]
        x = (np.arange(nx) + 0.5) / nx
        pA = np.repeat(0.5 + 0.4 * np.sin(4 * np.pi * x), kw["grid"][1] * kw["grid"][2])
        h.set_umbrella(np.stack([pA, 1.0 - pA]).astype(np.float32), umbrella)
    warm_up(torch, stream, flush, lambda: h.mc_steps(1, stream=sptr), warmup)
    h.kernel_times(reset=True)
    a0 = h.accepted()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    hold_stream(torch, stream, steps)
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev[i][0].record(stream)
        h.mc_steps(1, stream=sptr)
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    total_ms = sum(x.elapsed_time(y) for x, y in ev)
    kt = h.kernel_times(reset=True)
    acc = (h.accepted() - a0) / (steps * n_b)
    conv_n = int(h.conversions().sum()) if conversion else 0
    info = h.info()
    h.close()
    mv_ms, mv_n = kt["move"]
    fd_ms, fd_n = kt["field"]
    if umbrella:
        move_avg = mv_ms / max(1, mv_n)
    elif mv_n == steps and kt["bin"][1] == 0 and kt["reorder"][1] == 0:
        move_avg = total_ms / steps  # each window is one launch of the move kernel
    else:
        move_avg = move_kernel_ms(soma, torch, soma.System(**{**kw, "move": move, "wall_z": wall_z}), device, sptr,
                                  stream, flush, steps, warmup, info)
    achieved = move_kernel_bytes(n_b, n_c) / (move_avg * 1e-3) / 1e9
    out = {"value": steps * n_b / (total_ms * 1e-3), "unit": UNIT, "ms_per_step": total_ms / steps,
           "move_ms": move_avg, "achieved_gbs": achieved, "frac": achieved / hbm_peak, "acceptance": acc,
           "tuned": {k: info[k] for k in ("ctas_per_sm", "hist_mode", "move_warps")}, "note": note}
    if fd_n:
        out["field_ms"] = fd_ms / fd_n
    if conversion:
        out["conversions_per_step"] = float(conv_n) / (steps + warmup)
    # the committed ncu summary of this kernel specialisation and workload
    # (the plain uniform move of another workload too), when there is one
    variant = "_smart" if move else "_zones" if conversion else None if umbrella else ""
    if variant is not None:
        out["traffic"] = _profiled_traffic(workload, variant)
        iss = issue_roofline(workload, variant, move_avg, sm_max_mhz)
        if iss:
            out["issue_frac"] = iss["frac"]
    return out


def bench_batched(soma, workloads, torch, sptr, stream, hbm_peak, steps=20):
    """Aggregate moves/s of the 64-system batch in one handle (one launch per
    kernel per step for all systems, CUDA graphs) against the same systems run
    one after another, each in its own handle with plain launches (one
    soma_mc_steps call per system; create excluded).  roofline_frac: the
    batch's own algorithmic bytes per step (24 B per bead + 32 B per cell,
    summed over the systems) over the batched step time, against the
    measured copy bandwidth; the batch's positions (528 MB) exceed the L2."""
    specs = workloads.batch64()
    systems = [soma.System(**{k: v for k, v in d.items() if k != "f_A"}) for d in specs]
    moves = sum(s.n_beads for s in systems) * steps
    hb = soma.Handle(systems)
    hb.mc_steps(4, stream=sptr)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
    hb.mc_steps(steps, stream=sptr)
    with torch.cuda.stream(stream):
        b.record(stream)
    torch.cuda.synchronize()
    batched_ms = a.elapsed_time(b)
    hb.close()
    plain_ms = 0.0
    for s in systems:
        h = soma.Handle(s, graph_steps=0)
        h.mc_steps(2, stream=sptr)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            a.record(stream)
        h.mc_steps(steps, stream=sptr)  # one call: the library enqueues one plain launch per step
        with torch.cuda.stream(stream):
            b.record(stream)
        torch.cuda.synchronize()
        plain_ms += a.elapsed_time(b)
        h.close()
    step_bytes = sum(algorithmic_bytes(s.n_beads, s.n_cells) for s in systems)
    ms_step = batched_ms / steps
    return {"value": moves / (batched_ms * 1e-3), "plain_sequential": moves / (plain_ms * 1e-3),
            "speedup": plain_ms / batched_ms, "unit": UNIT, "systems": len(systems), "steps": steps,
            "beads": sum(s.n_beads for s in systems), "cells": sum(s.n_cells for s in systems),
            "ms_per_step": ms_step, "algorithmic_bytes_per_step": step_bytes,
            "roofline_frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm_peak,
            "speedup_at_roofline": plain_ms / steps / (step_bytes / (hbm_peak * 1e9) * 1e3)}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", default="melt_131072x32")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-steps", type=int, default=20)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-steady", action="store_true")
    p.add_argument("--no-smart", action="store_true")
    p.add_argument("--no-config2", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="the headline handle keeps the default launch shape (for profiler runs)")
    p.add_argument("--partition", action="store_true",
                   help="one system split by chains over the ranks, counts all-reduced every step (strong "
                        "scaling; --partition-workload names the system)")
    p.add_argument("--partition-workload", default=SECOND_WORKLOAD)
    p.add_argument("--no-energy", action="store_true")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.partition:
        run_partitioned(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
