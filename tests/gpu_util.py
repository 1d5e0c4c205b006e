"""Helpers shared by the GPU parity tests: build the library, mirror a GPU
system in the oracle, and compare one Monte Carlo step element by element."""
import os

import numpy as np

from oracle import Oracle
from paper_2606_09356_b300 import build as _build
from paper_2606_09356_b300 import soma

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def lib():
    _build.build()
    return soma.load_library()


def oracle_for(system, pos64=False):
    """The oracle of a system; pos64 selects the FP64 cell lookup of the
    FP64-position form."""
    return Oracle(system.n_poly, system.N, system.n_A, system.box, system.grid, system.chiN, system.kappaN,
                  A=system.A, seed=system.seed, sys_index=system.system_id, move=system.move,
                  wall_z=system.wall_z, pos64=int(pos64))


def unwrapped(h, sys=0):
    pos, img, step = h.get_state(sys)
    box = np.array(h.systems[sys].box)
    return pos.astype(np.float64) + img.astype(np.float64) * box, step


def band_for(system, k_b):
    """Margin band inside which FP32-vs-FP64 decisions may differ: 1e-5 or,
    for boxes whose last-bit error of a wrapped coordinate carried across the
    periodic boundary is larger, 4 k_b |b|_max ulp(L) with |b|_max = 1."""
    ulp = np.spacing(np.float32(max(system.box)))
    return max(1e-5, 4.0 * k_b * 1.0 * float(ulp))


def compare_step(h, sys=0, band=None, n_threads=NTHREADS, check_counts=True, w=None, orc=None, fields=None):
    """Run one GPU step and one oracle step from the same state and compare.

    Returns a dict of statistics.  Raises AssertionError on a mismatch: an
    accept decision that differs although |dE + ln u| >= band and both the old
    and the proposed position are further than 8 ulp(L) from a cell face
    (beads next to such a bead in the chain are set aside too), a position
    further than 1e-5 L from the oracle's, or counts that differ from the
    oracle's binning of the GPU's own positions.  ``w`` overrides the fields
    the oracle moves against (default: the fields of the current counts, or
    ``fields(orc, counts)``).  ``orc`` is the oracle to use; with its
    boundary-zone conversion on, the GPU's molecule types are imported
    before the step, the oracle converts before it moves, and the types and
    conversion counts after the step must agree bit for bit."""
    system = h.systems[sys]
    orc = oracle_for(system) if orc is None else orc
    conv = orc.types is not None
    k_b, _, _ = orc.params()
    band = band_for(system, k_b) if band is None else band
    X0, step = unwrapped(h, sys)
    if conv:
        orc.set_types(h.chain_types(sys))
    counts0 = orc.density(X0)
    if check_counts:
        assert np.array_equal(h.get_density(sys), counts0), "counts differ before the step"
    if w is None:
        w = orc.fields(counts0) if fields is None else fields(orc, counts0)
    if conv:
        conv0 = h.conversions(sys).astype(np.int64)
        c4 = orc.convert(X0, step)
    Xo = X0.copy()
    n_acc, acc, margin, face = orc.mc_step(Xo, w, step, n_threads=n_threads)
    a0 = h.accepted(sys)
    h.mc_steps(1)
    X1, step1 = unwrapped(h, sys)
    assert step1 == step + 1
    if conv:
        assert np.array_equal(h.chain_types(sys), orc.types), "molecule types differ after the conversions"
        assert np.array_equal(h.conversions(sys).astype(np.int64) - conv0, c4), "conversion counts differ"
    moved = np.any(X1 != X0, axis=1)
    face_tol = 8.0 * float(np.spacing(np.float32(max(system.box))))
    suspect = (np.abs(margin) < band) | (face < face_tol)
    # a flipped decision changes the neighbours' energies in the later set
    N = system.N
    sus = suspect.reshape(-1, N)
    spread = sus.copy()
    spread[:, 1:] |= sus[:, :-1]
    spread[:, :-1] |= sus[:, 1:]
    ok = ~spread.reshape(-1)
    bad = ok & (moved != acc.astype(bool))
    assert not bad.any(), (f"{bad.sum()} accept decisions differ outside the band "
                           f"(first bead {np.nonzero(bad)[0][:5]}, margins {margin[bad][:5]})")
    L = np.array(system.box)
    dev = np.abs(X1 - Xo)[ok] / L
    assert dev.size == 0 or dev.max() <= 1e-5, f"positions differ by {dev.max():.3g} L"
    if check_counts:
        assert np.array_equal(h.get_density(sys), orc.density(X1)), "counts differ from binning of GPU positions"
    gpu_acc = h.accepted(sys) - a0
    return dict(n=len(X0), suspect=int(spread.sum()), acc_gpu=int(gpu_acc), acc_orc=int(n_acc),
                moved=int(moved.sum()), max_dev=float(dev.max()) if dev.size else 0.0)
