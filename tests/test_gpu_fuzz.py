"""Randomised shapes against the oracle (needs a GPU): chain lengths across
the register and generic paths, odd and even N, anisotropic boxes, dyadic
and non-dyadic grids, both move kinds, walls, the umbrella, held fields,
boundary-zone conversion; and handles mixing such systems against the same
systems run alone."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def random_system(rng, i):
    N = int(rng.choice([1, 2, 3, 5, 8, 13, 31, 32, 33, 47, 64, 65, 100]))
    n_A = int(rng.integers(0, N + 1))
    n_poly = int(rng.integers(1, 400))
    move = int(rng.integers(0, 2))
    A = 0.0
    if N == 1:
        A = float(rng.uniform(0.05, 0.3))
    min_box = 16.0 / np.sqrt(3.0 * (N - 1)) if N > 1 else 0.5
    box = tuple(float(np.round(min_box * rng.uniform(1.0, 2.5), 3)) for _ in range(3))
    if move == 1 and N > 1:
        A = 0.0  # the default half-width satisfies the smart-move bounds
    if move == 1 and N == 1:
        A = min(A, 0.1 * min(box))  # Gaussian tail within half the box
    grid = tuple(int(rng.integers(1, 24)) for _ in range(3))
    if move == 1 and N > 64:
        move = 0  # smart moves run on the register path only
    return soma.System(n_poly=n_poly, N=N, n_A=n_A, box=box, grid=grid, chiN=float(rng.uniform(0, 40)),
                       kappaN=float(rng.uniform(0, 60)), A=A, seed=int(rng.integers(1, 2**40)), system_id=i,
                       move=move, wall_z=int(rng.integers(0, 2)))


def random_conversion(rng, s):
    """Boundary-zone conversion for half of the register-path systems: a
    random converted A block, zone widths and per-step rates (or None)."""
    if s.N > 64 or rng.integers(0, 2) == 0:
        return None
    Lz = s.box[2]
    lo = float(rng.uniform(0, 0.5 * Lz))
    hi = float(rng.uniform(0, 0.5 * Lz))
    return (int(rng.integers(0, s.N + 1)), lo, hi, tuple(float(v) for v in rng.uniform(0, 1, 4)))


@pytest.mark.parametrize("seed", range(80))
def test_random_shape_steps_match_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    s = random_system(rng, 0)
    orc = G.oracle_for(s)
    band = 1e-4 if s.move else None
    # the block shape cycles with the seed (no draw from rng: the shapes stay
    # those of the seed); resident CTAs above a shape's limit are clamped
    with soma.Handle(s, graph_steps=0, ctas_per_sm=int(rng.integers(0, 4)), move_warps=(8, 12, 24)[seed % 3]) as h:
        mode = int(rng.integers(0, 3))
        tg, lam = None, float(rng.uniform(1, 60))
        if mode == 1:  # umbrella toward a random target
            tg = rng.uniform(0.0, 1.5, size=(2, s.n_cells)).astype(np.float32)
            h.set_umbrella(tg, lam)
        elif mode == 2:  # held fields
            w = rng.normal(0, 0.5, size=(2, s.n_cells)).astype(np.float32)
            h.freeze_fields(w)
        conv = random_conversion(rng, s)
        if conv:
            orc.set_conversion(*conv)
            h.set_conversion(*conv)
        for _ in range(3):
            X0, _ = G.unwrapped(h)
            if conv:
                orc.set_types(h.chain_types())
            counts = orc.density(X0)
            if mode == 1:
                w64 = orc.fields_umbrella(counts, tg.astype(np.float64), lam)
            elif mode == 2:
                w64 = w.astype(np.float64)
            else:
                w64 = orc.fields(counts)
            st = G.compare_step(h, band=band, w=w64, orc=orc)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]


@pytest.mark.parametrize("seed", range(20))
def test_random_mixed_handles_equal_solo_runs(seed):
    rng = np.random.default_rng(2000 + seed)
    systems = [random_system(rng, i) for i in range(int(rng.integers(2, 7)))]
    steps = int(rng.integers(5, 30))
    opts = dict(graph_steps=int(rng.choice([0, 4])), sort_interval=int(rng.choice([0, 3])))
    convs = [random_conversion(rng, s) for s in systems]
    with soma.Handle(systems, **opts) as hb:
        for i, c in enumerate(convs):
            if c:
                hb.set_conversion(*c, sys=i)
        hb.mc_steps(steps)
        batched = [(hb.get_state(i)[0], hb.get_density(i), hb.accepted(i), hb.chain_types(i))
                   for i in range(len(systems))]
    for i, s in enumerate(systems):
        with soma.Handle(s, graph_steps=0, sort_interval=0) as h:
            if convs[i]:
                h.set_conversion(*convs[i])
            h.mc_steps(steps)
            solo = (h.get_state()[0], h.get_density(), h.accepted(), h.chain_types())
        for x, y in zip(batched[i], solo):
            assert np.array_equal(x, y)
