"""Hard walls in z (the particle subdomain as a slab, Sec. 3.2) on the GPU
against the oracle (needs a GPU): step-by-step parity, the folded initial
configuration, confinement, invariance, and the exact dimer law between
walls."""
import numpy as np
import pytest

import gpu_util as G
import pins
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


SHAPES = [
    dict(workloads.system_kwargs("melt_512x32")),
    dict(workloads.system_kwargs("melt_512x32"), move=soma.SOMA_MOVE_SMART),
    dict(n_poly=37, N=7, n_A=3, box=(4.0, 4.5, 5.0), grid=(16, 18, 20), chiN=15.0, kappaN=40.0, seed=7),
    dict(n_poly=40, N=80, n_A=30, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=25.0, kappaN=50.0, seed=7),  # generic
    dict(n_poly=200, N=1, n_A=1, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=5.0, kappaN=10.0, A=0.25),
]


@pytest.mark.parametrize("kw", SHAPES)
@pytest.mark.parametrize("ctas", [1, 3])
def test_wall_step_parity(kw, ctas):
    s = soma.System(wall_z=1, **kw)
    band = 1e-4 if s.move == soma.SOMA_MOVE_SMART else None
    with soma.Handle(s, ctas_per_sm=ctas, graph_steps=0) as h:
        for _ in range(4):
            st = G.compare_step(h, band=band)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]


def test_wall_initial_configuration_matches_oracle_and_stays_in_the_slab():
    s = soma.System(wall_z=1, **workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    ref = orc.init()
    with soma.Handle(s) as h:
        X, _ = G.unwrapped(h)
        assert np.abs(X - ref).max() <= 1e-5 * max(s.box)
        h.mc_steps(200)
        pos, img, _ = h.get_state()
    assert pos[:, 2].min() >= 0.0 and pos[:, 2].max() < s.box[2]
    assert not img[:, 2].any()


def test_wall_trajectories_invariant_to_graphs_reorders_and_batching():
    base = dict(n_poly=777, N=32, n_A=16, box=(4.0, 4.0, 5.0), grid=(16, 16, 20), chiN=20.0, kappaN=50.0)
    systems = [soma.System(**base, seed=60 + i, system_id=i, wall_z=i % 2, move=(i // 2) % 2) for i in range(4)]

    def run(ss, **opts):
        with soma.Handle(ss, **opts) as h:
            h.mc_steps(24)
            return [(h.get_state(i)[0], h.get_density(i), h.accepted(i)) for i in range(len(ss))]

    plain = [run([x], graph_steps=0, sort_interval=0)[0] for x in systems]
    graphed = [run([x], graph_steps=8, sort_interval=5)[0] for x in systems]
    batched = run(systems)
    for a, b, c in zip(plain, graphed, batched):
        for x, y, z in zip(a, b, c):
            assert np.array_equal(x, y) and np.array_equal(x, z)


def test_wall_dimer_cell_pair_law_in_frozen_field():
    """AB dimers on a 2^3 grid between walls in z: the exact law with no
    periodic images in z (cells 5 R_e wide: a long run mixes them)."""
    rng = np.random.default_rng(25)
    box, grid = (10.0, 10.0, 10.0), (2, 2, 2)
    s = soma.System(n_poly=65536, N=2, n_A=1, box=box, grid=grid, chiN=0.0, kappaN=0.0, A=1.0, wall_z=1)
    w = rng.normal(0.0, 0.7, size=(2, 8)).astype(np.float32)
    Ks = [pins._bond_cell_kernel(box[0], grid[0], 1.5), pins._bond_cell_kernel(box[1], grid[1], 1.5),
          pins._bond_cell_kernel(box[2], grid[2], 1.5, images=0)]
    cells = [(ix, iy, iz) for ix in range(2) for iy in range(2) for iz in range(2)]
    P = np.zeros((8, 8))
    for c1, (a1, b1, z1) in enumerate(cells):
        for c2, (a2, b2, z2) in enumerate(cells):
            P[c1, c2] = np.exp(-float(w[0, c1]) - float(w[1, c2])) * Ks[0][a1, a2] * Ks[1][b1, b2] * Ks[2][z1, z2]
    P /= P.sum()

    def cells_of(pos):
        i = np.minimum((pos * (np.array(grid) / np.array(box))).astype(np.int64), np.array(grid) - 1)
        return (i[:, 0] * grid[1] + i[:, 1]) * grid[2] + i[:, 2]

    with soma.Handle(s) as h:
        h.freeze_fields(w)
        h.mc_steps(1500)
        samples = []
        for _ in range(16):
            hist = np.zeros(64)
            for _ in range(10):
                h.mc_steps(25)
                c = cells_of(h.get_state()[0])
                np.add.at(hist, c[0::2] * 8 + c[1::2], 1)
            samples.append(hist / hist.sum())
    fails = []
    pins._block_test(fails, "gpu wall dimer", np.array(samples), P.reshape(-1), zmax=6.0)
    assert not fails, fails
