"""CUDA path against the oracle, element by element (needs a GPU).

Kernel (b) is compared bit for bit (integer counts of identical positions),
kernel (c) within a bound derived from its FP32 arithmetic, kernel (a) by
accept decisions and positions of whole steps started from identical states."""
import numpy as np
import pytest

import gpu_util as G
from oracle import Oracle
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def test_device_philox_matches_oracle():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:2] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4]
    key[:2] = [[0, 0], [0xFFFFFFFF] * 2]
    assert np.array_equal(soma.soma_philox4x32(ctr, key), Oracle.philox(ctr, key))


def _fields_bound(orc, counts):
    # |w32 - w64| <= 8 eps32 (|chiN phi| + kappaN (phiA + phiB + 1)) / N
    _, _, rho = orc.params()
    phiA, phiB = counts[0] / rho, counts[1] / rho
    d = orc.d
    scale = (abs(d.chiN) * np.maximum(phiA, phiB) + abs(d.kappaN) * (phiA + phiB + 1.0)) / d.N
    return 8 * np.finfo(np.float32).eps * (scale + 1e-30)


@pytest.mark.parametrize("hist", [soma.SOMA_HIST_FUSED, soma.SOMA_HIST_SEPARATE])
def test_density_and_fields_melt_512x32(hist):
    sysm = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(sysm)
    with soma.Handle(sysm, hist_mode=hist) as h:
        for _ in range(3):
            X, _ = G.unwrapped(h)
            counts = h.get_density()
            assert np.array_equal(counts, orc.density(X))
            assert counts[0].sum() == 512 * 16 and counts[1].sum() == 512 * 16
            w = h.get_fields()
            w64 = orc.fields(counts)
            assert np.all(np.abs(w - w64) <= _fields_bound(orc, counts))
            h.mc_steps(5)


def test_step_parity_melt_512x32_ten_steps():
    sysm = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(sysm, graph_steps=0) as h:
        tot_sus = 0
        for _ in range(10):
            st = G.compare_step(h)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]
            tot_sus += st["suspect"]
        assert tot_sus < 0.001 * 10 * sysm.n_beads


@pytest.mark.parametrize("kw", [
    dict(n_poly=37, N=7, n_A=3, box=(4.0, 4.5, 5.0), grid=(16, 18, 20), chiN=15.0, kappaN=40.0),    # odd N, ragged
    dict(n_poly=301, N=16, n_A=8, box=(2.5, 2.5, 3.0), grid=(10, 10, 12), chiN=20.0, kappaN=50.0),
    dict(n_poly=50, N=64, n_A=19, box=(2.0, 2.0, 2.0), grid=(16, 16, 16), chiN=25.0, kappaN=50.0),  # one warp per chain
    dict(n_poly=40, N=80, n_A=30, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=25.0, kappaN=50.0),     # generic path
    dict(n_poly=9, N=33, n_A=33, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=0.0, kappaN=30.0),       # homopolymer
    dict(n_poly=1, N=2, n_A=1, box=(12.0, 12.0, 12.0), grid=(3, 3, 3), chiN=5.0, kappaN=5.0),       # a single dimer
    dict(n_poly=200, N=1, n_A=1, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=5.0, kappaN=10.0, A=0.3),  # monomers
    dict(n_poly=300, N=24, n_A=9, box=(3.0, 3.3, 2.9), grid=(7, 11, 9), chiN=18.0, kappaN=45.0),     # non-dyadic cells
    dict(n_poly=64, N=16, n_A=8, box=(4.0, 4.0, 4.0), grid=(1, 1, 1), chiN=20.0, kappaN=50.0),      # a single cell
    dict(n_poly=70, N=63, n_A=0, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=20.0, kappaN=50.0),      # odd N, P = 32, all B
    dict(n_poly=3, N=4096, n_A=1000, box=(1.0, 1.0, 1.0), grid=(8, 8, 8), chiN=20.0, kappaN=50.0),  # longest chains
])
@pytest.mark.parametrize("ctas", [1, 3])
def test_step_parity_shapes(kw, ctas):
    sysm = soma.System(seed=7, **kw)
    with soma.Handle(sysm, ctas_per_sm=ctas, graph_steps=0) as h:
        for _ in range(4):
            G.compare_step(h)


def _sampled_parity(name, n_sample, steps=2, **opts):
    """Full-size system in the bench's launch configuration; the oracle
    recomputes a sample of chains one by one with the full system's fields."""
    sysm = soma.System(**workloads.system_kwargs(name))
    orc = G.oracle_for(sysm)
    k_b, _, _ = orc.params()
    band = G.band_for(sysm, k_b)
    rng = np.random.default_rng(17)
    ids = np.sort(rng.choice(sysm.n_poly, n_sample, replace=False)).astype(np.uint32)
    N = sysm.N
    sel = (ids[:, None].astype(np.int64) * N + np.arange(N)[None, :]).reshape(-1)
    with soma.Handle(sysm, **opts) as h:
        h.mc_steps(3)
        for _ in range(steps):
            X0, step = G.unwrapped(h)
            counts = h.get_density()
            assert counts[0].sum() == sysm.n_poly * sysm.n_A
            assert counts[1].sum() == sysm.n_poly * (N - sysm.n_A)
            w = orc.fields(counts)
            Xs = np.ascontiguousarray(X0[sel])
            _, acc, margin, face = orc.mc_step_chains(Xs, ids, w, step, n_threads=G.NTHREADS)
            h.mc_steps(1)
            X1, _ = G.unwrapped(h)
            moved = np.any(X1[sel] != X0[sel], axis=1)
            face_tol = 8.0 * float(np.spacing(np.float32(max(sysm.box))))
            sus = ((np.abs(margin) < band) | (face < face_tol)).reshape(-1, N)
            spread = sus.copy()
            spread[:, 1:] |= sus[:, :-1]
            spread[:, :-1] |= sus[:, 1:]
            ok = ~spread.reshape(-1)
            assert not (ok & (moved != acc.astype(bool))).any()
            dev = np.abs(X1[sel] - Xs)[ok] / np.array(sysm.box)
            assert dev.max() <= 1e-5
        # the whole grid: counts of the GPU's final positions, bit for bit
        X1, _ = G.unwrapped(h)
        assert np.array_equal(h.get_density(), orc.density(X1))


# the launch configuration bench.py times: autotuned shape, plain launches
# with per-kernel timing events
BENCH_OPTS = dict(autotune=1, graph_steps=0, kernel_timing=1)


def test_step_parity_melt_131072x32_full_size_sampled():
    _sampled_parity("melt_131072x32", 4096, **BENCH_OPTS)


def test_step_parity_melt_1048576x64_full_size_sampled():
    _sampled_parity("melt_1048576x64", 2048, steps=1, **BENCH_OPTS)


def test_observables_match_oracle():
    sysm = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(sysm)
    with soma.Handle(sysm) as h:
        h.mc_steps(7)
        X, _ = G.unwrapped(h)
        o = h.observables()
        r = orc.observables(X)
        for k in ("Re2", "Rg2", "Ebond", "Enb"):
            assert o[k] == pytest.approx(r[k], rel=1e-9, abs=1e-9), k
        assert o["step"] == 7 and o["attempted"] == 7 * sysm.n_beads
        assert 0.3 < o["acc"] < 0.9


def test_structure_factor_matches_oracle():
    sysm = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(sysm)
    m = np.array([(x, y, z) for x in range(-3, 4) for y in range(-3, 4) for z in range(0, 4)
                  if 0 < x * x + y * y + z * z <= 12], np.int32)
    with soma.Handle(sysm) as h:
        h.mc_steps(5)
        X, _ = G.unwrapped(h)
        S = h.structure_factor(m)
        R = orc.structure_factor(X, m)
        # FP32 phases of wrapped positions: |dphase| <= ~2e-6 rad per bead
        assert np.allclose(S, R, rtol=2e-4, atol=2e-4)


@pytest.mark.parametrize("variant", ["uniform", "smart", "walls"])
def test_steps_from_the_oracle_state_without_resync(variant):
    """The oracle's own initial configuration (its FP32 image: wrapped
    coordinate plus image count, the numbers the GPU stores) goes into the
    GPU by soma_set_state; then both sides step four times on their own,
    nothing passing from the GPU to the oracle.  Every decision and position
    agrees except for beads set aside for cause, with their chains: a
    margin inside the band or a position near a cell face, at any step so
    far, or an old or new cell whose counts differ between the two sides."""
    kw = dict(workloads.system_kwargs("melt_512x32"))
    if variant == "smart":
        kw["move"] = soma.SOMA_MOVE_SMART
    if variant == "walls":
        kw["wall_z"] = 1
    s = soma.System(**kw)
    orc = G.oracle_for(s)
    k_b, A, _ = orc.params()
    band = max(G.band_for(s, k_b), 1e-4 if variant == "smart" else 0.0)
    # after the first step the GPU keeps FP32-rounded wrapped coordinates and
    # the oracle exact FP64 ones: every step adds up to ulp(L) to their
    # difference, and a bead's dE moves by at most 2 k_b |d| per unit of it
    # for each of its two bonds (|d| <= 2 sqrt(3) A at the two ends)
    ulp = float(np.spacing(np.float32(max(s.box))))
    L = np.array(s.box)
    X = orc.init()
    img = np.floor(X / L)
    xw = (X - img * L).astype(np.float32)
    top = xw >= L.astype(np.float32)  # rounded up to L: the last cell's image is the next one
    xw[top] = 0.0
    img[top] += 1.0
    X = xw.astype(np.float64) + img * L  # the oracle continues from exactly these numbers
    N = s.N
    face_tol = 8.0 * float(np.spacing(np.float32(max(s.box))))
    excluded = np.zeros(s.n_poly, bool)
    with soma.Handle(s, graph_steps=0) as h:
        h.set_state(xw, img.astype(np.int16), 0)
        assert np.array_equal(h.get_density(), orc.density(X))
        for t in range(4):
            counts = orc.density(X)
            diff_cells = np.nonzero((h.get_density() != counts).any(axis=0))[0]
            w = orc.fields(counts)
            X0 = X.copy()
            cells0 = np.array([orc.cell_index(r) for r in X0]) if diff_cells.size else None
            _, acc, margin, face = orc.mc_step(X, w, t, n_threads=G.NTHREADS)
            Xg0, _ = G.unwrapped(h)  # the GPU's own positions before its step
            h.mc_steps(1)
            Xg, _ = G.unwrapped(h)
            band_t = band + 4.0 * k_b * 2.0 * np.sqrt(3.0) * A * ulp * t
            sus = (np.abs(margin) < band_t) | (face < face_tol)
            if diff_cells.size:
                cells1 = np.array([orc.cell_index(r) for r in X])
                sus |= np.isin(cells0, diff_cells) | np.isin(cells1, diff_cells)
            excluded |= sus.reshape(-1, N).any(axis=1)
            ok = np.repeat(~excluded, N)
            assert ok.mean() > 0.9  # chains set aside accumulate over the steps
            moved_g = np.any(Xg != Xg0, axis=1)
            assert not (ok & (moved_g != acc.astype(bool))).any(), t
            assert (np.abs(Xg - X)[ok] / L).max() <= 1e-5, t
