"""Bond-force-biased (smart) moves on the GPU against the oracle (needs a GPU).

Same bar as the uniform move: accept decisions and positions of whole steps
started from identical states, counts bit for bit, trajectories independent
of launch shape, graph capture, reorders and batching, and the Boltzmann
laws of chiN = kappaN = 0 chains."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu

SMART = soma.SOMA_MOVE_SMART
# FP32 margins carry the proposal-asymmetry term |xi|^2/2 (up to ~20 in the
# tails) with relative error ~1e-7 and Phi^-1 with a few ulp: 1e-4 is a wide band
BAND = 1e-4
SMALL = dict(n_poly=777, N=32, n_A=16, box=(4.0, 4.0, 5.0), grid=(16, 16, 20), chiN=20.0, kappaN=50.0, seed=3,
             move=SMART)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


@pytest.mark.parametrize("kw", [
    dict(n_poly=37, N=7, n_A=3, box=(4.0, 4.5, 5.0), grid=(16, 18, 20), chiN=15.0, kappaN=40.0),    # odd N, ragged
    dict(n_poly=301, N=16, n_A=8, box=(2.5, 2.5, 3.0), grid=(10, 10, 12), chiN=20.0, kappaN=50.0),
    dict(n_poly=50, N=64, n_A=19, box=(2.0, 2.0, 2.0), grid=(16, 16, 16), chiN=25.0, kappaN=50.0),  # one warp per chain
    dict(n_poly=9, N=33, n_A=33, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=0.0, kappaN=30.0),       # homopolymer
    dict(n_poly=1, N=2, n_A=1, box=(12.0, 12.0, 12.0), grid=(3, 3, 3), chiN=5.0, kappaN=5.0),       # a single dimer
    dict(n_poly=200, N=1, n_A=1, box=(2.0, 2.0, 2.0), grid=(4, 4, 4), chiN=5.0, kappaN=10.0, A=0.25),  # monomers
])
@pytest.mark.parametrize("ctas", [1, 3])
def test_smart_step_parity_shapes(kw, ctas):
    sysm = soma.System(seed=7, move=SMART, **kw)
    with soma.Handle(sysm, ctas_per_sm=ctas, graph_steps=0) as h:
        for _ in range(4):
            st = G.compare_step(h, band=BAND)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]


def test_smart_step_parity_melt_512x32_ten_steps():
    sysm = soma.System(**{**workloads.system_kwargs("melt_512x32"), "move": SMART})
    with soma.Handle(sysm, graph_steps=0) as h:
        tot_sus, acc = 0, 0
        for _ in range(10):
            st = G.compare_step(h, band=BAND)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]
            tot_sus += st["suspect"]
            acc += st["acc_gpu"]
        assert tot_sus < 0.002 * 10 * sysm.n_beads
        assert 0.5 < acc / (10 * sysm.n_beads) < 1.0


def test_smart_step_parity_in_held_fields():
    sysm = soma.System(**{**workloads.system_kwargs("melt_512x32"), "move": SMART})
    rng = np.random.default_rng(4)
    w = rng.normal(0.0, 0.8, size=(2, sysm.n_cells)).astype(np.float32)
    with soma.Handle(sysm, graph_steps=0) as h:
        h.freeze_fields(w)
        for _ in range(3):
            G.compare_step(h, band=BAND, w=w.astype(np.float64))


@pytest.mark.parametrize("workload,n_sample", [("melt_131072x32", 2048), ("melt_1048576x64", 1024)])
def test_smart_step_parity_full_size_sampled(workload, n_sample):
    """melt_131072x32 and melt_1048576x64 (64-bead chains, a whole warp per chain) with
    smart moves in the bench's launch configuration; the oracle recomputes
    a sample of chains with the full system's fields."""
    sysm = soma.System(**{**workloads.system_kwargs(workload), "move": SMART})
    orc = G.oracle_for(sysm)
    k_b, _, _ = orc.params()
    band = max(BAND, G.band_for(sysm, k_b))
    rng = np.random.default_rng(23)
    ids = np.sort(rng.choice(sysm.n_poly, n_sample, replace=False)).astype(np.uint32)
    N = sysm.N
    sel = (ids[:, None].astype(np.int64) * N + np.arange(N)[None, :]).reshape(-1)
    with soma.Handle(sysm, autotune=1, graph_steps=0, kernel_timing=1) as h:  # as bench.py times it
        h.mc_steps(3)
        X0, step = G.unwrapped(h)
        w = orc.fields(h.get_density())
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
        assert ok.mean() > 0.9
        assert not (ok & (moved != acc.astype(bool))).any()
        assert (np.abs(X1[sel] - Xs)[ok] / np.array(sysm.box)).max() <= 1e-5
        assert np.array_equal(h.get_density(), orc.density(X1))


def _run(system, steps, **opts):
    with soma.Handle(system, **opts) as h:
        h.mc_steps(steps)
        pos, img, step = h.get_state()
        return pos, img, h.get_density(), h.accepted(), step


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


def test_smart_launch_shape_graph_and_reorder_invariance():
    s = soma.System(**SMALL)
    ref = _run(s, 30, ctas_per_sm=2, graph_steps=0, sort_interval=0)
    for opts in (dict(ctas_per_sm=1), dict(hist_mode=soma.SOMA_HIST_SEPARATE), dict(graph_steps=16),
                 dict(graph_steps=7, sort_interval=5)):
        _same(ref, _run(s, 30, **{**dict(graph_steps=0, sort_interval=0), **opts}))


def test_mixed_move_kinds_batched_equal_plain():
    systems = [soma.System(**{**SMALL, "seed": 11 + i, "system_id": i, "move": m})
               for i, m in enumerate((soma.SOMA_MOVE_UNIFORM, SMART, SMART, soma.SOMA_MOVE_UNIFORM))]
    with soma.Handle(systems) as hb:
        hb.mc_steps(20)
        batched = [(hb.get_state(i)[0], hb.get_density(i), hb.accepted(i)) for i in range(len(systems))]
    for i, s in enumerate(systems):
        with soma.Handle(s) as h:
            h.mc_steps(20)
            _same(batched[i], (h.get_state()[0], h.get_density(), h.accepted()))


def test_batch64_smart_full_size_equals_solo_runs():
    """The 64-system batch with force-biased moves (the batch kernel whose
    system index is warp-uniform): after 3 steps the largest, the densest
    and the smallest systems equal the same systems stepped alone."""
    specs = workloads.batch64()
    systems = [soma.System(**{**{k: v for k, v in d.items() if k != "f_A"}, "move": SMART}) for d in specs]
    beads = [x.n_beads for x in systems]
    dens = [x.n_beads / x.n_cells for x in systems]
    picks = sorted({int(np.argmax(beads)), int(np.argmax(dens)), int(np.argmin(beads))})
    with soma.Handle(systems, graph_steps=0) as hb:
        hb.mc_steps(3)
        batched = {i: (hb.get_state(i)[0], hb.get_density(i), hb.accepted(i)) for i in picks}
    for i in picks:
        with soma.Handle(systems[i], graph_steps=0) as h:
            h.mc_steps(3)
            _same(batched[i], (h.get_state()[0], h.get_density(), h.accepted()))


def test_smart_ideal_chains_keep_gaussian_statistics():
    """chiN = kappaN = 0: the harmonic chain's Boltzmann law is stationary
    under the force-biased moves, so <b^2>(N-1) and <R_e^2> stay 1."""
    s = soma.System(n_poly=32768, N=32, n_A=16, box=(8.0, 8.0, 8.0), grid=(32, 32, 32), chiN=0.0, kappaN=0.0,
                    seed=21, move=SMART)
    with soma.Handle(s) as h:
        re2 = []
        for _ in range(20):
            h.mc_steps(25)
            re2.append(h.observables()["Re2"])
        X = h.unwrapped().reshape(s.n_poly, s.N, 3)
    b2 = (np.diff(X, axis=1) ** 2).sum(-1).mean() * (s.N - 1)
    assert abs(b2 - 1.0) < 5 * np.sqrt(2.0 / 3.0 / (s.n_poly * (s.N - 1)))
    assert abs(np.mean(re2) - 1.0) < 5 * np.sqrt(2.0 / 3.0 / s.n_poly)


def test_normal_deviates_match_the_exact_quantile():
    """Every one of the 2^24 arguments: the kernel's FP32 Phi^-1 against the
    exact quantile, and the mirror symmetry Phi^-1(1 - u) = -Phi^-1(u) bit
    for bit."""
    from scipy.special import ndtri
    m = np.arange(1 << 24, dtype=np.uint32)
    words = (m << 8) | (m & 0xFF)  # the low 8 bits of a word are not used
    xi = soma.soma_normal_deviates(words).astype(np.float64)
    ref = ndtri((m.astype(np.float64) + 0.5) * 2.0 ** -24)
    err = np.abs(xi - ref)
    print("max |xi - Phi^-1| =", err.max())
    assert err.max() <= 2e-6
    assert np.array_equal(xi[::-1], -xi)
