"""Boundary-zone molecule-type conversion (Sec. 3.2) on the GPU against the
oracle (needs a GPU): every step's conversions bit for bit (types and
counts per zone and direction), the moves with the new bead types, the
counts with the new types; trajectories independent of graphs, reorders,
launch shapes and batching; a checkpoint with types resumes bit for bit."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


# (system, n_A_alt, bottom width, top width, p = (bottom 0->1, 1->0, top 0->1, 1->0))
CASES = {
    "walls_diblock": (dict(n_poly=512, N=32, n_A=16, box=(4.0, 4.0, 4.0), grid=(16, 16, 16), chiN=20.0, kappaN=50.0,
                           wall_z=1), 4, 1.0, 0.75, (0.3, 0.1, 0.2, 0.4)),
    "periodic_smart": (dict(n_poly=300, N=24, n_A=9, box=(3.0, 3.3, 2.9), grid=(7, 11, 9), chiN=18.0, kappaN=45.0,
                            move=soma.SOMA_MOVE_SMART), 24, 0.5, 0.5, (0.5, 0.5, 0.5, 0.5)),
    "walls_beads": (dict(n_poly=4000, N=1, n_A=1, box=(2.0, 2.0, 3.0), grid=(4, 4, 6), chiN=0.0, kappaN=30.0,
                         A=0.2, wall_z=1), 0, 1.0, 1.0, (0.4, 0.2, 0.1, 0.3)),
    "odd_chains": (dict(n_poly=700, N=7, n_A=3, box=(4.0, 4.0, 4.0), grid=(8, 8, 8), chiN=25.0, kappaN=40.0,
                        wall_z=1), 5, 0.6, 0.9, (1.0, 0.0, 0.5, 0.5)),
}


def _setup(case):
    kw, n_alt, lo, hi, p = CASES[case]
    s = soma.System(**kw)
    orc = G.oracle_for(s)
    orc.set_conversion(n_alt, lo, hi, p)
    return s, orc, (n_alt, lo, hi, p)


@pytest.mark.parametrize("ctas", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_conversion_steps_like_the_oracle(case, ctas):
    s, orc, conv = _setup(case)
    band = 1e-4 if s.move == soma.SOMA_MOVE_SMART else None
    with soma.Handle(s, graph_steps=0, ctas_per_sm=ctas) as h:
        h.set_conversion(*conv)
        for _ in range(8):
            G.compare_step(h, orc=orc, band=band)
        total = h.conversions()
        assert total.sum() > 0
        t = h.chain_types()
        counts = h.get_density()
        n_alt = conv[0]
        assert counts[0].sum() == int((t == 0).sum()) * s.n_A + int((t == 1).sum()) * n_alt


def test_conversion_with_the_umbrella_on_steps_like_the_oracle():
    s, orc, conv = _setup("walls_diblock")
    rng = np.random.default_rng(5)
    tg = rng.uniform(0.2, 0.8, size=(2, s.n_cells)).astype(np.float32)
    lam = 40.0
    with soma.Handle(s, graph_steps=0) as h:
        h.set_conversion(*conv)
        h.set_umbrella(tg, lam)
        for _ in range(6):
            G.compare_step(h, orc=orc, fields=lambda o, c: o.fields_umbrella(c, tg.astype(np.float64), lam))


def _run(systems, steps, conv=None, **opts):
    with soma.Handle(systems, **opts) as h:
        for i, c in (conv or {}).items():
            h.set_conversion(*c, sys=i)
        h.mc_steps(steps)
        n = len(h.systems)
        return [(h.get_state(i)[0], h.get_density(i), h.chain_types(i), h.conversions(i), h.accepted(i))
                for i in range(n)]


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_zero_rates_leave_the_trajectory_unchanged():
    """Conversion on with zero rates (types honoured, nothing converts) is
    bit-identical to the plain step, whatever n_A_alt."""
    kw = CASES["walls_diblock"][0]
    s = soma.System(**kw)
    ref = _run(s, 12, graph_steps=0)[0]
    got = _run(s, 12, conv={0: (4, 1.0, 1.0, (0.0, 0.0, 0.0, 0.0))}, graph_steps=0)[0]
    for k in (0, 1, 4):
        assert np.array_equal(np.asarray(ref[k]), np.asarray(got[k]))
    assert not got[2].any() and not got[3].any()


def test_trajectory_independent_of_graphs_reorders_shapes_and_batching():
    systems = [soma.System(**CASES[c][0], seed=50 + i, system_id=i) for i, c in enumerate(sorted(CASES))]
    convs = {i: CASES[c][1:] for i, c in enumerate(sorted(CASES))}
    solo = [_run(s, 17, conv={0: convs[i]}, graph_steps=0, sort_interval=0)[0] for i, s in enumerate(systems)]
    for opts in (dict(graph_steps=5, sort_interval=4), dict(graph_steps=0, sort_interval=3, ctas_per_sm=1)):
        for i, s in enumerate(systems):
            _same(solo[i], _run(s, 17, conv={0: convs[i]}, **opts)[0])
    # a batch mixing converting and plain systems (one system without conversion)
    plain = soma.System(**dict(CASES["walls_diblock"][0], n_poly=333), seed=70, system_id=9)
    ref_plain = _run(plain, 17, graph_steps=0)[0]
    for opts in (dict(graph_steps=0), dict(graph_steps=5, sort_interval=6)):
        batched = _run(systems + [plain], 17, conv=convs, **opts)
        for i in range(len(systems)):
            _same(solo[i], batched[i])
        _same(ref_plain, batched[-1])


def test_checkpoint_with_types_resumes_bit_exact():
    s, _, conv = _setup("walls_diblock")
    with soma.Handle(s, graph_steps=0) as h:
        h.set_conversion(*conv)
        h.mc_steps(9)
        pos, img, step = h.get_state()
        types = h.chain_types()
        assert types.any()
        h.mc_steps(11)
        ref = (h.get_state()[0], h.get_density(), h.chain_types())
    with soma.Handle(s, graph_steps=4) as h2:
        h2.set_state(pos, img, step)
        h2.set_conversion(*conv)
        h2.set_chain_types(types)
        h2.mc_steps(11)
        _same(ref, (h2.get_state()[0], h2.get_density(), h2.chain_types()))


def test_switching_conversion_off_restores_the_own_molecules():
    s, _, conv = _setup("walls_beads")
    with soma.Handle(s, graph_steps=0) as h:
        h.set_conversion(*conv)
        h.mc_steps(5)
        assert h.chain_types().any()
        assert h.get_density()[0].sum() < s.n_poly
        h.set_conversion(-1)
        assert not h.chain_types().any()
        assert h.get_density()[0].sum() == s.n_poly  # rebuilt: every bead type A again
        h.mc_steps(2)
        assert h.get_density()[0].sum() == s.n_poly


def test_conversion_arguments_are_checked():
    s = soma.System(**CASES["walls_diblock"][0])
    with soma.Handle(s, graph_steps=0) as h:
        bad = [(33, 1.0, 1.0, (0.1,) * 4), (4, -0.1, 1.0, (0.1,) * 4), (4, 3.0, 1.5, (0.1,) * 4),
               (4, 1.0, 1.0, (0.1, 1.5, 0.1, 0.1)), (4, 1.0, float("nan"), (0.1,) * 4)]
        for args in bad:
            with pytest.raises(soma.SomaError) as e:
                h.set_conversion(*args)
            assert e.value.code == soma.SOMA_EINVAL
        with pytest.raises(soma.SomaError) as e:  # types need conversion on
            h.set_chain_types(np.zeros(s.n_poly, np.uint8))
        assert e.value.code == soma.SOMA_EINVAL
        h.set_conversion(4, 1.0, 1.0, (0.1,) * 4)
        with pytest.raises(soma.SomaError) as e:
            h.set_chain_types(np.full(s.n_poly, 2, np.uint8))
        assert e.value.code == soma.SOMA_EINVAL
        h.mc_steps(1)  # the handle stays usable
    long_chains = soma.System(n_poly=50, N=80, n_A=40, box=(4.0, 4.0, 4.0), grid=(8, 8, 8), chiN=1.0, kappaN=1.0)
    with soma.Handle(long_chains) as h:
        with pytest.raises(soma.SomaError) as e:
            h.set_conversion(10, 1.0, 1.0, (0.1,) * 4)
        assert e.value.code == soma.SOMA_ENOTSUP
    periodic = soma.System(**dict(CASES["walls_diblock"][0], wall_z=0))
    with soma.Handle(periodic, precision=soma.SOMA_PREC_FP64) as h:
        with pytest.raises(soma.SomaError) as e:
            h.set_conversion(4, 1.0, 1.0, (0.1,) * 4)
        assert e.value.code == soma.SOMA_ENOTSUP


def test_melt_131072x32_between_walls_with_conversion_full_size():
    """melt_131072x32 with walls and zones 2 R_e wide: one step at full size in the
    bench's launch configuration; every chain's type and the whole grid's
    counts bit for bit, a 2048-chain sample of the moves against the oracle."""
    s = soma.System(**dict(workloads.system_kwargs("melt_131072x32"), wall_z=1))
    orc = G.oracle_for(s)
    conv = (8, 2.0, 2.0, (0.05, 0.02, 0.03, 0.04))
    orc.set_conversion(*conv)
    k_b, _, _ = orc.params()
    band = G.band_for(s, k_b)
    rng = np.random.default_rng(19)
    ids = np.sort(rng.choice(s.n_poly, 2048, replace=False)).astype(np.uint32)
    N = s.N
    sel = (ids[:, None].astype(np.int64) * N + np.arange(N)[None, :]).reshape(-1)
    with soma.Handle(s, autotune=1, graph_steps=0, kernel_timing=1) as h:
        h.set_conversion(*conv)
        h.mc_steps(3)
        for _ in range(2):
            X0, step = G.unwrapped(h)
            orc.set_types(h.chain_types())
            counts = h.get_density()
            assert np.array_equal(counts, orc.density(X0))
            w = orc.fields(counts)
            c4 = orc.convert(X0, step)
            Xs = np.ascontiguousarray(X0[sel])
            _, acc, margin, face = orc.mc_step_chains(Xs, ids, w, step, n_threads=G.NTHREADS)
            c_before = h.conversions().astype(np.int64)
            h.mc_steps(1)
            assert np.array_equal(h.chain_types(), orc.types)
            assert np.array_equal(h.conversions().astype(np.int64) - c_before, c4)
            X1, _ = G.unwrapped(h)
            moved = np.any(X1[sel] != X0[sel], axis=1)
            face_tol = 8.0 * float(np.spacing(np.float32(max(s.box))))
            sus = ((np.abs(margin) < band) | (face < face_tol)).reshape(-1, N)
            spread = sus.copy()
            spread[:, 1:] |= sus[:, :-1]
            spread[:, :-1] |= sus[:, 1:]
            ok = ~spread.reshape(-1)
            assert not (ok & (moved != acc.astype(bool))).any()
            assert (np.abs(X1[sel] - Xs)[ok] / np.array(s.box)).max() <= 1e-5
            assert np.array_equal(h.get_density(), orc.density(X1))
