"""Properties that hold bit for bit on the GPU (needs a GPU): the trajectory
does not depend on launch shape, histogram strategy, graph capture, chain
reorders, batching with other systems, or a checkpoint round trip."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu

SMALL = dict(n_poly=777, N=32, n_A=16, box=(4.0, 4.0, 5.0), grid=(16, 16, 20), chiN=20.0, kappaN=50.0, seed=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


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


def test_launch_shape_histogram_graph_and_reorder_invariance():
    s = soma.System(**SMALL)
    ref = _run(s, 40, ctas_per_sm=2, hist_mode=soma.SOMA_HIST_FUSED, graph_steps=0, sort_interval=0)
    for opts in (dict(ctas_per_sm=1), dict(ctas_per_sm=0), dict(ctas_per_sm=2), dict(hist_mode=soma.SOMA_HIST_SEPARATE),
                 dict(graph_steps=16), dict(graph_steps=7, sort_interval=5), dict(sort_interval=1),
                 dict(autotune=1)):
        _same(ref, _run(s, 40, **{**dict(graph_steps=0, sort_interval=0), **opts}))


@pytest.mark.parametrize("kw", [dict(), dict(move=soma.SOMA_MOVE_SMART), dict(wall_z=1), dict(N=7, n_A=3),
                                dict(N=64, n_A=19), dict(N=1, n_A=1, A=0.3)],
                         ids=["uniform", "smart", "walls", "odd_N", "N64", "monomers"])
def test_block_shape_invariance(kw):
    """The move kernel with 8, 12 or 24 consumer warps per CTA (tiles of 8,
    12 or 24 warps' chains; the 24-warp ring in dynamic shared memory) steps
    the same trajectory, at every resident-CTA count."""
    s = soma.System(**{**SMALL, **kw})
    ref = _run(s, 30, move_warps=8, graph_steps=0, sort_interval=7)
    for w in (12, 24):
        for opts in (dict(move_warps=w), dict(move_warps=w, ctas_per_sm=1), dict(move_warps=w, graph_steps=5)):
            _same(ref, _run(s, 30, **{**dict(graph_steps=0, sort_interval=7), **opts}))
        with soma.Handle(s, move_warps=w) as h:
            assert h.info()["move_warps"] == w
        with soma.Handle(s, move_warps=w, autotune=1) as h:
            h.mc_steps(1)
            assert h.info()["move_warps"] == w  # fixed by the option, the autotuner keeps it
    with soma.Handle(s, move_warps=24) as h:
        assert h.info()["ctas_per_sm"] == 1  # 800 threads of 72 registers: one CTA per SM
    for bad in (10, 16, 32):
        with pytest.raises(soma.SomaError) as e:
            soma.Handle(s, move_warps=bad)
        assert e.value.code == soma.SOMA_EINVAL


def test_the_131072_chain_melt_at_every_block_shape():
    s = soma.System(**workloads.system_kwargs("melt_131072x32"))
    ref = _run(s, 6, move_warps=8, graph_steps=0)
    for w in (12, 24):
        _same(ref, _run(s, 6, move_warps=w, graph_steps=0))


def test_the_1048576_chain_melt_at_24_and_8_warps():
    """melt_1048576x64 at full size (67 M beads, 24 chains per 24-warp tile,
    43,691 tiles over one CTA per SM) steps the same trajectory at 24 and
    at 8 consumer warps per CTA."""
    s = soma.System(**workloads.system_kwargs("melt_1048576x64"))
    _same(_run(s, 2, move_warps=8, graph_steps=0), _run(s, 2, move_warps=24, graph_steps=0))


def test_tuned_sort_interval_keeps_the_trajectory():
    s = soma.System(**SMALL)
    ref = _run(s, 40, graph_steps=0, sort_interval=0)
    with soma.Handle(s, autotune=1, sort_interval=-1, graph_steps=0) as h:
        h.mc_steps(40)
        pos, img, step = h.get_state()
        k = h.info()["sort_interval"]
        got = (pos, img, h.get_density(), h.accepted(), step)
    assert k in (32, 64, 128, 256, 512, 1024)
    _same(ref, got)


def test_batched_equals_plain():
    specs = workloads.batch64()[:5]
    systems = [soma.System(**{k: v for k, v in d.items() if k != "f_A"}) for d in specs]
    # shrink the chain counts to keep the test short
    for s in systems:
        s.n_poly = min(s.n_poly, 3000)
    with soma.Handle(systems) as hb:
        hb.mc_steps(25)
        batched = [(hb.get_state(i)[0], hb.get_state(i)[1], hb.get_density(i), hb.accepted(i)) for i in range(5)]
    for i, s in enumerate(systems):
        with soma.Handle(s) as h:
            h.mc_steps(25)
            solo = (h.get_state()[0], h.get_state()[1], h.get_density(), h.accepted())
        _same(batched[i], solo)


def test_checkpoint_resume_is_bit_exact():
    s = soma.System(**SMALL)
    ref = _run(s, 30)
    with soma.Handle(s) as h:
        h.mc_steps(13)
        pos, img, step = h.get_state()
        acc13 = h.accepted()
    with soma.Handle(soma.System(**{**SMALL, "seed": 3})) as h2:
        h2.set_state(pos, img, step)
        h2.mc_steps(17)
        p2, i2, st2 = h2.get_state()
        assert st2 == 30
        assert np.array_equal(p2, ref[0]) and np.array_equal(i2, ref[1])
        assert np.array_equal(h2.get_density(), ref[2])
        assert h2.accepted() + acc13 == ref[3]


def test_reorder_keeps_logical_state():
    s = soma.System(**SMALL)
    with soma.Handle(s, sort_interval=0) as h:
        h.mc_steps(10)
        a = h.get_state()
        h.reorder()
        b = h.get_state()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_persistent_grid_invariance_full_size():
    """melt_131072x32 at full size: with 1, 2 and 3 resident CTAs per SM every CTA
    cycles its stage ring many times per step; the trajectory must not
    depend on how the tiles are spread over the persistent CTAs."""
    s = soma.System(**workloads.system_kwargs("melt_131072x32"))
    ref = None
    for c in (3, 1, 2):
        with soma.Handle(s, ctas_per_sm=c, graph_steps=0, sort_interval=0) as h:
            h.mc_steps(6)
            st = (h.get_state()[0], h.get_density(), h.accepted())
        if ref is None:
            ref = st
        else:
            _same(ref, st)


@pytest.mark.parametrize("variant", ["uniform", "smart", "walls"])
def test_long_run_grid_invariance_full_size(variant):
    """A stage-ring race would show up only now and then: melt_131072x32 at full
    size for many steps, CUDA graphs and chain reorders on, with 3 and 1
    resident CTAs per SM and with the 24-warp shape (its ring in dynamic
    shared memory), must stay bit-identical throughout."""
    kw = dict(workloads.system_kwargs("melt_131072x32"))
    if variant == "smart":
        kw["move"] = soma.SOMA_MOVE_SMART
    if variant == "walls":
        kw["wall_z"] = 1
    s = soma.System(**kw)
    steps = 1000 if variant == "uniform" else 300
    ref = None
    for opts in (dict(ctas_per_sm=3), dict(ctas_per_sm=1), dict(move_warps=24)):
        with soma.Handle(s, graph_steps=50, sort_interval=97, **opts) as h:
            h.mc_steps(steps)
            st = (h.get_state()[0], h.get_density(), h.accepted())
        if ref is None:
            ref = st
        else:
            _same(ref, st)


def test_long_run_batch64_grid_invariance():
    """The batch kernel's stage ring over 200 steps of the 64-system batch:
    default and one resident CTA per SM give the same trajectories."""
    specs = workloads.batch64()
    systems = [soma.System(**{k: v for k, v in d.items() if k != "f_A"}) for d in specs]
    ref = None
    for c in (0, 1):
        with soma.Handle(systems, ctas_per_sm=c, graph_steps=50) as hb:
            hb.mc_steps(200)
            st = [(hb.get_state(i)[0], hb.get_density(i), hb.accepted(i)) for i in range(len(systems))]
        if ref is None:
            ref = st
        else:
            for a, b in zip(ref, st):
                _same(a, b)


def test_batch64_full_size_equals_solo_runs():
    """The 64-system batch at full size, launched as bench.py times it (one
    handle, CUDA graphs): after 5 steps every system is bit-identical to the
    same system stepped alone."""
    specs = workloads.batch64()
    systems = [soma.System(**{k: v for k, v in d.items() if k != "f_A"}) for d in specs]
    with soma.Handle(systems, graph_steps=5) as hb:
        hb.mc_steps(5)
        batched = [(hb.get_state(i)[0], hb.get_density(i), hb.accepted(i)) for i in range(len(systems))]
    for i, s in enumerate(systems):
        with soma.Handle(s, graph_steps=0) as h:
            h.mc_steps(5)
            _same(batched[i], (h.get_state()[0], h.get_density(), h.accepted()))
