"""Coupling start-up on the GPU against the oracle (needs a GPU): the
umbrella restraint toward target volume fractions and the placement of
molecules from them (Sec. 3.2)."""
import numpy as np
import pytest

import gpu_util as G
from paper_2606_09356_b300 import soma, workloads

pytestmark = pytest.mark.gpu

LAMBDA = 40.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def _target(system, seed=3):
    """Lamellar target along x plus noise, float32 [2, n_c] (phi_A + phi_B = 1)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = system.grid
    x = (np.arange(nx) + 0.5) / nx
    pA = 0.5 + 0.4 * np.sin(2 * np.pi * 2 * x)[:, None, None] * np.ones((nx, ny, nz))
    pA = np.clip(pA + rng.normal(0, 0.05, size=pA.shape), 0.0, 1.0).reshape(-1)
    return np.stack([pA, 1.0 - pA]).astype(np.float32)


def _fields_bound(orc, counts, target, lam):
    _, _, rho = orc.params()
    phi = counts / rho
    d = orc.d
    scale = (abs(d.chiN) * phi.max(0) + abs(d.kappaN) * (phi.sum(0) + 1.0))[None, :] + lam * (phi + target)
    return 8 * np.finfo(np.float32).eps * (scale / d.N + 1e-30)


def test_umbrella_fields_match_oracle():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    tg = _target(s)
    with soma.Handle(s) as h:
        h.mc_steps(3)
        h.set_umbrella(tg, LAMBDA)
        for _ in range(3):
            counts = h.get_density()
            ref = orc.fields_umbrella(counts, tg.astype(np.float64), LAMBDA)
            assert np.all(np.abs(h.get_fields() - ref) <= _fields_bound(orc, counts, tg, LAMBDA))
            h.mc_steps(4)
        h.set_umbrella(None, 0.0)
        counts = h.get_density()
        assert np.allclose(h.get_fields(), orc.fields(counts), rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("kw", [
    dict(workloads.system_kwargs("melt_512x32")),
    dict(workloads.system_kwargs("melt_512x32"), move=soma.SOMA_MOVE_SMART),
    dict(n_poly=37, N=7, n_A=3, box=(4.0, 4.5, 5.0), grid=(16, 18, 20), chiN=15.0, kappaN=40.0, seed=7),
    dict(n_poly=40, N=80, n_A=30, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=25.0, kappaN=50.0, seed=7),  # generic
])
def test_umbrella_step_parity(kw):
    s = soma.System(**kw)
    orc = G.oracle_for(s)
    tg = _target(s)
    band = 1e-4 if s.move == soma.SOMA_MOVE_SMART else None
    with soma.Handle(s, graph_steps=0) as h:
        h.mc_steps(2)
        h.set_umbrella(tg, LAMBDA)
        for _ in range(4):
            X0, _ = G.unwrapped(h)
            w = orc.fields_umbrella(orc.density(X0), tg.astype(np.float64), LAMBDA)
            st = G.compare_step(h, band=band, w=w)
            assert abs(st["acc_gpu"] - st["acc_orc"]) <= st["suspect"]


def _run(systems, steps, umbrella, **opts):
    with soma.Handle(systems, **opts) as h:
        for i, tg in umbrella.items():
            h.set_umbrella(tg, LAMBDA, sys=i)
        h.mc_steps(steps)
        return [(h.get_state(i)[0], h.get_density(i), h.accepted(i)) for i in range(len(systems))]


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


def test_umbrella_invariant_to_graphs_and_batching():
    base = dict(n_poly=777, N=32, n_A=16, box=(4.0, 4.0, 5.0), grid=(16, 16, 20), chiN=20.0, kappaN=50.0)
    systems = [soma.System(**base, seed=40 + i, system_id=i) for i in range(3)]
    tg = _target(systems[1])
    ref = [_run([s], 24, {0: tg} if i == 1 else {}, graph_steps=0)[0] for i, s in enumerate(systems)]
    _same(ref[1], _run([systems[1]], 24, {0: tg}, graph_steps=8, sort_interval=5)[0])
    batched = _run(systems, 24, {1: tg})
    for a, b in zip(ref, batched):
        _same(a, b)


def test_umbrella_pulls_composition_toward_target():
    s = soma.System(**workloads.system_kwargs("melt_512x32"), move=soma.SOMA_MOVE_UNIFORM)
    tg = _target(s)
    _, _, rho = G.oracle_for(s).params()

    def distance(lam):
        with soma.Handle(s) as h:
            if lam:
                h.set_umbrella(tg, lam)
            h.mc_steps(300)
            phi = h.get_density() / rho
        return float(np.abs(phi - tg).mean())

    free, held = distance(0.0), distance(200.0)
    assert held < 0.8 * free


def test_place_matches_oracle():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    tg = _target(s, seed=8)
    ref = orc.place(tg)
    with soma.Handle(s) as h:
        h.mc_steps(5)
        h.place(tg)
        X, step = G.unwrapped(h)
        assert step == 5
        assert np.abs(X - ref).max() <= 1e-5 * max(s.box)
        assert np.array_equal(h.get_density(), orc.density(X))
        h.mc_steps(3)  # steps on from the placed state
        assert h.observables()["step"] == 8


def test_place_rejects_targets_without_weight_and_keeps_state():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    tg = np.zeros((2, s.n_cells), np.float32)
    tg[1] = 1.0  # bead 0 is type A: no weight
    with soma.Handle(s) as h:
        h.mc_steps(2)
        before = h.get_state()[0]
        with pytest.raises(soma.SomaError) as e:
            h.place(tg)
        assert e.value.code == soma.SOMA_EINVAL
        assert np.array_equal(h.get_state()[0], before)
        h.mc_steps(1)


def test_place_then_umbrella_reproduces_target():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    tg = _target(s, seed=9)
    _, _, rho = G.oracle_for(s).params()
    with soma.Handle(s) as h:
        h.place(tg)
        placed = h.get_density() / rho
        h.set_umbrella(tg, 100.0)
        h.mc_steps(200)
        held = h.get_density() / rho
    # correlation of the A profile with the target along x
    def corr(phi):
        a = phi[0].reshape(s.grid).mean(axis=(1, 2))
        b = tg[0].reshape(s.grid).mean(axis=(1, 2))
        return float(np.corrcoef(a, b)[0, 1])
    assert corr(placed) > 0.5
    assert corr(held) > 0.9


def test_place_in_a_multi_system_handle_equals_single():
    base = dict(n_poly=300, N=16, n_A=8, box=(4.0, 4.0, 4.0), grid=(16, 16, 16), chiN=20.0, kappaN=50.0)
    systems = [soma.System(**base, seed=70 + i, system_id=i) for i in range(3)]
    tg = _target(systems[1], seed=12)
    with soma.Handle(systems) as hb:
        hb.mc_steps(4)
        others = [hb.get_state(i)[0] for i in (0, 2)]
        hb.place(tg, sys=1)
        placed = hb.get_state(1)[0]
        assert all(np.array_equal(a, hb.get_state(i)[0]) for a, i in zip(others, (0, 2)))
        hb.mc_steps(5)
        after = [hb.get_state(i)[0] for i in range(3)]
    with soma.Handle(systems[1]) as h:
        h.mc_steps(4)
        h.place(tg)
        assert np.array_equal(h.get_state()[0], placed)
        h.mc_steps(5)
        assert np.array_equal(h.get_state()[0], after[1])


def test_umbrella_switched_on_keeps_supplied_fields_for_the_next_step():
    """Fields supplied by soma_set_density for the next step stay as supplied
    when the restraint is switched on afterwards; the restraint enters the
    fields built after that step."""
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    orc = G.oracle_for(s)
    tg = _target(s, seed=14)
    rng = np.random.default_rng(2)
    phi = rng.uniform(0.0, 1.0, size=(2, s.n_cells)).astype(np.float32)
    with soma.Handle(s, graph_steps=0) as h:
        h.mc_steps(2)
        h.set_density(phi)
        supplied = h.get_fields()
        h.set_umbrella(tg, LAMBDA)
        assert np.array_equal(h.get_fields(), supplied)
        h.mc_steps(1)  # moves against the supplied fields
        counts = h.get_density()
        ref = orc.fields_umbrella(counts, tg.astype(np.float64), LAMBDA)
        assert np.all(np.abs(h.get_fields() - ref) <= _fields_bound(orc, counts, tg, LAMBDA))


def test_device_tensors_as_targets_match_host_arrays():
    """Targets given as CUDA tensors (SOMA_DEVICE) place and restrain exactly
    as the same values given as host arrays."""
    import torch
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    tg = _target(s, seed=21)
    runs = []
    for on_device in (False, True):
        t = torch.from_numpy(tg).cuda() if on_device else tg
        with soma.Handle(s, graph_steps=0) as h:
            h.place(t)
            h.set_umbrella(t, 30.0)
            h.mc_steps(3)
            runs.append((h.get_state()[0], h.get_density(), h.get_fields()))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    with soma.Handle(s, graph_steps=0) as h:  # a tensor of another type is refused before the C call
        with pytest.raises(ValueError):
            h.place(torch.from_numpy(tg).double().cuda())


def test_place_on_the_131072_chain_melt_matches_oracle():
    """Placement on a 128^3 grid (2,097,152 cells: the running weight sums
    span many scan tiles) against the oracle, every chain."""
    s = soma.System(**workloads.system_kwargs("melt_131072x32"))
    orc = G.oracle_for(s)
    tg = _target(s, seed=13)
    ref = orc.place(tg)
    with soma.Handle(s) as h:
        h.place(tg)
        X, _ = G.unwrapped(h)
        assert np.abs(X - ref).max() <= 1e-5 * max(s.box)
        assert np.array_equal(h.get_density(), orc.density(X))
