"""Chain partitions on one GPU: the partitions of a system, each a handle of
its own chains, with their counts summed after every step (the exchange the
partitions of a multi-GPU run make by an all-reduce), reproduce the whole
system's handle bit for bit: positions, images, counts, acceptance, molecule
types and conversions."""
import numpy as np
import pytest
import torch

import gpu_util as G
from paper_2606_09356_b300 import partition, soma, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    G.lib()


def _run(system, ranges, steps, conversion=None, umbrella=None, **opts):
    st = torch.cuda.Stream()  # the steps and the exchanges share one stream
    whole = soma.Handle(system, **opts)
    parts = [soma.Handle(system, partition=r, **opts) for r in ranges]
    for h in [whole] + parts:
        if conversion:
            h.set_conversion(*conversion)
        if umbrella is not None:
            h.set_umbrella(*umbrella)
    torch.cuda.synchronize()
    partition.sum_on_one_device(parts, st)  # the exchange after creation
    for _ in range(steps):
        whole.mc_steps(1, stream=st.cuda_stream)
        for h in parts:
            h.mc_steps(1, stream=st.cuda_stream)
        partition.sum_on_one_device(parts, st)
    torch.cuda.synchronize()
    return whole, parts


def _check_same(system, whole, parts, conversion=False):
    pos, img, step = whole.get_state()
    pp = [h.get_state() for h in parts]
    assert np.array_equal(np.concatenate([p[0] for p in pp]), pos)
    assert np.array_equal(np.concatenate([p[1] for p in pp]), img)
    assert all(p[2] == step for p in pp)
    dens = whole.get_density()
    for h in parts:
        assert np.array_equal(h.get_density(), dens)
    assert sum(h.accepted() for h in parts) == whole.accepted()
    ow, op = whole.observables(), parts[0].observables()
    # from the exchanged counts and the whole system's rho_bar (an FP64 sum
    # over cells by atomics: equal up to its order of rounding)
    assert abs(ow["Enb"] - op["Enb"]) <= 1e-12 * abs(ow["Enb"])
    if conversion:
        assert np.array_equal(np.concatenate([h.chain_types() for h in parts]), whole.chain_types())
        assert np.array_equal(sum(h.conversions() for h in parts), whole.conversions())


@pytest.mark.parametrize("move,wall", [(soma.SOMA_MOVE_UNIFORM, 0), (soma.SOMA_MOVE_SMART, 0),
                                       (soma.SOMA_MOVE_UNIFORM, 1)], ids=["uniform", "smart", "walls"])
def test_partitions_reproduce_the_whole_system(move, wall):
    s = soma.System(**{**workloads.system_kwargs("melt_512x32"), "move": move, "wall_z": wall})
    # unequal ranges, one of a single chain; reorders inside the run
    whole, parts = _run(s, [(0, 170), (170, 171), (171, 512)], steps=12, sort_interval=5, graph_steps=0)
    _check_same(s, whole, parts)


@pytest.mark.parametrize("warps", [12, 24])
def test_partitions_at_every_block_shape(warps):
    """Partitions whose move kernel runs 12 or 24 consumer warps per CTA (so
    a partition's tiles hold 24 or 48 chains and its last tile is ragged)
    reproduce the whole system stepped at 8."""
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    st = torch.cuda.Stream()
    whole = soma.Handle(s, graph_steps=0, sort_interval=5, move_warps=8)
    parts = [soma.Handle(s, partition=r, graph_steps=0, sort_interval=5, move_warps=warps)
             for r in [(0, 101), (101, 389), (389, 512)]]
    assert all(h.info()["move_warps"] == warps for h in parts)
    torch.cuda.synchronize()
    partition.sum_on_one_device(parts, st)
    for _ in range(12):
        whole.mc_steps(1, stream=st.cuda_stream)
        for h in parts:
            h.mc_steps(1, stream=st.cuda_stream)
        partition.sum_on_one_device(parts, st)
    torch.cuda.synchronize()
    _check_same(s, whole, parts)


def test_partitions_with_conversion_and_odd_chains():
    s = soma.System(n_poly=301, N=7, n_A=3, box=(4.0, 4.0, 4.5), grid=(16, 16, 18), chiN=18.0, kappaN=40.0,
                    seed=5, wall_z=1)
    conv = (1, 1.0, 1.0, (0.2, 0.1, 0.15, 0.05))
    whole, parts = _run(s, [partition.chain_range(301, k, 4) for k in range(4)], steps=10, conversion=conv)
    _check_same(s, whole, parts, conversion=True)


def test_partitions_with_umbrella_restraint():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    x = (np.arange(16) + 0.5) / 16
    pA = np.repeat(0.5 + 0.4 * np.sin(2 * np.pi * x), 256)
    target = np.stack([pA, 1.0 - pA]).astype(np.float32)
    whole, parts = _run(s, [(0, 256), (256, 512)], steps=8, umbrella=(target, 30.0))
    _check_same(s, whole, parts)


def test_partitions_place_as_the_whole_system():
    """Placement from target fields draws per logical chain, so partitions
    place exactly the whole system's chains; steps after it stay equal."""
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    x = (np.arange(16) + 0.5) / 16
    pA = np.clip(np.repeat(0.5 + 0.45 * np.sin(2 * np.pi * x), 256), 0.0, 1.0)
    target = np.stack([pA, 1.0 - pA]).astype(np.float32)
    st = torch.cuda.Stream()
    whole = soma.Handle(s)
    parts = [soma.Handle(s, partition=r) for r in [(0, 200), (200, 512)]]
    for h in [whole] + parts:
        h.place(target)
    torch.cuda.synchronize()
    partition.sum_on_one_device(parts, st)  # placement re-bins: exchange
    for _ in range(5):
        whole.mc_steps(1, stream=st.cuda_stream)
        for h in parts:
            h.mc_steps(1, stream=st.cuda_stream)
        partition.sum_on_one_device(parts, st)
    torch.cuda.synchronize()
    _check_same(s, whole, parts)


def test_two_partitions_of_the_131072_chain_melt():
    """The melt of 131,072 chains of 32 beads (grid 128^3) in two halves, in
    the benchmark's launch configuration (persistent move kernel at full
    occupancy, fused histogram)."""
    s = soma.System(**workloads.system_kwargs("melt_131072x32"))
    whole, parts = _run(s, [(0, 65536), (65536, 131072)], steps=4, graph_steps=0)
    _check_same(s, whole, parts)


def test_steps_on_the_default_stream_are_refused():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s, partition=(0, 512)) as h:
        with pytest.raises(ValueError):
            partition.step(h, lambda t: None, torch.cuda.default_stream())


def test_exchange_buffer_is_the_counts_of_the_next_step():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    with soma.Handle(s) as h:
        h.mc_steps(3)
        h.sync()
        t = partition.counts_tensor(h)
        inter = t.cpu().numpy().astype(np.uint32).reshape(-1, 2)
        assert np.array_equal(inter.T, h.get_density())


def test_partition_arguments():
    s = soma.System(**workloads.system_kwargs("melt_512x32"))
    for r in ((0, 0), (-1, 5), (10, 5), (0, 513)):
        with pytest.raises(soma.SomaError) as e:
            soma.Handle(s, partition=r)
        assert e.value.code == soma.SOMA_EINVAL
    with pytest.raises(soma.SomaError) as e:
        soma.Handle(s, partition=(0, 256), autotune=1)
    assert e.value.code == soma.SOMA_EINVAL
    long_chains = soma.System(n_poly=64, N=80, n_A=40, box=(4.0, 4.0, 4.0), grid=(8, 8, 8), chiN=0.0, kappaN=0.0)
    with pytest.raises(soma.SomaError) as e:
        soma.Handle(long_chains, partition=(0, 32))
    assert e.value.code == soma.SOMA_ENOTSUP
    with soma.Handle(s, partition=(0, 256)) as h:
        with pytest.raises(soma.SomaError) as e:
            h.mc_steps(2)  # one step per call: the exchange follows every step
        assert e.value.code == soma.SOMA_EINVAL
        with pytest.raises(soma.SomaError) as e:
            h.autotune()
        assert e.value.code == soma.SOMA_ENOTSUP
        assert h.info()["rho_bar"] == 4.0 and h.info()["n_beads"] == 256 * 32
        assert partition.counts_tensor(h).device == torch.device(f"cuda:{h.device}")
