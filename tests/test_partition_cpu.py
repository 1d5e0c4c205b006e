"""The chain partition's protocol on CPU (no GPU): two gloo ranks each step
their own range of one system's chains against fields from the counts summed
over both ranks, and reproduce the whole system's trajectory bit for bit.
The oracle stands in for the library on each rank; what is tested is the
bookkeeping the library and its callers share: the contiguous chain ranges,
random numbers by logical chain id, partial counts, the all-reduce (sum),
the fields of the whole system's density, and the exchange before the first
step."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_09356_b300 import partition

SYSTEM = dict(n_poly=96, N=12, n_A=5, box=(2.0, 2.0, 2.0), grid=(8, 8, 8), chiN=20.0, kappaN=50.0, seed=7)
STEPS = 6


def _oracle(n_poly, move=0):
    from oracle import Oracle
    s = SYSTEM
    return Oracle(n_poly, s["N"], s["n_A"], s["box"], s["grid"], s["chiN"], s["kappaN"], seed=s["seed"], move=move)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, move, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = partition.chain_range(SYSTEM["n_poly"], rank, world)
    whole = _oracle(SYSTEM["n_poly"], move)  # fields (rho_bar of the whole system) and the initial chains
    local = _oracle(e - b, move)             # the partial histogram of this rank's chains
    ids = np.arange(b, e, dtype=np.uint32)
    X = np.ascontiguousarray(whole.init().reshape(SYSTEM["n_poly"], -1)[b:e].reshape(-1, 3))
    reduce = partition.all_reduce_sum()

    def exchanged_counts():
        t = torch.from_numpy(local.density(X).astype(np.int32))
        reduce(t)
        return t.numpy().astype(np.uint32)

    counts = exchanged_counts()  # before the first step
    acc = 0
    for t in range(STEPS):
        n, _, _, _ = whole.mc_step_chains(X, ids, whole.fields(counts), t)
        acc += n
        counts = exchanged_counts()
    out[rank] = (b, e, X.copy(), counts.copy(), acc)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("move", [0, 1], ids=["uniform", "smart"])
def test_two_gloo_partitions_reproduce_the_whole_system(move):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, 2, port, move, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    whole = _oracle(SYSTEM["n_poly"], move)
    X = whole.init()
    total = whole.run(X, 0, STEPS)["accepted"]
    (b0, e0, X0, c0, a0), (b1, e1, X1, c1, a1) = res[0], res[1]
    assert (b0, e0, b1, e1) == (0, 48, 48, 96)
    assert np.array_equal(np.concatenate([X0, X1]), X)  # bit for bit
    assert np.array_equal(c0, c1) and np.array_equal(c0, whole.density(X))
    assert a0 + a1 == total


def test_chain_ranges_cover_the_system_once():
    for n, w in ((512, 1), (512, 3), (7, 7), (131072, 8), (1048577, 4)):
        r = [partition.chain_range(n, k, w) for k in range(w)]
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(r[k][1] == r[k + 1][0] for k in range(w - 1))
        sizes = [e - b for b, e in r]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        partition.chain_range(3, 0, 4)
