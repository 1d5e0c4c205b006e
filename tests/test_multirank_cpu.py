"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own replica
system (no data-path collective), whole-job throughput = moves of all ranks
over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    kw = bench.rank_system_kwargs("melt_131072x32", rank)
    # rank r pretends its timed region took 10 * (r + 1) ms for 1000 * (r + 1) moves
    max_ms, moves, value = bench.aggregate(10.0 * (rank + 1), 1000.0 * (rank + 1), dist, device="cpu")
    out[rank] = (kw["system_id"], kw["n_poly"], max_ms, moves, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_own_replicas():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == 0 and res[1][0] == 1          # distinct random streams
    assert res[0][1] == res[1][1] == 131072           # same workload shape (weak scaling)
    for r in range(2):
        assert res[r][2] == pytest.approx(20.0)        # slowest rank's time
        assert res[r][3] == pytest.approx(3000.0)      # all ranks' moves
        assert res[r][4] == pytest.approx(3000.0 / 0.020)


def test_single_rank_aggregate():
    import bench
    assert bench.aggregate(4.0, 8000.0) == (4.0, 8000.0, 2e6)
