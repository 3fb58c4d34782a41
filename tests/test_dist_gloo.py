"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each an independent
replica; the job's time is the max over ranks and its work the sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench.dist_env()
    t, units = bench.dist_reduce(1.0 + rank, 100 * (rank + 1))
    # replicas draw from disjoint Philox streams: counter word 2 is the replica id
    import oracle as O
    a = O.philox4x32_10([5, 0, rank, 0], [7, 0]).tolist()
    gathered = [None] * world
    dist.all_gather_object(gathered, a)
    out[rank] = (ws, r, t, units, gathered[0] != gathered[1])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ws, r, t, units, distinct = out[rank]
        assert ws == world and r == rank
        assert t == 2.0 and units == 300.0
        assert distinct


def test_single_process_reduce_is_identity():
    import bench
    assert bench.dist_reduce(3.5, 7) == (3.5, 7.0)


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import hmc_synth as S
    from paper_1009_0457_gb300.shard import balance_replicas
    sites = [int(np.prod(sp["shape"])) for sp in S.ensemble_specs()]
    mine = balance_replicas(sites, world)[rank]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    loads = [None] * world
    dist.all_gather_object(loads, sum(sites[r] for r in mine))
    out[rank] = (parts, loads, max(sites), len(sites))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ensemble_replicas_shared_out_over_gloo_ranks(world):
    """Every rank computes its own share of the 64-replica ensemble; gathered, the shares
    are disjoint, cover every replica once, agree between ranks and differ in sites by
    at most one replica's."""
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    parts, loads, biggest, n = out[0]
    for r in range(world):
        assert out[r][0] == parts and out[r][1] == loads
    flat = sorted(x for p in parts for x in p)
    assert flat == list(range(n))
    assert max(loads) - min(loads) <= biggest


def test_balance_replicas_single_rank_and_empty():
    from paper_1009_0457_gb300.shard import balance_replicas
    assert balance_replicas([5, 3, 9], 1) == [[0, 1, 2]]
    assert balance_replicas([4, 4], 3) == [[0], [1], []]
    with pytest.raises(ValueError):
        balance_replicas([1], 0)
