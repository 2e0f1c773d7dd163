"""Multi-GPU path of the benchmark is replicas only (independent realisations,
no data exchange): two gloo ranks on CPU check the seed partition, the
max-over-ranks time and the whole-job throughput accounting."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank, 3)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    slow = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, gathered, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_partition_seeds_and_take_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slow in res:
        flat = [s for part in gathered for s in part]
        assert len(set(flat)) == len(flat) == 6          # disjoint realisations
        assert slow == 15.0                               # max over ranks
    import bench
    one = bench.aggregate_throughput(1, 16, 512, 5, 1000.0)
    two = bench.aggregate_throughput(2, 16, 512, 5, 1000.0)
    assert abs(two - 2 * one) < 1e-9 * one              # weak scaling: work grows with ranks
