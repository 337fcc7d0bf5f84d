"""Multi-GPU means replicas: each rank answers its own query shard on its own copy of the
graph, and the only exchange is the benchmark's reduction (slowest step time, total
traversed edges).  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms, te = bench.replica_reduce(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    q.put((rank, step_ms, te))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_reduce_max_time_and_total_edges():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 20.0, 3000), (1, 20.0, 3000)]


def test_replica_shards_are_distinct_and_well_formed():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    a = synth.workload_queries(2, el, count=16, shard=0)
    b = synth.workload_queries(2, el, count=16, shard=1)
    assert len(a) == len(b) == 32
    assert [q.vertex for q in a] != [q.vertex for q in b]
    out_deg, in_deg = synth.degrees(el)
    for q in a + b:
        assert out_deg[q.vertex] > 0 and in_deg[q.vertex] > 0
