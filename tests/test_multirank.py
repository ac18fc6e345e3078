"""Host logic of the multi-GPU path, on CPU with two gloo ranks.

The tracker shards without any data exchange (events are independent; so are sectors inside the
sector tracker), so N GPUs run N replicas.  What needs checking is the bookkeeping: every rank
tracks its own event, the job time is the slowest rank's, and the whole-job throughput counts
all ranks' events.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1712_09407_gb300 import eventgen
    local = 1.0 + rank                      # rank 1 is the slower replica
    mx = bench.reduce_max(local, world, "cpu")
    ev = eventgen.config_event(0, event=bench.replica_event(rank))
    dist.barrier()
    out.put((rank, mx, bench.replica_throughput(mx, 10, world), float(ev.y[:50].sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_events():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, v0, s0), (r1, mx1, v1, s1) = res
    assert mx0 == mx1 == 2.0
    assert v0 == v1 == 2 * 10 / 2.0
    assert s0 != s1                          # the replicas tracked different events


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.replica_throughput(2.0, 10, 1) == 5.0
