"""The multi-GPU form is replicas: every rank indexes its own read set and
the benchmark aggregates with the slowest rank's time.  That host logic runs
here on two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.make_workload("short", rank, n_reads=2000)
    local_ms = 100.0 + 50.0 * rank
    slowest = bench.max_over_ranks(local_ms, dist, device="cpu")
    value = bench.whole_job_mbps(w.bases, world, 3, slowest)
    q.put((rank, slowest, value, int(w.reads[:200].astype(np.int64).sum()), w.bases))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, sig0, b0), (r1, ms1, v1, sig1, b1) = out
    assert ms0 == ms1 == 150.0  # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(b0 * 2 * 3 / 0.150 / 1e6)
    assert b0 == b1 and sig0 != sig1  # same shape, each rank its own reads
