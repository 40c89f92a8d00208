"""The multi-GPU path of the benchmark is replicas only (one problem does not
shard: every group needs the full probe sums of the previous one).  Its host
logic -- process group setup, barrier, max over ranks of the timing and the
whole-job rate -- runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_setup(world, backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    # rank k "took" 1 + k seconds for 100 units: the job rate uses the slowest
    rate = bench.replica_rate(100, 1.0 + rank, w)
    slow = bench.max_over_ranks(1.0 + rank, w)
    out.put((rank, rate, slow))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, slow in res:
        assert slow == 2.0
        assert rate == pytest.approx(2 * 100 / 2.0)
