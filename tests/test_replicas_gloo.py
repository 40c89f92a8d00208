"""The multi-GPU path of the benchmark: replicas for one problem (it does not
shard: every group needs the full probe sums of the previous one), and the
batched workload's independent problems split between ranks with no
data-path collective.  Its host logic -- process group setup, barrier, max
over ranks of the timing, the whole-job rate and the problem split -- runs
here as two gloo ranks on the CPU."""
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


def _shard_rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    from paper_2205_04295_b300 import synth
    r, w, _ = bench.dist_setup(world, backend="gloo")
    costs = [bench.problem_cost(synth.batch_problem(p)) for p in range(64)]
    mine = bench.batch_shard(costs, r, w)
    got = [None] * w
    dist.all_gather_object(got, mine)
    # each rank "took" time proportional to its share: the job time is the slowest
    slow = bench.max_over_ranks(float(sum(costs[p] for p in mine)), w)
    out.put((r, got, slow))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1]                       # both ranks agree on the split
    a, b = res[0][1]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
    assert res[0][2] == res[1][2]
