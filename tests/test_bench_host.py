"""Host-side pieces of the benchmark (no GPU): the oracle timings that the
reference arm reports, on a tiny workload."""
from paper_2205_04295_b300 import synth


def test_oracle_sample_and_all_core_figure():
    import bench
    wl = synth.tiny(W=32, M=2, ny=4, nx=4, step=12.0, seed=5)
    d = bench.host_inputs_for_groups(wl, 8)
    rate, done, dt, ng = bench.oracle_sample(wl, d, 0.2)
    assert rate > 0 and done > 0 and ng >= 1
    r = bench.oracle_all_cores(wl, 2, 0.5)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0


def test_batch_shard_partitions_and_balances():
    """Every problem of the batched workload runs on exactly one rank, and the
    ranks' shares of the work are near-equal (longest first, least loaded)."""
    import bench
    wls = [synth.batch_problem(p) for p in range(64)]
    costs = [bench.problem_cost(w) for w in wls]
    for world in (1, 2, 4, 8):
        shards = [bench.batch_shard(costs, r, world) for r in range(world)]
        flat = sorted(p for s in shards for p in s)
        assert flat == list(range(64))
        loads = [sum(costs[p] for p in s) for s in shards]
        assert max(loads) <= 1.1 * sum(costs) / world + max(costs)


def test_spread_spiral_has_the_group_size_of_the_full_spiral():
    """The profiling workload `spiral_256_n2000_spread5` stands in for the
    10^4-position spiral at a fifth of its positions: same extent, so its
    greedy disjoint groups (whose far field sets the passes' L2 behaviour)
    have the full spiral's size.  spread = 1 is the full spiral itself."""
    import numpy as np
    import bench
    from paper_2205_04295_b300 import pty
    wls = bench.workloads()
    head = wls["spiral_256"]()
    assert np.array_equal(synth.spiral_256(spread=1.0).pos_true, head.pos_true)
    sparse = wls["spiral_256_n2000_spread5"]()
    assert sparse.N == 2000 and sparse.W == head.W and sparse.M == head.M
    sizes = {}
    for name, wl in (("head", head), ("sparse", sparse)):
        g = pty.group_positions(wl.pos.astype(np.float32), wl.W)
        sizes[name] = np.array([len(x) for x in g])
    # 164 groups of 61 patches on average against 39 of 51
    assert abs(np.median(sizes["sparse"]) / np.median(sizes["head"]) - 1.0) < 0.2
    assert sizes["sparse"].max() >= 0.9 * sizes["head"].max()
