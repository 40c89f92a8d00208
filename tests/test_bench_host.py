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
