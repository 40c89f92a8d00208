"""The batched persistent form: many uneven problems in one cooperative,
graph-captured launch.  Each problem must come out exactly as it does when
run alone through pty_run_iterations (same kernels, same order of every
reduction), and hence match the oracle; a dependency that is never met must
end in PTY_ETIMEOUT, not a hang, and leave the GPU usable."""
import numpy as np
import pytest

from helpers import build, rel_l2
from oracle import rpie
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu


def small_mix():
    return [synth.tiny(W=32, M=1, ny=4, nx=5, step=6.0, seed=51),
            synth.tiny(W=64, M=2, ny=5, nx=4, step=10.0, seed=52, jitter=1.0),
            synth.tiny(W=96, M=3, ny=3, nx=3, step=16.0, seed=53, photons=1e6),
            synth.tiny(W=128, M=2, ny=3, nx=4, step=20.0, seed=54, photons=1e6),
            synth.tiny(W=64, M=1, ny=6, nx=6, step=8.0, seed=55),
            synth.tiny(W=192, M=3, ny=2, nx=2, step=40.0, seed=56, photons=1e6)]


def run_batch(wls, ds, n_iter, **sched):
    from paper_2205_04295_b300 import pty
    b = pty.Batch([(w.W, w.M, w.N, w.Hy, w.Hx) for w in wls])
    if sched:
        b.schedule(**sched)
    for p, d in zip(b.problems, ds):
        p.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    return b


def test_batch_equals_standalone_runs_and_oracle():
    from paper_2205_04295_b300 import pty
    wls = small_mix()
    ds = [build(w) for w in wls]
    b = run_batch(wls, ds, 3)
    b.run(3)
    assert list(b.status()) == [0] * len(wls)
    for w, d, p in zip(wls, ds, b.problems):
        solo = pty.Problem(w.W, w.M, w.N, w.Hy, w.Hx)
        solo.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        solo.run(3)
        np.testing.assert_array_equal(p.object(False), solo.object(False))
        np.testing.assert_array_equal(p.probe(False), solo.probe(False))
    for k in (0, 2):
        st = rpie.State.create(ds[k]["O0"], ds[k]["P0"], ds[k]["pos"])
        rpie.run(st, ds[k]["I"], rpie.RPIEParams(), 3)
        assert rel_l2(b.problems[k].object(False), st.O) <= 1e-4
        assert rel_l2(b.problems[k].probe(False), st.P) <= 1e-4
    b.close()


def test_batch_50_iterations_against_the_oracle():
    """All six problems of the uneven mix, 50 M-rPIE iterations in one
    persistent launch (the batched workload's iteration count), against the
    FP64 oracle run problem by problem: relative L2 <= 1e-3 (the bar for long
    runs) on object and probe, and the error curve to 1e-3."""
    wls = small_mix()
    ds = [build(w) for w in wls]
    b = run_batch(wls, ds, 50)
    b.run(50)
    assert list(b.status()) == [0] * len(wls)
    for k, (w, d) in enumerate(zip(wls, ds)):
        st = rpie.State.create(d["O0"], d["P0"], d["pos"])
        rpie.run(st, d["I"], rpie.RPIEParams(), 50)
        assert rel_l2(b.problems[k].object(False), st.O) <= 1e-3, k
        assert rel_l2(b.problems[k].probe(False), st.P) <= 1e-3, k
    b.close()


def test_group_cap_schedule_matches_standalone_and_oracle():
    """The autotuner may cap the positions per disjoint group (a different,
    equally valid schedule): with the same cap the batched form equals the
    standalone runs bitwise and the oracle (max_group on its side too)."""
    from paper_2205_04295_b300 import pty
    wls = small_mix()[:3]
    ds = [build(w) for w in wls]
    b = run_batch(wls, ds, 3)
    b.run(3, pty.rpie_params(max_group=4))
    assert list(b.status()) == [0] * len(wls)
    for k, (w, d) in enumerate(zip(wls, ds)):
        solo = pty.Problem(w.W, w.M, w.N, w.Hy, w.Hx)
        solo.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        solo.run(3, pty.rpie_params(max_group=4))
        np.testing.assert_array_equal(b.problems[k].object(False), solo.object(False))
        st = rpie.State.create(d["O0"], d["P0"], d["pos"])
        rpie.run(st, d["I"], rpie.RPIEParams(max_group=4), 3)
        assert rel_l2(b.problems[k].object(False), st.O) <= 1e-4
        assert rel_l2(b.problems[k].probe(False), st.P) <= 1e-4
    b.close()


def test_schedule_variants_give_identical_results():
    wls = small_mix()[:4]
    ds = [build(w) for w in wls]
    outs = []
    for sched in ({}, dict(split_rows=1, split_cols=1, split_probe=1, ctas=40),
                  dict(split_rows=16, split_cols=8, split_probe=16)):
        b = run_batch(wls, ds, 2, **sched)
        b.run(2)
        outs.append([(p.object(False), p.probe(False)) for p in b.problems])
        b.close()
    for o in outs[1:]:
        for (a, pa), (c, pc) in zip(outs[0], o):
            np.testing.assert_array_equal(a, c)
            np.testing.assert_array_equal(pa, pc)


def test_never_met_dependency_times_out_cleanly():
    import time
    from paper_2205_04295_b300 import pty
    wls = small_mix()[:3]
    ds = [build(w) for w in wls]
    b = run_batch(wls, ds, 1, timeout_ms=200, stall_problem=1)
    t0 = time.time()
    with pytest.raises(pty.PtyError) as e:
        b.run(1)
    assert e.value.code == pty.PTY_ETIMEOUT
    assert time.time() - t0 < 5.0
    st = b.status()
    assert st[1] == pty.PTY_ETIMEOUT
    b.close()
    # the context is still usable
    w = wls[0]
    solo = pty.Problem(w.W, w.M, w.N, w.Hy, w.Hx)
    solo.set_data(ds[0]["I"], ds[0]["pos"], ds[0]["O0"], ds[0]["P0"])
    solo.run(1)
    assert np.all(np.isfinite(solo.object(False)))


def test_full_64_problem_batch_sampled():
    """The 64-problem uneven batch (W in {64,96,128,192}, N in 50..900, M in
    1..3, objects sized to the scans): two iterations in one launch; three
    sampled problems must equal their standalone runs bitwise."""
    from paper_2205_04295_b300 import pty
    wls = [synth.batch_problem(p) for p in range(64)]
    ds = [build(w) for w in wls]
    b = run_batch(wls, ds, 2)
    b.run(2)
    assert np.all(b.status() == 0)
    for k in (0, 17, 63):
        w, d = wls[k], ds[k]
        solo = pty.Problem(w.W, w.M, w.N, w.Hy, w.Hx)
        solo.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        solo.run(2)
        np.testing.assert_array_equal(b.problems[k].object(False), solo.object(False))
        np.testing.assert_array_equal(b.problems[k].probe(False), solo.probe(False))
    b.close()
