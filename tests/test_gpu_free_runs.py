"""100-iteration free runs of the 128x128 / 3-mode / 1600-position jittered
raster (supplied positions off by up to 3 px) against the FP64 oracle's own
runs, stored by tests/golden/make_w128_free_runs.py (it calls only the
oracle and the shared input generator).

* M-rPIE alone: object and probe within 1e-3 relative L2 (the bar for long
  runs) and the error curve within 1e-3.
* With XCORR_A registration (U = 20) and Adam steps (lr 0.5 px) from
  iteration 10:
  - the ten plain iterations: error curve within 1e-5;
  - the first refining iteration: every measured shift equals the oracle's
    except at a near-tie (relative gap between the two best fine-grid values
    below NEAR_TIE, from the oracle's float64 values or the kernel's own),
    and every other position is within 0.01 px of the oracle's;
  - after 100 iterations.  On this workload most registrations are close
    calls (the oracle's float64 gap is below 1e-5 for about 40 % of them:
    the correlation peak is flat on the 1/20 px grid), and Adam turns a
    0.05 px difference into steps of up to lr, so the runs separate after
    the first near-tie flip.  How far two runs drift apart is a property of
    the method on this workload, measured by the oracle itself: the same
    run from a probe guess perturbed by 1e-7 (a float32 rounding) is stored
    too (1e-7 in the probe guess moves the probe by 12 %, the positions by
    0.75 px RMS and the error curve by 0.8 % after 100 iterations).  The GPU
    run, whose first near-tie flips come ten iterations earlier than the
    perturbed oracle's, must stay within 5x that drift of the oracle (probe,
    positions, error curve)."""
import hashlib
import os

import numpy as np
import pytest

from helpers import build, rel_l2
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NEAR_TIE = 1e-5


def load(name):
    return np.load(os.path.join(GOLD, name))


def workload():
    wl = synth.refine_128()
    d = build(wl)
    return wl, d, hashlib.sha256(np.ascontiguousarray(d["I"]).tobytes()).hexdigest()


def rms(a, b):
    return float(np.sqrt(((np.asarray(a, np.float64) - b) ** 2).sum(1).mean()))


def test_plain_100_iterations_full_128_scan():
    from paper_2205_04295_b300 import pty
    g = load("plain_w128_m3_n1600.npz")
    wl, d, sha = workload()
    assert sha == str(g["counts_sha256"]), "the seeded inputs no longer match the stored run"
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    eg = prob.run(100, pty.rpie_params())
    assert rel_l2(prob.object(False), g["O"]) <= 1e-3
    assert rel_l2(prob.probe(False), g["P"]) <= 1e-3
    np.testing.assert_allclose(eg, g["err"], rtol=1e-3)


def test_refine_100_iterations_full_128_scan():
    from paper_2205_04295_b300 import pty
    g = load("refine_w128_m3_n1600.npz")
    gp = load("refine_w128_m3_n1600_perturbed.npz")
    wl, d, sha = workload()
    assert sha == str(g["counts_sha256"]), "the seeded inputs no longer match the stored run"
    U, start = int(g["U"]), int(g["start"])
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    pg = pty.rpie_params()
    rg = pty.refine_params(upsample=U, lr=float(g["lr"]), start_iter=start)
    err = list(prob.refine(start, pg, rg))
    np.testing.assert_allclose(err, g["err"][:start], rtol=1e-5)
    e, sh = prob.refine(1, pg, rg, shifts=True)
    err += list(e)
    gaps = prob.refine_gaps()
    flip = np.any(np.rint(sh * U).astype(np.int64) != g["shift_first"], axis=1)
    tie = (g["gap_first"] <= NEAR_TIE) | (gaps <= NEAR_TIE)
    assert not np.any(flip & ~tie), np.nonzero(flip & ~tie)
    assert flip.mean() <= 0.05
    dpos = np.abs(prob.positions(False) - g["pos_first"]).max(1)
    assert np.all(dpos[~flip] <= 0.01), dpos[~flip].max()
    err += list(prob.refine(int(g["n_iter"]) - start - 1, pg, rg))
    # the oracle's own drift under a rounding-size perturbation of its input
    drift_P = rel_l2(gp["P"], g["P"])
    drift_pos = rms(gp["pos"], g["pos"])
    drift_err = float(np.max(np.abs(gp["err"] - g["err"]) / g["err"]))
    ours_P = rel_l2(prob.probe(False), g["P"])
    ours_pos = rms(prob.positions(False), g["pos"])
    ours_err = float(np.max(np.abs(np.asarray(err) - g["err"]) / g["err"]))
    print("drift of the perturbed oracle: P %.3g, positions %.3g px, error %.3g;"
          " GPU vs oracle: P %.3g, positions %.3g px, error %.3g"
          % (drift_P, drift_pos, drift_err, ours_P, ours_pos, ours_err))
    assert ours_P <= 5 * drift_P
    assert ours_pos <= 5 * drift_pos
    assert ours_err <= 5 * drift_err
