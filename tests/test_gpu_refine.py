"""Parity of XCORR_A / XCORR_B registration + Adam position refinement (CUDA)
with the FP64 oracle.

The registration ends in an argmax over a 1/U-pixel grid; the oracle
evaluates every value in float64 and compares them at float32 resolution
(see oracle.registration), the kernels in float32.  Measured shifts must
agree exactly except where the two best grid values are within NEAR_TIE of
each other (the gap the oracle reports from its float64 values, or the
kernel's own): such flips are counted and must all be near-ties.
Long runs are checked in lock-step: every iteration starts the GPU from the
oracle's state (object, probe, positions, Adam moments) and the single-
iteration transition is compared, so registration error is separated from
the drift that one flipped argmax causes in a free run.  Bars: positions
within 0.01 px, object and probe relative L2 <= 1e-5 per transition."""
import numpy as np
import pytest

from helpers import build, rel_l2
from oracle import rpie
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu

NEAR_TIE = 1e-5


def pair(wl, d, lr=0.5, U=20, start=0, point="A", **kw):
    from paper_2205_04295_b300 import pty
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    pg, po = pty.rpie_params(**kw), rpie.RPIEParams(**kw)
    rg = pty.refine_params(upsample=U, lr=lr, start_iter=start, point=point)
    ro = rpie.RefineParams(upsample=U, lr=lr, start_iter=start, point=point)
    return prob, st, pg, po, rg, ro


def step_both(prob, st, d, pg, po, rg, ro):
    eg, sh = prob.refine(1, pg, rg, shifts=True)
    eo = rpie.iterate(st, d["I"], po, ro)
    return eg[0], eo, sh, prob.refine_gaps()


def compare_step(prob, st, sh, gaps):
    """Returns the mask of flipped shifts after checking they are near-ties."""
    flip = np.abs(sh - st.last_shift).max(1) > 1e-5
    tie = (gaps <= NEAR_TIE) | (st.gap <= NEAR_TIE)
    assert not np.any(flip & ~tie), "shift differs at a clear maximum: %s" % np.nonzero(flip & ~tie)
    pos = prob.positions(False)
    d = np.abs(pos - st.pos).max(1)
    assert np.all(d[~flip] <= 0.01), d[~flip].max()
    return flip


def load_state(prob, st):
    prob.set_object(st.O.astype(np.complex64))
    prob.set_probe(st.P.astype(np.complex64))
    prob.set_positions(st.pos.astype(np.float32))
    prob.set_adam_state(st.m.astype(np.float32), st.v.astype(np.float32), st.t, st.it)


def test_one_iteration_shifts_positions_object_probe():
    wl = synth.tiny(W=64, M=2, ny=5, nx=5, step=10.0, seed=31, photons=1e6, jitter=1.5, err=2.0)
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d)
    eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
    flip = compare_step(prob, st, sh, gaps)
    assert flip.sum() <= 2
    assert rel_l2(prob.object(False), st.O) <= 1e-5
    assert rel_l2(prob.probe(False), st.P) <= 1e-5
    assert abs(eg - eo) <= 1e-5 * eo


def test_start_iter_and_lockstep_256():
    wl = synth.tiny(W=256, M=5, ny=2, nx=3, step=48.0, seed=32, photons=1e6, jitter=1.0, err=1.5)
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, start=1)
    step_both(prob, st, d, pg, po, rg, ro)                     # plain iteration
    np.testing.assert_array_equal(prob.positions(False), d["pos"])
    for _ in range(3):
        load_state(prob, st)
        _, _, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        compare_step(prob, st, sh, gaps)
        assert rel_l2(prob.object(False), st.O) <= 1e-5
        assert rel_l2(prob.probe(False), st.P) <= 1e-5
    m, v, t, it = prob.adam_state()
    assert t == 3 and it == 4 and st.t == 3


def test_coarse_only_registration():
    wl = synth.tiny(W=32, M=1, ny=4, nx=4, step=6.0, seed=33, jitter=1.0, err=2.0)
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, U=1, start=1)
    step_both(prob, st, d, pg, po, rg, ro)
    load_state(prob, st)
    eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
    np.testing.assert_allclose(sh, st.last_shift, atol=1e-6)


def subset_128(ny=5, nx=5):
    full = synth.refine_128()
    sel = (np.arange(40)[:ny, None] * 40 + np.arange(nx)[None, :]).ravel()
    wl = synth.refine_128()
    wl.pos, wl.pos_true = full.pos[sel], full.pos_true[sel]
    lo = np.floor(wl.pos_true.min(0)) - 8
    wl.pos_true = wl.pos_true - lo
    wl.pos = np.clip(wl.pos - lo, 0, None).astype(np.float32)
    wl.Hy = wl.Hx = int(np.ceil(max(wl.pos_true.max(), wl.pos.max()))) + 128 + 8
    return wl


def test_refine_128_modes3_100_iterations_lockstep():
    """128x128 patterns, 3 modes, the first 5x5 block of the jittered 40x40
    raster with its +-3 px supplied error, U = 20, lr 0.5: 100 iterations,
    refinement from iteration 10, every transition compared."""
    wl = subset_128()
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, start=10)
    flips = 0
    for it in range(100):
        load_state(prob, st)
        eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        if it >= 10:
            flips += compare_step(prob, st, sh, gaps).sum()
        assert rel_l2(prob.object(False), st.O) <= 1e-5
        assert rel_l2(prob.probe(False), st.P) <= 1e-5
        assert abs(eg - eo) <= 1e-5 * eo
    assert flips <= 0.05 * 90 * wl.N


def test_refine_128_free_run_tracks_oracle():
    """The same subset run freely for 30 iterations (refinement from 10).
    Until the first near-tie argmax flips, the runs agree to 1e-5 in object
    and to 0.01 px in position; after it, one shift differs by 1/U and the
    trajectories separate, so only the error curve is compared (10 %)."""
    wl = subset_128()
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, start=10)
    eg, eo = [], []
    first_flip = None
    for it in range(30):
        a, b, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        eg.append(a)
        eo.append(b)
        if first_flip is None:
            flip = compare_step(prob, st, sh, gaps) if it >= 10 else np.zeros(wl.N, bool)
            if flip.any():
                first_flip = it
            else:
                assert rel_l2(prob.object(False), st.O) <= 1e-5
                assert abs(a - b) <= 1e-4 * b
    np.testing.assert_allclose(eg, eo, rtol=0.1)


def test_full_size_refine_128_one_iteration():
    """The full 128x128 / 3-mode / 1600-position scan, one refining iteration
    (one Adam step) in the benchmark's launch configuration."""
    wl = synth.refine_128()
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d)
    eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
    flip = compare_step(prob, st, sh, gaps)
    assert flip.mean() <= 0.05
    assert rel_l2(prob.object(False), st.O) <= 1e-5
    assert rel_l2(prob.probe(False), st.P) <= 1e-5


@pytest.mark.parametrize("W,M", [(64, 2), (256, 5)])
def test_xcorr_b_lockstep(W, M):
    """XCORR_B: the model intensity against the measured counts.  First
    iteration plain, then three refining transitions in lock-step."""
    wl = (synth.tiny(W=64, M=2, ny=5, nx=5, step=10.0, seed=34, photons=1e6, jitter=1.5, err=2.0)
          if W == 64 else
          synth.tiny(W=256, M=5, ny=2, nx=3, step=48.0, seed=35, photons=1e6, jitter=1.0, err=1.5))
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, start=1, point="B")
    step_both(prob, st, d, pg, po, rg, ro)
    for _ in range(3):
        load_state(prob, st)
        eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        flip = compare_step(prob, st, sh, gaps)
        assert flip.sum() <= max(1, 0.05 * wl.N)
        assert rel_l2(prob.object(False), st.O) <= 1e-5
        assert rel_l2(prob.probe(False), st.P) <= 1e-5
        assert abs(eg - eo) <= 1e-5 * eo


def test_xcorr_b_128_modes3_lockstep():
    """The 5 x 5 block of the 128 x 128 / 3-mode raster, XCORR_B from
    iteration 10, 20 transitions in lock-step."""
    wl = subset_128()
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, start=10, point="B")
    flips = 0
    for it in range(30):
        load_state(prob, st)
        eg, eo, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        if it >= 10:
            flips += compare_step(prob, st, sh, gaps).sum()
        assert rel_l2(prob.object(False), st.O) <= 1e-5
        assert rel_l2(prob.probe(False), st.P) <= 1e-5
    assert flips <= 0.05 * 20 * wl.N


def rms_position_error(pos, true):
    """RMS distance to the true positions after removing the mean offset (a
    common translation of all positions is not observable)."""
    e = np.asarray(pos, np.float64) - true
    e = e - e.mean(0)
    return float(np.sqrt((e ** 2).sum(1).mean()))


@pytest.mark.parametrize("curv", [0.0, 4.0 * np.pi])
def test_xcorr_a_vs_b_study(curv):
    """The comparison of the two switch positions of Fig. 2 on a simulated
    64 x 64 / 2-mode raster with +-2 px position errors, 60 iterations,
    registration from iteration 10.  With a flat-phase probe (curv = 0) the
    far-field intensity barely moves when the object does, XCORR_B carries no
    position signal and its positions run away, while XCORR_A improves them:
    the paper's finding that A is the point to use.  A strongly curved probe
    (curv = 4 pi, the probe of the other workloads) makes the detector image
    a shadow image of the object, and then XCORR_B has a signal too."""
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=64, M=2, ny=5, nx=5, step=12.0, seed=71, photons=1e6, jitter=1.0, err=2.0)
    wl.probe_curv = curv
    d = build(wl)
    e0 = rms_position_error(d["pos"], wl.pos_true)
    out = {}
    for point in ("A", "B"):
        prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
        prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        prob.refine(60, pty.rpie_params(), pty.refine_params(upsample=20, lr=0.5, start_iter=10,
                                                              point=point))
        out[point] = rms_position_error(prob.positions(False), wl.pos_true)
    assert out["A"] < e0
    if curv == 0.0:
        assert out["B"] > 3 * e0 > out["A"]
    else:
        assert out["B"] < e0


@pytest.mark.parametrize("W,M", [(32, 1), (64, 2), (96, 2), (128, 3), (192, 2), (256, 5)])
def test_tensor_core_registration_matches_fp32_cores_and_oracle(W, M):
    """The fine-grid DFT on the tensor cores (3xTF32 tcgen05 MMAs, tiles of
    128 rows, zero-padded past W) against the same DFT on the FP32 cores and
    against the oracle: from the same state, one refining iteration; shifts
    equal except at near-ties, positions, object and probe to the usual bars."""
    from paper_2205_04295_b300 import pty
    ny, nx, step = (5, 5, 6.0) if W <= 64 else ((3, 3, 0.25 * W) if W <= 128 else (2, 3, 0.2 * W))
    wl = synth.tiny(W=W, M=M, ny=ny, nx=nx, step=step, seed=36 + W, photons=1e6, jitter=1.0, err=1.5)
    d = build(wl)
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    po, ro = rpie.RPIEParams(), rpie.RefineParams(upsample=20, lr=0.5, start_iter=1)
    rpie.iterate(st, d["I"], po, ro)                     # a non-flat object to register
    res = []
    for fp32 in (False, True):
        prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, fp32_registration=fp32)
        prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        load_state(prob, st)
        _, sh = prob.refine(1, pty.rpie_params(), pty.refine_params(upsample=20, lr=0.5, start_iter=1),
                            shifts=True)
        res.append((sh, prob.refine_gaps(), prob.positions(False), prob.object(False)))
    st2 = rpie.State.create(st.O, st.P, st.pos)
    st2.m, st2.v, st2.t, st2.it = st.m.copy(), st.v.copy(), st.t, st.it
    rpie.iterate(st2, d["I"], po, ro)
    (sh_tc, gap_tc, pos_tc, O_tc), (sh_32, gap_32, pos_32, O_32) = res
    tie = (gap_tc <= NEAR_TIE) | (gap_32 <= NEAR_TIE) | (st2.gap <= NEAR_TIE)
    flip = np.abs(sh_tc - sh_32).max(1) > 1e-5
    assert not np.any(flip & ~tie)
    flip_o = np.abs(sh_tc - st2.last_shift).max(1) > 1e-5
    assert not np.any(flip_o & ~tie)
    ok = ~(flip | flip_o)
    assert np.all(np.abs(pos_tc - st2.pos).max(1)[ok] <= 0.01)
    # the object update itself does not depend on the registration
    np.testing.assert_array_equal(O_tc, O_32)
    assert rel_l2(O_tc, st2.O) <= 1e-5


def test_positions_clamped_at_the_object_border():
    """A supplied position on the object's border with a large Adam step (lr
    3 px) is clamped so that its crop stays inside, on both sides."""
    wl = synth.tiny(W=64, M=1, ny=3, nx=3, step=12.0, seed=37, photons=1e6, jitter=1.0, err=2.0)
    d = build(wl)
    d["pos"][0] = [0.0, 0.0]
    d["pos"][-1] = [wl.Hy - wl.W, wl.Hx - wl.W]
    prob, st, pg, po, rg, ro = pair(wl, d, lr=3.0, start=1)
    step_both(prob, st, d, pg, po, rg, ro)
    for _ in range(3):
        load_state(prob, st)
        _, _, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        compare_step(prob, st, sh, gaps)
        pos = prob.positions(False)
        assert pos.min() >= 0.0 and pos[:, 0].max() <= wl.Hy - wl.W and pos[:, 1].max() <= wl.Hx - wl.W


def test_fine_grid_beyond_the_tensor_core_tile_falls_back():
    """U = 25 gives K = 38 fine-grid points per axis, more than the tensor-core
    kernel's 32-column tile: the FP32-core kernel takes it, with the same
    parity as at U = 20."""
    wl = synth.tiny(W=64, M=2, ny=4, nx=4, step=10.0, seed=38, photons=1e6, jitter=1.0, err=2.0)
    d = build(wl)
    prob, st, pg, po, rg, ro = pair(wl, d, U=25, start=1)
    step_both(prob, st, d, pg, po, rg, ro)
    for _ in range(2):
        load_state(prob, st)
        _, _, sh, gaps = step_both(prob, st, d, pg, po, rg, ro)
        flip = compare_step(prob, st, sh, gaps)
        assert flip.sum() <= 1
        assert rel_l2(prob.object(False), st.O) <= 1e-5
