"""The fused single-kernel patch path for W <= 128 (one thread-block cluster
of S CTAs per patch, each holding every mode's W/S rows and, between two
transposes through distributed shared memory, W/S columns; no far-field
scratch) against the FP64 oracle on the same seeded inputs and the same
grouped schedule, and against the three-pass path.

The fused kernel repeats the three-pass arithmetic step for step (same line
DFTs, same constraint and update expressions, same summation orders over the
modes); the probe sums are grouped differently (one slot per cluster instead
of one per CTA column).  The two paths agree to rounding.

Bars as for the three passes: relative L2 <= 1e-5 after one iteration
(object, probe, their changes, the model intensities, the error), <= 1e-3
after 100."""
import numpy as np
import pytest

from helpers import build, rel_l2
from oracle import model, rpie
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu

TOL1 = 1e-5


def problem(wl, d, S=0, scratch_bytes=0):
    from paper_2205_04295_b300 import pty
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, scratch_bytes=scratch_bytes)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    if S:
        prob.set_tiling(fused=S, scratch_bytes=scratch_bytes)
        assert prob.tiling()["fused"] == S
    return prob


def params_pair(**kw):
    from paper_2205_04295_b300 import pty
    return pty.rpie_params(**kw), rpie.RPIEParams(**kw)


def check_one_iteration(wl, d, S, scratch_bytes=0, **kw):
    pg, po = params_pair(**kw)
    prob = problem(wl, d, S, scratch_bytes)
    prob.profile(0)
    prob.stats(reset=True)
    eg = prob.run(1, pg)[0]
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    eo = rpie.iterate(st, d["I"], po)
    Og, Pg = prob.object(False), prob.probe(False)
    assert rel_l2(Og, st.O) <= TOL1
    assert rel_l2(Pg, st.P) <= TOL1
    assert rel_l2(Og - d["O0"], st.O - d["O0"]) <= TOL1
    assert rel_l2(Pg - d["P0"], st.P - d["P0"]) <= TOL1
    Ig = prob.model_intensities(False)
    Io = model.model_intensities(st.O, st.P, d["pos"])
    assert rel_l2(Ig, Io) <= TOL1
    assert abs(eg - eo) <= TOL1 * eo
    # the fused kernel ran, the passes did not
    st_ = prob.stats()
    assert st_["launches"]["patch"] > 0
    assert st_["launches"]["rows_fwd"] == st_["launches"]["cols"] == st_["launches"]["rows_inv"] == 0
    return prob, st


CASES = {
    "w32_m2": (lambda: synth.tiny(W=32, M=2, ny=5, nx=5, step=6.0), (1, 2, 4)),
    "w64_m1_plain": (lambda: synth.plain_rpie_64(), (1, 2, 4, 8)),
    "w64_m4": (lambda: synth.tiny(W=64, M=4, ny=4, nx=4, step=10.0, seed=21), (4, 8)),
    "w96_m1": (lambda: synth.tiny(W=96, M=1, ny=3, nx=4, step=20.0, seed=26), (2, 4)),
    "w96_m2": (lambda: synth.tiny(W=96, M=2, ny=3, nx=4, step=20.0, seed=3), (4,)),
    "w128_m3": (lambda: synth.tiny(W=128, M=3, ny=3, nx=3, step=24.0, seed=4, photons=1e6), (8,)),
    "w128_m1": (lambda: synth.tiny(W=128, M=1, ny=3, nx=3, step=24.0, seed=22), (4, 8)),
}
PARAMS = [(c, S) for c, (_, Ss) in CASES.items() for S in Ss]


@pytest.mark.parametrize("case,S", PARAMS, ids=["%s_S%d" % p for p in PARAMS])
def test_one_iteration_parity(case, S):
    wl = CASES[case][0]()
    check_one_iteration(wl, build(wl), S)


def test_regularisers_and_modes():
    wl = synth.tiny(W=32, M=3, ny=7, nx=6, step=5.0, seed=11, jitter=1.5)
    d = build(wl)
    check_one_iteration(wl, d, 2, alpha_O=0.7, alpha_P=0.6, beta=0.4, gamma=0.25)
    check_one_iteration(wl, d, 1, max_group=1)
    check_one_iteration(wl, d, 2, update_probe=False)


def test_single_group_matches_three_pass():
    """Nine disjoint boxes form one group: object, probe and error after it
    agree with the three-pass path to rounding (1e-6)."""
    wl = synth.tiny(W=64, M=3, ny=3, nx=3, step=72.0, seed=23, photons=1e6)
    d = build(wl)
    from paper_2205_04295_b300 import pty
    outs = []
    for S in (0, 2, 4):
        prob = problem(wl, d, S)
        assert len(prob.groups()) == 1
        e = prob.run(1, pty.rpie_params())[0]
        outs.append((prob.object(False), prob.probe(False), e))
    O0 = d["O0"]
    for O, P, e in outs[1:]:
        assert rel_l2(O - O0, outs[0][0] - O0) <= 1e-6
        assert rel_l2(P, outs[0][1]) <= 1e-6
        assert abs(e - outs[0][2]) <= 1e-6 * outs[0][2]


def test_more_patches_than_resident_clusters():
    """A group larger than the clusters that fit at once: each cluster takes
    several patches in turn and accumulates its probe-sum slot."""
    wl = synth.tiny(W=32, M=2, ny=24, nx=24, step=40.0, seed=24)
    d = build(wl)
    check_one_iteration(wl, d, 4)


def test_runs_are_bitwise_deterministic():
    wl = synth.tiny(W=64, M=3, ny=5, nx=5, step=8.0, seed=14)
    d = build(wl)
    outs = []
    for _ in range(2):
        prob = problem(wl, d, 2)
        e = prob.run(3)
        outs.append((prob.object(False), prob.probe(False), e))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)


def test_plain_rpie_100_iterations():
    """64x64 / 1 mode / 10x10 raster, 100 free iterations on the fused path
    (four CTAs per patch): bar 1e-3."""
    wl = synth.plain_rpie_64()
    d = build(wl)
    pg, po = params_pair()
    prob = problem(wl, d, 4)
    eg = prob.run(100, pg)
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    eo = rpie.run(st, d["I"], po, 100)
    assert rel_l2(prob.object(False), st.O) <= 1e-3
    assert rel_l2(prob.probe(False), st.P) <= 1e-3
    np.testing.assert_allclose(eg, eo, rtol=1e-3)


@pytest.mark.parametrize("point", ["A", "B"])
def test_registration_single_group_matches_three_pass(point):
    """With registration the fused kernel also writes the crop planes the
    registration reads (XCORR_A: row DFTs of o_j and o'_j; XCORR_B: model
    intensity and counts): in one group, shifts agree with the three-pass
    path except at near-ties, positions within 0.01 px, the object to
    rounding."""
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=64, M=2, ny=3, nx=3, step=72.0, seed=25, photons=1e6, jitter=1.0, err=2.0)
    d = build(wl)
    outs = []
    for S in (0, 2):
        prob = problem(wl, d, S)
        rg = pty.refine_params(upsample=20, lr=0.5, point=point)
        assert len(prob.groups()) == 1
        e, sh = prob.refine(1, pty.rpie_params(), rg, shifts=True)
        outs.append((sh, prob.positions(False), prob.object(False), prob.refine_gaps()))
    flip = np.abs(outs[0][0] - outs[1][0]).max(1) > 1e-5
    tie = (outs[0][3] <= 1e-5) | (outs[1][3] <= 1e-5)
    assert not np.any(flip & ~tie)
    dp = np.abs(outs[0][1] - outs[1][1]).max(1)
    assert np.all(dp[~flip] <= 1e-4)
    assert rel_l2(outs[1][2] - d["O0"], outs[0][2] - d["O0"]) <= 1e-6


def test_registration_parity_with_chunks():
    """XCORR_A registration on the fused path against the oracle, with a
    scratch of 3 patches (every group runs in chunks): shifts agree except at
    near-ties, positions within 0.01 px, object and probe within 1e-5."""
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=64, M=2, ny=5, nx=5, step=10.0, seed=31, photons=1e6, jitter=1.5, err=2.0)
    d = build(wl)
    sb = 3 * 4 * 64 * 64 * 8
    prob = problem(wl, d, 2, scratch_bytes=sb)
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    pg, po = pty.rpie_params(), rpie.RPIEParams()
    rg = pty.refine_params(upsample=20, lr=0.5)
    ro = rpie.RefineParams(upsample=20, lr=0.5)
    eg, sh = prob.refine(1, pg, rg, shifts=True)
    eo = rpie.iterate(st, d["I"], po, ro)
    gaps = prob.refine_gaps()
    flip = np.abs(sh - st.last_shift).max(1) > 1e-5
    tie = (gaps <= 1e-5) | (st.gap <= 1e-5)
    assert not np.any(flip & ~tie)
    assert flip.sum() <= 2
    dp = np.abs(prob.positions(False) - st.pos).max(1)
    assert np.all(dp[~flip] <= 0.01)
    assert rel_l2(prob.object(False), st.O) <= 1e-5
    assert rel_l2(prob.probe(False), st.P) <= 1e-5
    assert abs(eg[0] - eo) <= 1e-5 * eo


def test_unsupported_fused_tilings_are_rejected():
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=64, M=3, ny=2, nx=2, step=10.0)
    d = build(wl)
    prob = problem(wl, d)
    for S in (3, 16, -1):
        with pytest.raises(pty.PtyError, match="EINVAL"):
            prob.set_tiling(fused=S)
    with pytest.raises(pty.PtyError, match="does not fit"):
        prob.set_tiling(fused=1)  # two 3-mode 64 x 64 slabs exceed the shared memory
    assert prob.tiling()["fused"] == 0
    prob.set_tiling(fused=4)
    assert prob.tiling()["fused"] == 4
    prob.set_tiling()
    assert prob.tiling()["fused"] == 0
    wl2 = synth.tiny(W=256, M=1, ny=2, nx=2, step=40.0)
    prob2 = problem(wl2, build(wl2))
    with pytest.raises(pty.PtyError, match="does not fit"):
        prob2.set_tiling(fused=1)
