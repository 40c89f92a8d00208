"""XCORR_A against XCORR_B in the oracle (Adam-based position refinement
section, Fig. 2, and the simulated comparison of the two switch positions
the paper summarises in its discussion): a 64 x 64 / 2-mode raster with +-2 px
errors on the supplied positions, 60 M-rPIE iterations with registration
from iteration 10 (U = 20, Adam lr 0.5 px).

Measured with the FP64 oracle (RMS position error after removing the mean
offset, initial 1.61 px):

    probe phase curvature   XCORR_A after 60   XCORR_B after 60
    0 (flat)                1.46               18.7 (runs away)
    pi                      1.21               19.6 (runs away)
    4 pi                    0.89               0.38

With a flat or mildly curved probe the far-field intensity is nearly
invariant to a shift of the object, so the detector-plane correlation has no
position signal and its noise drives the positions off; the object-plane
correlation of XCORR_A keeps working, as the paper reports.  A strongly
curved probe turns the far field into a magnified shadow image of the
object, and only there does XCORR_B see the shift."""
import numpy as np
import pytest

from helpers import build
from oracle import rpie
from paper_2205_04295_b300 import synth


def rms(pos, true):
    e = np.asarray(pos, np.float64) - true
    e = e - e.mean(0)
    return float(np.sqrt((e ** 2).sum(1).mean()))


@pytest.mark.parametrize("curv,bad_b", [(0.0, True), (4.0 * np.pi, False)])
def test_oracle_xcorr_a_vs_b(curv, bad_b):
    wl = synth.tiny(W=64, M=2, ny=5, nx=5, step=12.0, seed=71, photons=1e6, jitter=1.0, err=2.0)
    wl.probe_curv = curv
    d = build(wl)
    e0 = rms(d["pos"], wl.pos_true)
    out = {}
    for point in ("A", "B"):
        st = rpie.State.create(d["O0"], d["P0"], d["pos"])
        rfn = rpie.RefineParams(upsample=20, lr=0.5, start_iter=10, point=point)
        rpie.run(st, d["I"], rpie.RPIEParams(), 60, rfn)
        out[point] = rms(st.pos, wl.pos_true)
    assert out["A"] < 0.95 * e0
    if bad_b:
        assert out["B"] > 5 * e0
    else:
        assert out["B"] < out["A"]
