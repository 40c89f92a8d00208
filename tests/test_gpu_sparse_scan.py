"""Sparse scanning on the GPU path (the discussion of Fig. 5): a 64x64,
two-mode raster and its checkerboard half, M-rPIE (gamma = 0.1) against
M-ePIE (gamma = 1) with the probe known, 20 iterations each through the
library.  Both runs follow the oracle (relative L2 of the object within
1e-3 after 20 iterations), and M-rPIE leaves the smaller object error in the
zone the canvas map covers well."""
import numpy as np
import pytest

from helpers import rel_l2
from oracle import model, rpie
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu


def test_sparse_raster_rpie_against_epie():
    import torch
    from paper_2205_04295_b300 import pty
    from test_oracle_sparse_scan import scaled_error
    n, W = 8, 64
    wl = synth.tiny(W=W, M=2, ny=n, nx=n, step=W / 4, seed=11, photons=1e6)
    d = synth.build(wl)
    I = np.asarray(d["I"]).astype(np.uint16)
    iy, ix = np.divmod(np.arange(wl.N), n)
    sel = np.nonzero((iy + ix) % 2 == 0)[0]
    pos = d["pos"][sel]
    C = model.canvas_map(d["P_true"], model.crop_corners(pos), (wl.Hy, wl.Hx))
    well = C > 0.3 * C.max()
    errs = {}
    for name, gamma in (("ePIE", 1.0), ("rPIE", 0.1)):
        prob = pty.Problem(W, 2, len(sel), wl.Hy, wl.Hx)
        prob.set_data(I[sel], pos, d["O0"], d["P_true"].astype(np.complex64))
        prob.run(20, pty.rpie_params(gamma=gamma, update_probe=False))
        Og = prob.object(False)
        prob.close()
        st = rpie.State.create(d["O0"], d["P_true"], pos)
        rpie.run(st, I[sel], rpie.RPIEParams(gamma=gamma, update_probe=False), 20)
        assert rel_l2(Og, st.O) <= 1e-3
        errs[name] = scaled_error(Og.astype(np.complex128), d["O_true"], well)
    assert errs["rPIE"] < 0.95 * errs["ePIE"], errs
