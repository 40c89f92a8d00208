"""Writes the FP64 oracle's 100-iteration free runs of the 128x128 / 3-mode /
1600-position jittered raster (supplied positions off by up to 3 px; M-rPIE
section, Eqs. 5-7; Adam-based position refinement section, Eqs. 8-9,
Algorithm 1).  Calls only ``oracle`` and the shared seeded input generator;
nothing here touches the CUDA library.

    python tests/golden/make_w128_free_runs.py plain|refine|perturbed

plain      M-rPIE alone, 100 iterations -> plain_w128_m3_n1600.npz: the
           error curve and the final object and probe (complex128 rounded to
           complex64; the bar after 100 iterations is 1e-3 relative L2).
refine     XCORR_A registration (U = 20) and Adam steps (lr 0.5 px) from
           iteration 10 -> refine_w128_m3_n1600.npz: the error curve, the
           positions, measured shifts (integer multiples of 1/U) and float64
           near-tie gaps of the first refining iteration, the final positions
           and probe.
perturbed  the same run from a probe guess perturbed by 1e-7 relative
           (seeded complex noise, the size of a float32 rounding) ->
           refine_w128_m3_n1600_perturbed.npz: error curve, final positions
           and probe.  The distance between the two refining runs measures
           how strongly the method's own trajectory amplifies a rounding-size
           difference on this workload.

The SHA-256 of the counts is stored so that a test can check that it
regenerates the same inputs.
"""
import hashlib
import os
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # one BLAS thread: a fixed summation order

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rpie  # noqa: E402
from paper_2205_04295_b300 import synth  # noqa: E402

N_ITER, START, U, LR = 100, 10, 20, 0.5
HERE = os.path.dirname(os.path.abspath(__file__))
PERTURB = 1e-7


def perturbed_probe(P0):
    rng = np.random.default_rng(1)
    xi = (rng.normal(size=P0.shape) + 1j * rng.normal(size=P0.shape)) / np.sqrt(2.0)
    return np.asarray(P0, np.complex128) * (1.0 + PERTURB * xi)


def main(kind):
    wl = synth.refine_128()
    d = synth.build(wl)
    I = synth.counts_u16(d["I"])
    sha = np.array(hashlib.sha256(I.tobytes()).hexdigest())
    P0 = perturbed_probe(d["P0"]) if kind == "perturbed" else d["P0"]
    st = rpie.State.create(d["O0"], P0, d["pos"])
    prm = rpie.RPIEParams()
    rfn = None if kind == "plain" else rpie.RefineParams(upsample=U, lr=LR, start_iter=START)
    err = np.zeros(N_ITER)
    extra = {}
    t0 = time.time()
    for it in range(N_ITER):
        err[it] = rpie.iterate(st, I, prm, rfn)
        if rfn is not None and it == START:
            extra = dict(pos_first=st.pos.copy(),
                         shift_first=np.rint(st.last_shift * U).astype(np.int16),
                         gap_first=np.asarray(st.gap, np.float64).copy())
        print("%s iteration %d  error %.6e  %.0f s" % (kind, it, err[it], time.time() - t0), flush=True)
    out = dict(err=err, P=st.P.astype(np.complex64), counts_sha256=sha, n_iter=N_ITER)
    if kind == "plain":
        out["O"] = st.O.astype(np.complex64)
        name = "plain_w128_m3_n1600.npz"
    else:
        out.update(pos=st.pos, start=START, U=U, lr=LR, **extra)
        if kind == "perturbed":
            out["perturbation"] = PERTURB
        name = "refine_w128_m3_n1600%s.npz" % ("_perturbed" if kind == "perturbed" else "")
    np.savez_compressed(os.path.join(HERE, name), **out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "plain")
