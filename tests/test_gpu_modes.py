"""GPU probe-mode orthogonalisation (pty_orthogonalize_probe) against the
FP64 oracle (oracle/modes.py) on the same probes: the new modes, their
powers, the invariants, and that iterations continue from the result."""
import numpy as np
import pytest

from helpers import build, rel_l2
from oracle import modes
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu


def problem(wl, d, P=None):
    from paper_2205_04295_b300 import pty
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"] if P is None else P)
    return prob


@pytest.mark.parametrize("W,M,seed", [(64, 3, 81), (128, 2, 82), (256, 5, 83)])
def test_orthogonalize_matches_oracle(W, M, seed):
    wl = synth.tiny(W=W, M=M, ny=2, nx=2, step=W / 4, seed=seed)
    d = build(wl)
    rng = np.random.default_rng(seed)
    # a non-orthogonal probe: the initial guess with mixed-in modes
    mix = np.eye(M) + 0.3 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))
    P = np.tensordot(mix, d["P0"], axes=(1, 0)).astype(np.complex64)
    prob = problem(wl, d, P)
    w = prob.orthogonalize_probe()
    Pg = prob.probe(False)
    Po, wo = modes.orthogonalize(P.astype(np.complex128))
    np.testing.assert_allclose(w, wo, rtol=1e-6)
    assert rel_l2(Pg, Po) <= 1e-5
    G = modes.gram(Pg)
    assert np.abs(G - np.diag(np.diag(G))).max() <= 1e-5 * np.abs(G).max()
    tot = (np.abs(P.astype(np.complex128)) ** 2).sum(0)
    assert rel_l2((np.abs(Pg.astype(np.complex128)) ** 2).sum(0), tot) <= 1e-5


def test_orthogonalize_is_deterministic_and_iterations_continue():
    wl = synth.tiny(W=64, M=3, ny=4, nx=4, step=12.0, seed=84, photons=1e6)
    d = build(wl)
    outs = []
    for _ in range(2):
        prob = problem(wl, d)
        prob.run(2)
        w = prob.orthogonalize_probe()
        e = prob.run(2)
        outs.append((prob.probe(False), prob.object(False), w, e))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(outs[0][3])) and np.all(np.diff(outs[0][2]) <= 0)
