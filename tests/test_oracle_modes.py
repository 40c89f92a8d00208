"""Pins of the probe-mode orthogonalisation oracle (oracle/modes.py) against
facts that do not come from it: the mixed state (density matrix) and the
per-pixel total intensity are invariant, the new modes are orthogonal with
powers equal to the Gram eigenvalues in decreasing order, and already
orthogonal modes are only reordered and re-phased."""
import numpy as np
import pytest

from oracle import modes


def rand_modes(M, W, seed):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((M, W, W)) + 1j * rng.standard_normal((M, W, W))
    return P * (0.5 ** np.arange(M))[:, None, None]  # distinct powers


@pytest.mark.parametrize("M,W,seed", [(2, 6, 0), (3, 8, 1), (5, 5, 2)])
def test_mixed_state_is_invariant(M, W, seed):
    P = rand_modes(M, W, seed)
    Pn, w = modes.orthogonalize(P)
    np.testing.assert_allclose(modes.density(Pn), modes.density(P), atol=1e-12 * np.abs(P).max() ** 2 * M)
    np.testing.assert_allclose((np.abs(Pn) ** 2).sum(0), (np.abs(P) ** 2).sum(0), rtol=1e-12)


@pytest.mark.parametrize("M,W,seed", [(2, 6, 3), (4, 7, 4)])
def test_new_modes_are_orthogonal_with_ordered_powers(M, W, seed):
    Pn, w = modes.orthogonalize(rand_modes(M, W, seed))
    G = modes.gram(Pn)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-12 * np.abs(G).max()
    np.testing.assert_allclose(np.diag(G).real, w, rtol=1e-12)
    assert np.all(np.diff(w) <= 0)
    # Gram eigenvalues by the characteristic polynomial for M = 2 (closed form)
    if M == 2:
        P = rand_modes(M, W, seed)
        a, d = np.sum(np.abs(P[0]) ** 2), np.sum(np.abs(P[1]) ** 2)
        b = np.sum(P[0].conj() * P[1])
        disc = np.sqrt((a - d) ** 2 + 4 * abs(b) ** 2)
        np.testing.assert_allclose(w, [(a + d + disc) / 2, (a + d - disc) / 2], rtol=1e-12)


def test_orthogonal_modes_are_only_reordered_and_rephased():
    rng = np.random.default_rng(5)
    W = 8
    # three orthogonal modes: disjoint supports, powers 1 < 4 < 9
    P = np.zeros((3, W, W), np.complex128)
    for k, amp in enumerate((1.0, 2.0, 3.0)):
        P[k, :, 3 * k:3 * k + 2] = amp * np.exp(1j * rng.uniform(0, 6.28, (W, 2))) / np.sqrt(2 * W)
    Pn, w = modes.orthogonalize(P)
    np.testing.assert_allclose(w, [9.0, 4.0, 1.0], rtol=1e-12)
    for m, k in enumerate((2, 1, 0)):
        # same mode up to a unit phase
        ph = np.vdot(P[k], Pn[m]) / np.vdot(P[k], P[k])
        assert abs(abs(ph) - 1) < 1e-12
        np.testing.assert_allclose(Pn[m], ph * P[k], atol=1e-12)


def test_phase_convention_largest_entry_real_positive():
    P = rand_modes(3, 6, 6)
    A = P.reshape(3, -1)
    Pn, w = modes.orthogonalize(P)
    # recover V from P' = V^T P (least squares over the pixels)
    V = np.linalg.lstsq(A.T, Pn.reshape(3, -1).T, rcond=None)[0]
    for m in range(3):
        i = int(np.argmax(np.abs(V[:, m])))
        assert abs(V[i, m].imag) < 1e-10 and V[i, m].real > 0
