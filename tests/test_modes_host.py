"""The library's host Hermitian eigensolver (used by the probe-mode
orthogonalisation) against numpy.linalg.eigh with the same ordering and phase
convention as the oracle (no GPU needed)."""
import numpy as np
import pytest

from oracle import modes
from paper_2205_04295_b300 import pty


def rand_herm(M, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    Q, _ = np.linalg.qr(B)
    lam = np.sort(rng.uniform(0.1, 10.0, M) * spread ** np.arange(M))[::-1]
    return (Q * lam) @ Q.conj().T, lam


@pytest.mark.parametrize("M,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (8, 4), (16, 5)])
def test_host_eigensolver_matches_eigh(M, seed):
    A, lam = rand_herm(M, seed)
    w, V = pty.hermitian_eig(A)
    we, Ve = np.linalg.eigh(A)
    order = np.argsort(-we, kind="stable")
    np.testing.assert_allclose(w, we[order], rtol=1e-12, atol=1e-12 * lam.max())
    np.testing.assert_allclose(V, modes.fix_phases(Ve[:, order]), atol=1e-10)
    np.testing.assert_allclose(V @ np.diag(w) @ V.conj().T, A, atol=1e-10 * lam.max())


def test_host_eigensolver_diagonal_and_widely_spread():
    A = np.diag([1.0, 5.0, 3.0]).astype(np.complex128)
    w, V = pty.hermitian_eig(A)
    np.testing.assert_array_equal(w, [5.0, 3.0, 1.0])
    np.testing.assert_array_equal(np.abs(V), np.eye(3)[:, [1, 2, 0]])
    A, lam = rand_herm(5, 9, spread=0.5)  # occupancies spread like 0.5^k
    w, V = pty.hermitian_eig(A)
    np.testing.assert_allclose(V @ np.diag(w) @ V.conj().T, A, atol=1e-10 * lam.max())


def test_host_eigensolver_rejects_bad_input():
    with pytest.raises(pty.PtyError):
        pty.hermitian_eig(np.full((2, 2), np.nan + 0j))
    with pytest.raises(pty.PtyError):
        pty.hermitian_eig(np.eye(17, dtype=np.complex128))
