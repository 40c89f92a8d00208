"""Orthogonalisation of the probe modes (test infrastructure only).

The paper decomposes the beam into M mutually incoherent probe modes (M-rPIE
section, Eq. 4) and follows the multimode ePIE of Thibault & Menzel (Nature
494, 68, 2013).  Between iterations the modes can be replaced by an
orthogonal set spanning the same mixed state: with the M x M Gram matrix
G_kl = sum_r conj(P_k(r)) P_l(r) = V diag(lambda) V^H (Hermitian, lambda in
decreasing order), the new modes are P'_m = sum_k V_km P_k.  They are mutually
orthogonal with |P'_m|^2 summed over r equal to lambda_m, and the density
matrix rho(r, r') = sum_k P_k(r) conj(P_k(r')) is unchanged (V is unitary).

Each eigenvector is fixed only up to a unit phase; the reading used here
(and by the library) makes the largest-magnitude entry of each column of V
(the first such row on ties) real and positive.  Degenerate eigenvalues leave
the basis of their eigenspace free; callers compare invariants then.

numpy.linalg.eigh is the library primitive for the eigendecomposition.
"""
import numpy as np


def gram(P):
    """G_kl = sum_r conj(P_k(r)) P_l(r), complex128 (M, M)."""
    A = np.asarray(P, dtype=np.complex128).reshape(P.shape[0], -1)
    return A.conj() @ A.T


def fix_phases(V):
    """Make the largest-magnitude entry of each column real and positive."""
    V = np.array(V, dtype=np.complex128)
    for m in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, m])))  # first maximum
        V[:, m] *= np.exp(-1j * np.angle(V[i, m]))
    return V


def orthogonalize(P):
    """(P', lambda): orthogonal modes spanning the same mixed state, ordered by
    decreasing power lambda_m = sum_r |P'_m(r)|^2."""
    P = np.asarray(P, dtype=np.complex128)
    w, V = np.linalg.eigh(gram(P))
    order = np.argsort(-w, kind="stable")
    w, V = w[order], fix_phases(V[:, order])
    Pn = np.tensordot(V.T, P, axes=(1, 0))  # P'_m = sum_k V_km P_k
    return Pn, w


def density(P):
    """rho(r, r') = sum_k P_k(r) conj(P_k(r')) over the flattened pixels."""
    A = np.asarray(P, dtype=np.complex128).reshape(P.shape[0], -1)
    return A.T @ A.conj()
