"""Forward model of the oracle (Background section, Eqs. 1-3; M-rPIE
section, Eq. 4).

Readings (the paper leaves these open):

* D_z in the far field is taken as the unitary 2-D DFT (``norm="ortho"``).
  The Fraunhofer quadratic phase and scale of Eq. 2 cancel in the modulus
  step, which keeps the phase, and the scale is absorbed into the probe's
  photon normalisation.
* Diffraction patterns are stored detector-centred: the zero frequency sits
  at pixel (W/2, W/2), i.e. the stored pattern is ``fftshift`` of the
  unshifted |Psi|^2.
* The crop box of position j has its top-left corner at
  ``floor(pos_j + 0.5)`` (round half up) of the float32 position, positions
  being (y, x) in object pixels.
"""
import numpy as np


def F(x):
    """Unitary forward 2-D DFT over the last two axes (far-field D_z, Eq. 2)."""
    return np.fft.fft2(x, norm="ortho")


def Finv(x):
    """Unitary inverse 2-D DFT over the last two axes (D_{-z})."""
    return np.fft.ifft2(x, norm="ortho")


def to_detector(a):
    """Unshifted (DC at index 0) -> stored detector layout (DC at W/2)."""
    return np.fft.fftshift(a, axes=(-2, -1))


def from_detector(a):
    """Stored detector layout (DC at W/2) -> unshifted (DC at index 0)."""
    return np.fft.ifftshift(a, axes=(-2, -1))


def crop_corners(pos):
    """Integer top-left crop corners, floor(pos + 0.5), shape (N, 2) int64.

    The rounding decides an integer, so it is taken on the float32 value of
    the position (the precision positions are stored in), evaluated exactly.
    """
    pos = np.asarray(pos, dtype=np.float32).astype(np.float64)
    return np.floor(pos + 0.5).astype(np.int64)


def crop(O, corner, W):
    """o_j: the W x W region of the object lit at position j (Eq. 4)."""
    cy, cx = int(corner[0]), int(corner[1])
    if cy < 0 or cx < 0 or cy + W > O.shape[0] or cx + W > O.shape[1]:
        raise ValueError("crop box outside the object")
    return O[cy:cy + W, cx:cx + W]


def exit_waves(P, o):
    """psi_p = P_p * o_j for every mode p (Eq. 1 applied per mode)."""
    return P * o[None, :, :]


def model_intensity_unshifted(P, o):
    """Eq. 4: I_j = sum_p |D_z{P_p o_j}|^2, unshifted layout, float64."""
    Psi = F(exit_waves(P, o))
    return np.sum(np.abs(Psi) ** 2, axis=0)


def model_intensities(O, P, pos):
    """Eq. 4 for every position, in the stored detector layout, (N, W, W)."""
    P = np.asarray(P, dtype=np.complex128)
    O = np.asarray(O, dtype=np.complex128)
    W = P.shape[-1]
    corners = crop_corners(pos)
    out = np.empty((len(corners), W, W))
    for j, c in enumerate(corners):
        out[j] = to_detector(model_intensity_unshifted(P, crop(O, c, W)))
    return out


def canvas_map(P, corners, shape):
    """Scan density on the object ("canvas map", the M-rPIE discussion around
    Fig. 5): the summed probe intensity sum_j sum_p |P_p(r - c_j)|^2 that the
    positions deposit on each object pixel."""
    W = P.shape[-1]
    p2 = np.sum(np.abs(P) ** 2, axis=0)
    C = np.zeros(shape, dtype=np.float64)
    for cy, cx in np.asarray(corners, dtype=np.int64):
        C[cy:cy + W, cx:cx + W] += p2
    return C
