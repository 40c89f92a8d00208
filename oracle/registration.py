"""XCORR_A subpixel registration (Adam-based position refinement section).

The paper measures the shift between the crop o_j before its update and the
refined crop o'_j by "2D weighted phase correlation" computed with the
upsampled matrix-multiply DFT of Guizar-Sicairos, Thurman & Fienup
(Opt. Lett. 33, 156, 2008): a coarse cross-correlation peak on the pixel grid,
then the cross-correlation re-evaluated only on a fine grid of spacing 1/U
around that peak, by two small matrix products, with no zero padding.

Definitions used here (readings of a passage the paper keeps short):

* A = DFT(a), B = DFT(b), X = B * conj(A) (unnormalised cross power; the
  "weighting" is |A||B|, what the 2008 method computes).
* c(r) = sum_u X(u) exp(+2 pi i u.r / W), u the signed integer frequency in
  [-W/2, W/2).  If b(r) = a(r + d) then c peaks at r = -d.
* coarse peak: first maximum of |c|^2 on the integer grid in row-major order,
  each coordinate wrapped to [-W/2, W/2).
* fine grid: K = ceil(1.5 U) points per axis at s0 + (k - K//2)/U,
  k = 0..K-1; the result is the first maximum of |c|^2 on it (row-major).

Precision: every value is evaluated in complex128 / float64 (the DFTs of
the crops, the cross power X, the coarse inverse DFT, the matrix DFT
E_r X E_c and |c|^2).  Only the final comparison of the argmax, which picks
an integer (a grid index), is taken on the float64 values rounded to
float32 (``decide``), the precision of the paper's PyTorch code and of the
CUDA kernels, so that both sides decide at the same resolution; equal
float32 values go to the first index.  ``decide=np.float64`` compares the
float64 values themselves.  The reported gap (best minus second best,
relative to the best) is always taken from the float64 values, so it says
how close the decision was independently of either side's rounding.

Written from the paper's description and the published method, not from any
third-party code.
"""
import math

import numpy as np


def signed_freqs(W):
    """Signed integer DFT frequencies, index order: 0, 1, .., W/2-1, -W/2, .., -1."""
    return np.fft.fftfreq(W) * W


def wrap(i, W):
    """Map a pixel index in [0, W) to a signed shift in [-W/2, W/2)."""
    return i - W if i >= W // 2 else i


def first_argmax(vals, decide=np.float32):
    """Index of the first maximum (flat, row-major) of ``vals`` compared at the
    resolution of ``decide``."""
    return int(np.argmax(np.asarray(vals, dtype=np.float64).astype(decide)))


def xcorr_peak(a, b, U, decide=np.float32):
    """Peak (sy, sx) of the cross-correlation of b against a, to 1/U pixel.

    Returns ``(shift, gap)`` where ``shift`` is a float64 pair and ``gap`` is the
    relative difference between the best and second-best fine-grid values of
    |c|^2 in float64 (a near-tie indicator; 1.0 when U <= 1).
    """
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    Wy, Wx = a.shape
    X = np.fft.fft2(b) * np.conj(np.fft.fft2(a))
    # coarse: c on the integer grid is W^2 * ifft2(X); the scale does not move the peak
    c = np.fft.ifft2(X)
    k = first_argmax(np.abs(c) ** 2, decide)
    r0, c0 = divmod(k, Wx)
    sy, sx = float(wrap(r0, Wy)), float(wrap(c0, Wx))
    if U <= 1:
        return np.array([sy, sx]), 1.0
    up, ys, xs = upsampled_xcorr(X, (sy, sx), U)
    flat = up.ravel()
    k1, k2 = divmod(first_argmax(flat, decide), up.shape[1])
    srt = np.sort(flat)
    gap = float((srt[-1] - srt[-2]) / srt[-1]) if srt[-1] > 0 else 0.0
    return np.array([ys[k1], xs[k2]]), gap


def upsampled_xcorr(X, center, U, K=None):
    """|c|^2 on the K x K fine grid centred (as above) on ``center``, as the two
    matrix products E_r X E_c (complex128); returns (|c|^2, ys, xs)."""
    Wy, Wx = X.shape
    K = int(math.ceil(1.5 * U)) if K is None else K
    half = K // 2
    ys = center[0] + (np.arange(K) - half) / U
    xs = center[1] + (np.arange(K) - half) / U
    Er = np.exp(2j * np.pi * np.outer(ys, signed_freqs(Wy)) / Wy)   # K x Wy
    Ec = np.exp(2j * np.pi * np.outer(signed_freqs(Wx), xs) / Wx)   # Wx x K
    return np.abs(Er @ np.asarray(X, dtype=np.complex128) @ Ec) ** 2, ys, xs
