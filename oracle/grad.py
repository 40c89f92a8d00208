"""Differentiable forward model and its analytic gradient (FP64).

Forward model (bilinear crop so that positions are differentiable):

    o_j(r)  = sum_{a,b in {0,1}} w_a(fy) w_b(fx) O(iy + r_y + a, ix + r_x + b),
              iy = floor(y_j), fy = y_j - iy, w_0 = 1 - f, w_1 = f
    Psi_jp  = F(P_p o_j)                            (Eqs. 1, 2, 4)
    A_j     = sqrt(sum_p |Psi_jp|^2 + delta)        (smoothed model amplitude)
    L       = sum_j sum_u (A_j - sqrt(I_j))^2       (amplitude loss)

Gradients use PyTorch's convention for complex tensors, dL/dRe + i dL/dIm
(= 2 dL/dz*):

    G_Psi  = 2 (1 - sqrt(I) / A) Psi
    G_psi  = F^-1 G_Psi                             (F unitary)
    dL/dP_p += conj(o_j) G_psi_p
    G_o    = sum_p conj(P_p) G_psi_p ; scattered to dL/dO by the bilinear transpose
    dL/dy_j = Re sum_r conj(G_o(r)) do_j(r)/dy      (likewise for x)

delta = 0 is the plain amplitude loss, whose gradient direction is undefined
where the model intensity S vanishes (a cone point of sqrt(S)); delta > 0
(one photon by default) makes L smooth there, and the gradient above is the
exact gradient of L for every delta.
"""
import numpy as np

from .model import F, Finv, from_detector


def bilinear_crop(O, p, W):
    """Returns (o, do/dy, do/dx, (iy, ix), (fy, fx)) for one position p = (y, x)."""
    y, x = float(p[0]), float(p[1])
    iy, ix = int(np.floor(y)), int(np.floor(x))
    fy, fx = y - iy, x - ix
    if iy < 0 or ix < 0 or iy + W + 1 > O.shape[0] or ix + W + 1 > O.shape[1]:
        raise ValueError("bilinear crop outside the object")
    a = O[iy:iy + W, ix:ix + W]
    b = O[iy:iy + W, ix + 1:ix + W + 1]
    c = O[iy + 1:iy + W + 1, ix:ix + W]
    d = O[iy + 1:iy + W + 1, ix + 1:ix + W + 1]
    o = (1 - fy) * (1 - fx) * a + (1 - fy) * fx * b + fy * (1 - fx) * c + fy * fx * d
    dy = (1 - fx) * (c - a) + fx * (d - b)
    dx = (1 - fy) * (b - a) + fy * (d - c)
    return o, dy, dx, (iy, ix), (fy, fx)


def loss(O, P, pos, I, delta=1.0):
    """Amplitude loss L (no normalisation)."""
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    W = P.shape[-1]
    L = 0.0
    for j in range(len(pos)):
        o = bilinear_crop(O, pos[j], W)[0]
        S = np.sum(np.abs(F(P * o[None])) ** 2, axis=0)
        sqI = np.sqrt(from_detector(np.asarray(I[j], dtype=np.float64)))
        L += float(np.sum((np.sqrt(S + delta) - sqI) ** 2))
    return L


def loss_and_grad(O, P, pos, I, delta=1.0):
    """Returns (L, dL/dO, dL/dP, dL/dpos) in the convention above."""
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    W = P.shape[-1]
    gO = np.zeros_like(O)
    gP = np.zeros_like(P)
    gpos = np.zeros((len(pos), 2))
    L = 0.0
    for j in range(len(pos)):
        o, dy, dx, (iy, ix), (fy, fx) = bilinear_crop(O, pos[j], W)
        Psi = F(P * o[None])
        amp = np.sqrt(np.sum(np.abs(Psi) ** 2, axis=0) + delta)
        sqI = np.sqrt(from_detector(np.asarray(I[j], dtype=np.float64)))
        L += float(np.sum((amp - sqI) ** 2))
        G_psi = Finv(2.0 * (1.0 - sqI / amp)[None] * Psi)
        gP += np.conj(o)[None] * G_psi
        G_o = np.sum(np.conj(P) * G_psi, axis=0)
        gO[iy:iy + W, ix:ix + W] += (1 - fy) * (1 - fx) * G_o
        gO[iy:iy + W, ix + 1:ix + W + 1] += (1 - fy) * fx * G_o
        gO[iy + 1:iy + W + 1, ix:ix + W] += fy * (1 - fx) * G_o
        gO[iy + 1:iy + W + 1, ix + 1:ix + W + 1] += fy * fx * G_o
        gpos[j, 0] = float(np.real(np.sum(np.conj(G_o) * dy)))
        gpos[j, 1] = float(np.real(np.sum(np.conj(G_o) * dx)))
    return L, gO, gP, gpos
