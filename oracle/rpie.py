"""One M-rPIE iteration over the grouped schedule, with optional XCORR_A +
Adam position refinement (M-rPIE and Adam-based position refinement
sections; Eqs. 4-9, Algorithm 1).

Per group S (a set of positions with pairwise-disjoint crop boxes), with O and
P the estimates at the start of the group:

    Pint(r)  = sum_p |P_p(r)|^2,   Pmax = max_r Pint(r)
    for j in S:
        o        = crop of O at corner_j                           (Eq. 4)
        psi_p    = P_p o                                            (Eq. 1)
        Psi_p    = F psi_p                                          (Eq. 2)
        S_j      = sum_p |Psi_p|^2
        err     += sum_u (sqrt(S_j) - sqrt(I_j))^2
        Psi'_p   = sqrt(I_j) Psi_p / (sqrt(S_j) + eps)              (Eq. 7, detector plane)
        D_p      = F^-1 Psi'_p - psi_p
        o'       = o + alpha_O sum_p D_p conj(P_p)
                         / (gamma Pmax + (1-gamma) Pint + reg_eps Pmax)   (Eq. 6)
        write o' back into O (disjoint boxes: no conflicts)
        num_p   += D_p conj(o);  den += beta max|o|^2 + (1-beta)|o|^2
        [refine] s_j = peak of xcorr(o, o')  (XCORR_A; XCORR_B: xcorr(S_j, I_j)),
                 g_j = -s_j
    P_p += alpha_P num_p / (den + reg_eps sum_j max|o_j|^2)         (Eq. 5, ratio of sums)

Readings: Eq. 7 as printed applies sqrt(I) to the exit-plane wave and sums
over positions; it is read as the usual modulus constraint in the detector
plane, every mode scaled by sqrt(I_j) over the root of the summed mode
intensities.  eps is taken at the one-photon amplitude level (eps = 1 by
default): with eps -> 0 the constrained wave at a detector pixel where the
model is (numerically) dark but photons were counted has full amplitude and
the phase of rounding noise, so the iteration stops being a continuous
function of its inputs.  Where an update denominator is exactly zero its
numerator is zero as well and the update there is skipped.  Both updates
read the pre-update o_j and P (the right-hand sides of
Eqs. 5-6 are unprimed).  Inside a group the probe update is the ratio of the
summed numerators and denominators; for a group of one position it is Eq. 5
exactly, and ``max_group=1`` gives the paper's sequential algorithm.  M-rPIE
with beta = gamma = 1 is M-ePIE (M-rPIE section).  The reported error is
sum (sqrt S - sqrt I)^2 over all patterns / sum I, taken before the
constraint.  With refinement on, every position measured in the iteration gets
one Adam step at the end of the iteration (Eqs. 8-9, Algorithm 1) and the
positions are clamped to keep the crop inside the object; regrouping happens
at the start of the next iteration.
"""
from dataclasses import dataclass

import numpy as np

from .adam import adam_step
from .grouping import greedy_groups
from .model import F, Finv, crop_corners, from_detector
from .registration import xcorr_peak


@dataclass
class RPIEParams:
    alpha_O: float = 1.0      # object step size (Eq. 6)
    alpha_P: float = 1.0      # probe step size (Eq. 5)
    beta: float = 1.0         # probe regulariser (Eq. 5); 1 -> ePIE-like
    gamma: float = 0.1        # object regulariser (Eq. 6)
    eps: float = 1.0          # modulus-constraint guard, amplitude units (sqrt photons)
    reg_eps: float = 1e-12    # relative guard of the update denominators
    max_group: int = 0        # 0 = unlimited, 1 = sequential paper algorithm
    update_probe: bool = True


@dataclass
class RefineParams:
    upsample: int = 20        # U
    lr: float = 0.5           # Adam step size, pixels
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    start_iter: int = 0       # first iteration (0-based, global) that refines
    max_step: float = 0.0     # per-axis clamp of one Adam step, 0 = none
    point: str = "A"          # where the error signal is taken (Fig. 2): "A" or "B"


@dataclass
class State:
    O: np.ndarray             # complex128 (Hy, Hx)
    P: np.ndarray             # complex128 (M, W, W)
    pos: np.ndarray           # float64 (N, 2), (y, x) top-left, object pixels
    m: np.ndarray = None
    v: np.ndarray = None
    t: int = 0                # Adam steps taken
    it: int = 0               # iterations run
    last_shift: np.ndarray = None
    gap: np.ndarray = None        # per position: relative best/second gap of the last registration

    @classmethod
    def create(cls, O0, P0, pos0):
        pos = np.asarray(pos0, dtype=np.float64).copy()
        return cls(O=np.asarray(O0, dtype=np.complex128).copy(),
                   P=np.asarray(P0, dtype=np.complex128).copy(), pos=pos,
                   m=np.zeros_like(pos), v=np.zeros_like(pos),
                   last_shift=np.zeros_like(pos), gap=np.ones(len(pos)))


def rpie_group(O, P, I, corners, members, prm, U=0, point="A"):
    """Update O (in place) for every position of one group and P at its end.

    With U > 0 every position's registration shift is measured at ``point``
    (the two switch positions of the refinement scheme, Fig. 2):

    * "A" (XCORR_A): the crop o_j before its update against the refined crop
      o'_j, in the object plane (complex images);
    * "B" (XCORR_B): the model intensity S_j = sum_p |Psi_p|^2 of the current
      estimate against the measured intensity I_j, in the detector plane
      (real images), both in the unshifted layout (a common circular shift
      of the two images does not move a circular correlation peak).

    Returns (error numerator, shifts (len(members), 2), gaps).
    """
    W = P.shape[-1]
    Pint = np.sum(np.abs(P) ** 2, axis=0)
    Pmax = Pint.max()
    obj_den = prm.gamma * Pmax + (1.0 - prm.gamma) * Pint + prm.reg_eps * Pmax
    num = np.zeros_like(P)
    den = np.zeros((W, W))
    omax_sum = 0.0
    err = 0.0
    shifts = np.zeros((len(members), 2))
    gaps = []
    for i, j in enumerate(members):
        cy, cx = int(corners[j][0]), int(corners[j][1])
        o = O[cy:cy + W, cx:cx + W].copy()
        psi = P * o[None]
        Psi = F(psi)
        S = np.sum(np.abs(Psi) ** 2, axis=0)
        Ij = from_detector(np.asarray(I[j], dtype=np.float64))
        sqI = np.sqrt(Ij)
        err += float(np.sum((np.sqrt(S) - sqI) ** 2))
        Psi_c = Psi * (sqI / (np.sqrt(S) + prm.eps))[None]
        D = Finv(Psi_c) - psi
        upd = np.sum(D * np.conj(P), axis=0)
        o_new = o + prm.alpha_O * np.divide(upd, obj_den, out=np.zeros_like(upd), where=obj_den > 0)
        O[cy:cy + W, cx:cx + W] = o_new
        a2 = np.abs(o) ** 2
        om = float(a2.max())
        num += D * np.conj(o)[None]
        den += prm.beta * om + (1.0 - prm.beta) * a2
        omax_sum += om
        if U:
            if point == "A":
                shifts[i], gap = xcorr_peak(o, o_new, U)
            else:
                shifts[i], gap = xcorr_peak(S, Ij, U)
            gaps.append(gap)
    if prm.update_probe:
        pden = np.broadcast_to(den + prm.reg_eps * omax_sum, num.shape)
        P += prm.alpha_P * np.divide(num, pden, out=np.zeros_like(num), where=pden > 0)
    return err, shifts, gaps


def clamp_positions(pos, W, Hy, Hx):
    """Keep every crop box inside the object: 0 <= y <= Hy-W, 0 <= x <= Hx-W."""
    out = pos.copy()
    out[:, 0] = np.clip(out[:, 0], 0.0, Hy - W)
    out[:, 1] = np.clip(out[:, 1], 0.0, Hx - W)
    return out


def iterate(state, I, prm, rfn=None, order=None, groups=None):
    """Run one iteration in place on ``state``; returns the normalised error.

    ``groups`` (optional) overrides the greedy partition, for tests.
    """
    W = state.P.shape[-1]
    refine_on = rfn is not None and state.it >= rfn.start_iter
    U = rfn.upsample if refine_on else 0
    if groups is None:
        groups = greedy_groups(state.pos, W, order, prm.max_group)
    corners = crop_corners(state.pos)
    err = 0.0
    g_meas = np.zeros_like(state.pos)
    for members in groups:
        e, sh, gaps = rpie_group(state.O, state.P, I, corners, members, prm, U,
                                 rfn.point if refine_on else "A")
        err += e
        if refine_on:
            g_meas[members] = -sh
            state.gap[members] = gaps
    if refine_on:
        state.t += 1
        pos, state.m, state.v = adam_step(state.pos, state.m, state.v, g_meas,
                                          state.t, rfn.lr, rfn.b1, rfn.b2,
                                          rfn.eps, rfn.max_step)
        state.pos = clamp_positions(pos, W, *state.O.shape)
        state.last_shift = g_meas
    state.it += 1
    total = float(np.sum(np.asarray(I, dtype=np.float64)))
    return err / total if total > 0 else 0.0


def run(state, I, prm, n_iter, rfn=None, order=None):
    """n_iter iterations; returns the list of per-iteration errors."""
    return [iterate(state, I, prm, rfn, order) for _ in range(n_iter)]
