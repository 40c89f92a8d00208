"""Seeded synthetic ptychography scans (the paper's virtual experiment,
Methods section), shaped like soft-X-ray TwinMic scans.

This module is the ONE input generator shared by the CUDA path and the CPU
oracle.  It holds none of the reconstruction's arithmetic: it builds a true
object, true probe modes, a scan, the simulated detector counts and the
initial guesses, and nothing else.  The detector simulation propagates the
true exit waves with ``torch.fft`` (a library DFT) at the TRUE, sub-pixel
positions (sub-pixel shifts are applied to the probe by the Fourier shift
theorem), adds Poisson noise and clips to uint16.  Neither side of a parity
comparison depends on this step being exact: both consume the counts as given.

Recipe (all randomness from NumPy PCG64 seeded per workload, except the
Poisson draw, which uses a torch.Generator with the same seed):

* object: amplitude = periodic Gaussian-smoothed (sigma 2 px) uniform noise
  min-max mapped to [0.5, 1]; phase = independent smoothed noise mapped to
  [-pi/2, pi/2];
* probe: circular aperture of radius R = 3W/8 times exp(i c (r/R)^2), c = 4 pi
  unless a workload says otherwise (c = 0: a flat-phase, focused probe);
  modes = base x {1, x/R, y/R, xy/R^2, (x^2-y^2)/R^2}, Gram-Schmidt
  orthogonalised, mode powers = occupancy x photons per pattern;
* data: I_j = clip(Poisson(sum_p |DFT(P_p(r - f_j) O(t_j + r))|^2), 0, 65535),
  detector-centred (zero frequency at (W/2, W/2));
* initial guesses: O0 = 1; P0 = each true mode's magnitude blurred
  (sigma 1 px) with its phase scaled by 0.8.
"""
from dataclasses import dataclass, field
import math

import numpy as np
import torch


@dataclass
class Workload:
    name: str
    W: int
    M: int
    Hy: int
    Hx: int
    photons: float
    occupancy: tuple
    pos_true: np.ndarray          # float64 (N, 2) true (y, x) corners
    pos: np.ndarray               # float32 (N, 2) supplied corners
    n_iter: int = 1
    refine: bool = False
    upsample: int = 20
    lr: float = 0.5
    seed: int = 0
    probe_curv: float = 4.0 * math.pi   # probe phase at the aperture edge (radians)
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return len(self.pos)


def _smooth_noise(rng, shape, sigma):
    """Uniform noise smoothed by a periodic Gaussian (FFT convolution)."""
    a = rng.random(shape, dtype=np.float64)
    ky = np.fft.fftfreq(shape[0])[:, None]
    kx = np.fft.rfftfreq(shape[1])[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (ky ** 2 + kx ** 2))
    return np.fft.irfft2(np.fft.rfft2(a) * g, s=shape)


def _minmax(a, lo, hi):
    a0, a1 = a.min(), a.max()
    return lo + (hi - lo) * (a - a0) / (a1 - a0)


def make_object(Hy, Hx, rng):
    amp = _minmax(_smooth_noise(rng, (Hy, Hx), 2.0), 0.5, 1.0)
    ph = _minmax(_smooth_noise(rng, (Hy, Hx), 2.0), -np.pi / 2, np.pi / 2)
    return (amp * np.exp(1j * ph)).astype(np.complex64)


def make_probe(W, M, photons, occupancy, curv=4.0 * math.pi):
    R = 3.0 * W / 8.0
    c = (W - 1) / 2.0
    y, x = np.mgrid[0:W, 0:W].astype(np.float64)
    y, x = y - c, x - c
    r2 = (x * x + y * y) / (R * R)
    base = (r2 <= 1.0) * np.exp(1j * curv * r2)
    shapes = [np.ones_like(x), x / R, y / R, x * y / R ** 2, (x * x - y * y) / R ** 2]
    # further modes (up to 16): more monomials x^a y^b / R^(a+b), by degree
    for a_, b_ in ((2, 0), (2, 1), (1, 2), (3, 0), (0, 3), (2, 2), (3, 1), (1, 3), (4, 0),
                   (0, 4), (3, 2)):
        shapes.append(x ** a_ * y ** b_ / R ** (a_ + b_))
    if M > len(shapes):
        raise ValueError("at most %d probe modes are generated" % len(shapes))
    modes = []
    for k in range(M):
        v = base * shapes[k]
        for u in modes:
            v = v - np.vdot(u, v) * u
        v = v / np.linalg.norm(v)
        modes.append(v)
    occ = np.asarray(occupancy, dtype=np.float64)
    occ = occ / occ.sum()
    P = np.stack([np.sqrt(photons * occ[k]) * modes[k] for k in range(M)])
    return P.astype(np.complex64)


def _blur(a, sigma):
    ky = np.fft.fftfreq(a.shape[-2])[:, None]
    kx = np.fft.fftfreq(a.shape[-1])[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (ky ** 2 + kx ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(a) * g))


def initial_probe(P):
    out = []
    for Pk in P.astype(np.complex128):
        out.append(np.clip(_blur(np.abs(Pk), 1.0), 0, None) * np.exp(1j * 0.8 * np.angle(Pk)))
    return np.stack(out).astype(np.complex64)


def raster(ny, nx, step, offset=(0.0, 0.0)):
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([offset[0] + step * iy.ravel(), offset[1] + step * ix.ravel()], 1).astype(np.float64)


def fermat_spiral(n, scale):
    k = np.arange(n, dtype=np.float64)
    r = scale * np.sqrt(k)
    th = np.deg2rad(137.508) * k
    return np.stack([r * np.sin(th), r * np.cos(th)], 1)


def simulate_counts(O, P, pos_true, photons_seed, device="cpu", chunk=None):
    """Detector counts (N, W, W) uint16 at the true sub-pixel positions.

    Returns (I as a torch uint16... stored as int32 tensor cast) -> numpy/tensor
    on ``device``, plus the clipped fraction.
    """
    dev = torch.device(device)
    M, W, _ = P.shape
    N = len(pos_true)
    Ot = torch.as_tensor(O, device=dev)
    FP = torch.fft.fft2(torch.as_tensor(P, device=dev))             # (M, W, W)
    u = torch.fft.fftfreq(W, device=dev, dtype=torch.float64)        # cycles / px
    it = np.floor(pos_true).astype(np.int64)
    fr = torch.as_tensor(pos_true - it, device=dev)
    it_t = torch.as_tensor(it, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(photons_seed))
    if chunk is None:
        chunk = max(1, int(2 ** 28 // (M * W * W * 8)))
        if dev.type == "cpu":
            chunk = max(1, chunk // 4)
    out = torch.empty((N, W, W), dtype=torch.int32, device=dev)
    clipped = 0
    ar = torch.arange(W, device=dev)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        rows = (it_t[s:e, 0, None] + ar[None, :])                    # (B, W)
        cols = (it_t[s:e, 1, None] + ar[None, :])
        o = Ot[rows[:, :, None], cols[:, None, :]]                   # (B, W, W)
        ph = torch.exp(-2j * math.pi * (fr[s:e, 0, None, None] * u[None, :, None]
                                        + fr[s:e, 1, None, None] * u[None, None, :]))
        Ps = torch.fft.ifft2(FP[None] * ph[:, None].to(FP.dtype))    # P(r - f)
        Psi = torch.fft.fft2(Ps * o[:, None], norm="ortho")
        lam = torch.fft.fftshift((Psi.real ** 2 + Psi.imag ** 2).sum(1), dim=(-2, -1))
        cnt = torch.poisson(lam.to(torch.float32), generator=gen)
        clipped += int((cnt > 65535).sum().item())
        out[s:e] = cnt.clamp_(0, 65535).to(torch.int32)
    return out, clipped / float(N * W * W)


def build(wl, device="cpu"):
    """Materialise a workload: returns a dict of arrays (host numpy unless the
    counts were simulated on a CUDA device, then ``I`` is a CUDA uint16 tensor
    view stored as int16 bits -- see ``counts_u16``)."""
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    O = make_object(wl.Hy, wl.Hx, rng)
    P = make_probe(wl.W, wl.M, wl.photons, wl.occupancy, wl.probe_curv)
    cnt, clipped = simulate_counts(O, P, wl.pos_true, wl.seed, device=device)
    return dict(O_true=O, P_true=P, I=cnt, clipped=clipped,
                O0=np.ones((wl.Hy, wl.Hx), dtype=np.complex64),
                P0=initial_probe(P), pos=wl.pos.astype(np.float32).copy(),
                pos_true=wl.pos_true.copy())


def counts_u16(cnt):
    """int32 counts tensor -> numpy uint16 (host) or torch uint16 (device)."""
    if cnt.device.type == "cpu":
        return cnt.numpy().astype(np.uint16)
    return cnt.to(torch.uint16)


# ---------------------------------------------------------------- workloads
def _occ(M):
    if M == 1:
        return (1.0,)
    if M == 2:
        return (0.8, 0.2)
    if M == 3:
        return (0.7, 0.2, 0.1)
    return tuple(0.5 ** k for k in range(M))


def plain_rpie_64(seed=1000):
    """64x64 patterns, one mode, 10x10 raster at step 8 (corner offset 12),
    object 160x160, 1e5 photons, 20 iterations."""
    pos = raster(10, 10, 8.0, (12.0, 12.0))
    return Workload("rpie_w64_m1_n100", 64, 1, 160, 160, 1e5, (1.0,), pos,
                    pos.astype(np.float32), n_iter=20, seed=seed)


def refine_128(seed=2000):
    """128x128 patterns, 3 modes (0.7/0.2/0.1), 40x40 raster at step 12 with
    U(+-2) jitter, U(+-3) error on the supplied positions, object 700x700,
    1e6 photons, 100 iterations with U = 20, lr = 0.5."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    W, H = 128, 700
    base = raster(40, 40, 12.0)
    ext = 39 * 12 + W
    off = (H - ext) / 2.0
    true = base + off + rng.uniform(-2, 2, base.shape)
    sup = np.clip(true + rng.uniform(-3, 3, base.shape), 0, H - W)
    return Workload("refine_w128_m3_n1600", W, 3, H, H, 1e6, _occ(3), true,
                    sup.astype(np.float32), n_iter=100, refine=True, upsample=20,
                    lr=0.5, seed=seed)


def spiral_256(seed=3000, n=10000, spread=1.0):
    """256x256 patterns, 5 modes, Fermat spiral of 10^4 positions
    (r = 12.5 sqrt(k), 137.508 deg), object 2800x2800, 1e6 photons.
    spread > 1 scales the radii by sqrt(spread): n positions over the extent
    n * spread would cover (a sparser scan whose disjoint groups have the
    size of the denser scan's with n * spread positions)."""
    W, H = 256, 2800
    sp = fermat_spiral(n, 12.5 * math.sqrt(spread))
    c = (H - W) / 2.0
    true = sp + c
    name = "spiral_w256_m5_n%d" % n + ("" if spread == 1.0 else "_spread%g" % spread)
    return Workload(name, W, 5, H, H, 1e6, _occ(5), true,
                    true.astype(np.float32), n_iter=1, seed=seed)


def sweep_256(seed=5000, ny=200, nx=200):
    """256x256 patterns, 4 modes, 200x200 jittered raster at step 16 (+-2),
    +-2 px supplied error, object 8192x8192, 1e7 photons, refinement on."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    W, H = 256, 8192
    base = raster(ny, nx, 16.0)
    ext = np.array([(ny - 1) * 16 + W, (nx - 1) * 16 + W], dtype=np.float64)
    off = (H - ext) / 2.0
    true = base + off + rng.uniform(-2, 2, base.shape)
    sup = np.clip(true + rng.uniform(-2, 2, base.shape), 0, H - W)
    return Workload("sweep_w256_m4_n%d" % (ny * nx), W, 4, H, H, 1e7, _occ(4), true,
                    sup.astype(np.float32), n_iter=1, refine=True, seed=seed)


def batch_problem(p, seed0=4000):
    """Problem p of the 64-problem uneven batch: W in {64,96,128,192},
    N ~ U[50, 900], M ~ U{1..3}, raster step W/8 with +-2 jitter, object =
    scan extent + 64 px."""
    rng = np.random.Generator(np.random.PCG64(seed0 + p))
    W = int(rng.choice([64, 96, 128, 192]))
    N = int(rng.integers(50, 901))
    M = int(rng.integers(1, 4))
    step = W / 8.0
    nx = int(math.ceil(math.sqrt(N)))
    ny = int(math.ceil(N / nx))
    base = raster(ny, nx, step)[:N]
    ext = np.array([(ny - 1) * step + W, (nx - 1) * step + W])
    H = (np.ceil(ext) + 64).astype(int)
    true = base + 32.0 + rng.uniform(-2, 2, base.shape)
    true = np.clip(true, 0, np.array([H[0] - W - 1, H[1] - W - 1]))
    return Workload("batch%02d_w%d_m%d_n%d" % (p, W, M, N), W, M, int(H[0]), int(H[1]),
                    1e6, _occ(M), true, true.astype(np.float32), n_iter=50,
                    seed=seed0 + p)


def tiny(W=32, M=2, ny=5, nx=5, step=6.0, seed=77, photons=1e5, jitter=0.0, err=0.0):
    """Small case for fast oracle/parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    base = raster(ny, nx, step)
    ext = np.array([(ny - 1) * step + W, (nx - 1) * step + W])
    H = (np.ceil(ext) + 16).astype(int)
    true = base + 8.0 + rng.uniform(-jitter, jitter, base.shape)
    sup = np.clip(true + rng.uniform(-err, err, base.shape), 0,
                  np.array([H[0] - W, H[1] - W]))
    return Workload("tiny_w%d_m%d" % (W, M), W, M, int(H[0]), int(H[1]), photons,
                    _occ(M), true, sup.astype(np.float32), seed=seed)
