"""Pins of the oracle gradient: central finite differences in FP64 of every
real and imaginary component (of a sample of object pixels, all probe entries
of one mode, and all positions) on a reduced problem whose fractional
positions keep clear of bilinear kinks."""
import numpy as np

from oracle import grad


def reduced_problem(seed=0):
    rng = np.random.default_rng(seed)
    W, M, H = 16, 2, 32
    O = (0.5 + 0.5 * rng.random((H, H))) * np.exp(1j * rng.uniform(-1, 1, (H, H)))
    P = rng.normal(size=(M, W, W)) + 1j * rng.normal(size=(M, W, W))
    base = np.array([[y, x] for y in (2.0, 7.0, 12.0) for x in (3.0, 8.0, 13.0)])
    pos = base + rng.uniform(0.2, 0.8, base.shape)
    I = rng.uniform(0, 40, size=(len(pos), W, W))
    return O, P, pos, I


def central(f, x0, h):
    return (f(x0 + h) - f(x0 - h)) / (2 * h)


def test_gradient_matches_central_differences():
    O, P, pos, I = reduced_problem()
    for delta in (0.0, 1.0):
        check_fd(O, P, pos, I, delta)


def check_fd(O, P, pos, I, delta):
    L, gO, gP, gpos = grad.loss_and_grad(O, P, pos, I, delta=delta)
    assert np.isclose(L, grad.loss(O, P, pos, I, delta=delta))
    h = 1e-6
    rng = np.random.default_rng(1)
    pix = [tuple(p) for p in rng.integers(2, 30, size=(12, 2))] + [(2, 3), (18, 21)]
    for (y, x) in pix:
        for comp, unit in ((np.real, 1.0), (np.imag, 1j)):
            def f(t):
                Oc = O.copy()
                Oc[y, x] += t * unit
                return grad.loss(Oc, P, pos, I, delta=delta)
            fd = central(f, 0.0, h)
            assert np.isclose(fd, comp(gO[y, x]), rtol=1e-5, atol=1e-5 * (1 + abs(fd)))
    for (k, y, x) in [(0, 3, 4), (1, 8, 8), (0, 15, 0), (1, 0, 15)]:
        for comp, unit in ((np.real, 1.0), (np.imag, 1j)):
            def f(t):
                Pc = P.copy()
                Pc[k, y, x] += t * unit
                return grad.loss(O, Pc, pos, I, delta=delta)
            fd = central(f, 0.0, h)
            assert np.isclose(fd, comp(gP[k, y, x]), rtol=1e-5, atol=1e-5 * (1 + abs(fd)))
    for j in range(len(pos)):
        for ax in range(2):
            def f(t):
                pc = pos.copy()
                pc[j, ax] += t
                return grad.loss(O, P, pc, I, delta=delta)
            fd = central(f, 0.0, h)
            assert np.isclose(fd, gpos[j, ax], rtol=1e-5, atol=1e-5 * (1 + abs(fd)))


def test_integer_positions_reduce_to_plain_crop():
    O, P, pos, I = reduced_problem(2)
    pos = np.floor(pos)
    o, dy, dx, (iy, ix), _ = grad.bilinear_crop(O, pos[0], 16)
    np.testing.assert_array_equal(o, O[iy:iy + 16, ix:ix + 16])


def test_fd_on_a_32x32_crop_of_the_spiral_workload():
    """FP64 central differences at the 256x256 / 5-mode / 10^4-position spiral
    geometry: an object pixel of a 32x32 crop at the scan centre (the loss
    restricted to the patches whose bilinear box covers the crop) and two
    positions (each moves only its own patch's loss)."""
    from paper_2205_04295_b300 import synth
    wl = synth.spiral_256()
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    O = synth.make_object(wl.Hy, wl.Hx, rng).astype(np.complex128)
    P = synth.initial_probe(synth.make_probe(wl.W, wl.M, wl.photons, wl.occupancy))
    pos = np.floor(wl.pos.astype(np.float64)) + 0.37
    y0 = x0 = 1390
    fl = np.floor(pos)
    cover = np.nonzero((fl[:, 0] <= y0 + 31) & (fl[:, 0] + wl.W >= y0) &
                       (fl[:, 1] <= x0 + 31) & (fl[:, 1] + wl.W >= x0))[0]
    cnt, _ = synth.simulate_counts(O.astype(np.complex64), synth.make_probe(wl.W, wl.M, wl.photons, wl.occupancy),
                                   wl.pos_true[cover], 5)
    I = cnt.numpy().astype(np.uint16)
    sub = pos[cover]
    L, gO, gP, gpos = grad.loss_and_grad(O, P, sub, I, delta=1.0)
    h = 1e-6
    yy, xx = y0 + 13, x0 + 21
    for comp, unit in ((np.real, 1.0), (np.imag, 1j)):
        def f(t):
            Oc = O.copy()
            Oc[yy, xx] += t * unit
            return grad.loss(Oc, P, sub, I, delta=1.0)
        fd = central(f, 0.0, h)
        assert np.isclose(fd, comp(gO[yy, xx]), rtol=1e-5, atol=1e-6 * abs(L))
    for k in (0, len(sub) - 1):
        for ax in range(2):
            def f(t):
                pc = sub[k:k + 1].copy()
                pc[0, ax] += t
                return grad.loss(O, P, pc, I[k:k + 1], delta=1.0)
            fd = central(f, 0.0, h)
            assert np.isclose(fd, gpos[k, ax], rtol=1e-5, atol=1e-6 * abs(L))
