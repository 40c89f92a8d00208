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
