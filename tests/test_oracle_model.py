"""Pins of the oracle's DFT and forward model against definitions that do not
go through the oracle's own code: a brute-force O(N^4) DFT, Parseval, closed
forms for constant inputs."""
import numpy as np
import pytest

from oracle import model


def brute_dft2(x):
    """Unitary 2-D DFT written as the double sum of its definition."""
    H, W = x.shape
    out = np.zeros((H, W), dtype=np.complex128)
    for u in range(H):
        for v in range(W):
            s = 0j
            for y in range(H):
                for z in range(W):
                    s += x[y, z] * np.exp(-2j * np.pi * (u * y / H + v * z / W))
            out[u, v] = s / np.sqrt(H * W)
    return out


@pytest.mark.parametrize("n", [4, 6, 8, 12])
def test_fft_matches_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    np.testing.assert_allclose(model.F(x), brute_dft2(x), atol=1e-12)


def test_fft_parseval_and_inverse():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 32, 32)) + 1j * rng.normal(size=(3, 32, 32))
    X = model.F(x)
    assert np.allclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2), rtol=1e-13)
    np.testing.assert_allclose(model.Finv(X), x, atol=1e-14 * 10)


def test_detector_layout_puts_dc_at_centre():
    W = 16
    I = model.model_intensity_unshifted(np.ones((1, W, W), complex), np.ones((W, W), complex))
    stored = model.to_detector(I)
    assert np.argmax(stored) == (W // 2) * W + W // 2
    assert np.isclose(stored[W // 2, W // 2], W * W)      # |sum 1|^2 / W^2 * W^2


def test_crop_corner_rounding():
    pos = np.array([[2.5, 2.49], [0.0, 0.5], [7.999, 3.5000001]])
    np.testing.assert_array_equal(model.crop_corners(pos), [[3, 2], [0, 1], [8, 4]])


def test_constant_object_single_mode_closed_form():
    rng = np.random.default_rng(2)
    W = 16
    P = rng.normal(size=(1, W, W)) + 1j * rng.normal(size=(1, W, W))
    c = 0.7 * np.exp(0.3j)
    O = np.full((40, 40), c)
    I = model.model_intensities(O, P, np.array([[3.0, 5.0]]))[0]
    expect = np.abs(c) ** 2 * np.abs(brute_dft2(P[0])) ** 2
    np.testing.assert_allclose(model.from_detector(I), expect, rtol=1e-12)


def test_per_pattern_parseval_and_incoherent_mode_sum():
    rng = np.random.default_rng(3)
    W, M = 16, 3
    P = rng.normal(size=(M, W, W)) + 1j * rng.normal(size=(M, W, W))
    O = rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))
    pos = np.array([[2.2, 7.7], [10.0, 0.0]])
    I = model.model_intensities(O, P, pos)
    for j, c in enumerate(model.crop_corners(pos)):
        o = O[c[0]:c[0] + W, c[1]:c[1] + W]
        assert np.isclose(I[j].sum(), np.sum(np.abs(P * o) ** 2), rtol=1e-12)
        single = sum(model.from_detector(model.model_intensities(O, P[k:k + 1], pos[j:j + 1])[0])
                     for k in range(M))
        np.testing.assert_allclose(model.from_detector(I[j]), single, rtol=1e-12)
        coherent = np.abs(brute_dft2(np.sum(P * o, axis=0))) ** 2
        assert not np.allclose(model.from_detector(I[j]), coherent, rtol=1e-3)
