"""Pins of the XCORR_A registration and the Adam controller: exact recovery of
shifts applied by the Fourier shift theorem, agreement with a zero-padded
(U W)^2 inverse FFT (brute force upsampling), Adam closed forms, and the sign
of the whole refinement loop on consistent data."""
import numpy as np
import pytest

from oracle import adam, model, registration, rpie


def smooth_patch(W, rng, sigma=2.0):
    a = rng.normal(size=(W, W)) + 1j * rng.normal(size=(W, W))
    k = np.fft.fftfreq(W)
    g = np.exp(-2 * (np.pi * sigma) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    return np.fft.ifft2(np.fft.fft2(a) * g)


def shifted(a, d):
    """b(r) = a(r + d), circular, by the Fourier shift theorem with signed freqs."""
    W = a.shape[0]
    f = registration.signed_freqs(W)
    ph = np.exp(2j * np.pi * (f[:, None] * d[0] + f[None, :] * d[1]) / W)
    return np.fft.ifft2(np.fft.fft2(a) * ph)


DT = [np.float32, np.float64]   # resolution of the argmax decision


@pytest.mark.parametrize("dt", DT)
@pytest.mark.parametrize("d", [(3.0, -5.0), (0.0, 0.0), (-7.0, 11.0), (31.0, -32.0)])
def test_integer_shifts_exact(d, dt):
    rng = np.random.default_rng(1)
    a = smooth_patch(64, rng)
    s, _ = registration.xcorr_peak(a, shifted(a, np.array(d)), 20, dt)
    # equal modulo the patch size; the coarse peak lies in [-W/2, W/2)
    np.testing.assert_allclose(np.mod(s + np.array(d), 64), 0.0, atol=1e-12)
    assert np.all((s >= -32) & (s < 32))


@pytest.mark.parametrize("dt", DT)
@pytest.mark.parametrize("k", [(1, 3), (-7, 13), (19, -19), (-31, 2)])
def test_grid_subpixel_shifts_exact(k, dt):
    U = 20
    rng = np.random.default_rng(2)
    a = smooth_patch(64, rng)
    d = np.array([2 + k[0] / U, -1 + k[1] / U])
    s, _ = registration.xcorr_peak(a, shifted(a, d), U, dt)
    np.testing.assert_allclose(s, -d, atol=1e-9)


def test_random_shifts_within_half_a_fine_step():
    U = 20
    rng = np.random.default_rng(3)
    for _ in range(10):
        a = smooth_patch(48, rng)
        d = rng.uniform(-6, 6, 2)
        s, _ = registration.xcorr_peak(a, shifted(a, d), U)
        assert np.all(np.abs(s + d) <= 0.5 / U + 1e-9)


def test_matches_zero_padded_brute_force():
    W, U = 16, 4
    rng = np.random.default_rng(4)
    for _ in range(5):
        a = smooth_patch(W, rng, sigma=1.0)
        b = smooth_patch(W, rng, sigma=1.0) * 0.3 + shifted(a, rng.uniform(-3, 3, 2))
        X = np.fft.fft2(b) * np.conj(np.fft.fft2(a))
        # place X at its signed frequencies on a (U W)^2 grid; the inverse FFT
        # then samples c(r) at r = n / U over the whole patch
        big = np.zeros((U * W, U * W), complex)
        f = registration.signed_freqs(W).astype(int)
        big[np.ix_(f % (U * W), f % (U * W))] = X
        c = np.abs(np.fft.ifft2(big)) ** 2
        n = np.unravel_index(np.argmax(c), c.shape)
        want = np.array([registration.wrap(n[0], U * W), registration.wrap(n[1], U * W)]) / U
        s, _ = registration.xcorr_peak(a, b, U, np.float64)
        np.testing.assert_allclose(s, want, atol=1e-12)


def test_adam_constant_gradient_closed_form():
    g = np.array([[0.3, -2.0], [0.0, 1e-3]])
    pos = np.zeros_like(g)
    m = np.zeros_like(g)
    v = np.zeros_like(g)
    for t in range(1, 8):
        new, m, v = adam.adam_step(pos, m, v, g, t, lr=0.5)
        # bias-corrected moments are g and g^2, so each step is lr g / (|g| + eps)
        np.testing.assert_allclose(new - pos, 0.5 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
        pos = new
    new, _, _ = adam.adam_step(pos, np.zeros_like(g), np.zeros_like(g), np.zeros_like(g), 1, lr=0.5)
    np.testing.assert_array_equal(new, pos)
    new, _, _ = adam.adam_step(pos, m, v, 100 * g, 8, lr=0.5, max_step=0.25)
    assert np.all(np.abs(new - pos) <= 0.25)


def test_refinement_moves_an_offset_position_toward_the_truth():
    # Consistent noise-free data; object and probe start at the truth and the
    # probe is held; one supplied position is (1.5, -1) px off.  XCORR_A + Adam
    # must reduce that error on both axes.
    rng = np.random.default_rng(5)
    W, H = 32, 64
    O = smooth_patch(H, rng, sigma=1.5)
    O = 0.6 + 0.4 * np.abs(O) / np.abs(O).max() * np.exp(1j * np.angle(O))
    P = smooth_patch(W, rng, sigma=1.0)
    true = np.array([[10.0, 12.0], [20.0, 8.0], [14.0, 22.0]])
    I = model.model_intensities(O, P[None], true)
    sup = true.copy()
    sup[0] += np.array([1.5, -1.0])
    st = rpie.State.create(O, P[None], sup)
    prm = rpie.RPIEParams(alpha_O=1.0, update_probe=False, gamma=0.5, eps=1e-6)
    rfn = rpie.RefineParams(upsample=20, lr=0.3)
    e0 = np.abs(st.pos[0] - true[0])
    for _ in range(4):
        rpie.iterate(st, I, prm, rfn)
    e1 = np.abs(st.pos[0] - true[0])
    assert np.all(e1 < e0)


def _shift_real(a, d):
    """Real image a(r + d), circular, by the Fourier shift theorem."""
    return np.real(shifted(a, d))


@pytest.mark.parametrize("d", [(1.0, -2.0), (0.35, 0.8), (-1.55, 0.05)])
def test_xcorr_b_measures_the_detector_plane_shift(d):
    """XCORR_B correlates the model intensity S_j with the measured I_j.  When
    the measured pattern is the model's own intensity moved by d (a 1/U-grid
    shift), one refining group must report g_j = d exactly; a swapped pair
    of images (planted) would report -d."""
    U = 20
    rng = np.random.default_rng(6)
    W, H = 32, 40
    O = 0.7 + 0.3 * smooth_patch(H, rng, sigma=2.0)
    P = smooth_patch(W, rng, sigma=3.0)[None] * 40.0
    corner = np.array([[3, 5]])
    S = model.model_intensities(O, P, corner)[0]            # detector layout
    d = np.array(d)
    I = np.clip(_shift_real(S, d), 0.0, None)[None]   # counts are non-negative
    prm = rpie.RPIEParams(alpha_O=0.0, alpha_P=0.0)
    _, sh, gaps = rpie.rpie_group(O.copy(), P.copy(), I, corner, [0], prm, U, point="B")
    np.testing.assert_allclose(-sh[0], d, atol=1e-9)
    # consistent data: XCORR_B finds no shift, and neither does XCORR_A (with
    # zero step sizes it compares o_j with itself)
    for point in ("A", "B"):
        _, sh0, _ = rpie.rpie_group(O.copy(), P.copy(), S[None], corner, [0], prm, U, point=point)
        np.testing.assert_allclose(sh0[0], 0.0, atol=1e-12)
