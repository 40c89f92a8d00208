"""The line FFTs of the library (the building block of every pass) against
NumPy's FFT, for every supported W, forward and inverse."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W", [32, 64, 96, 128, 192, 256])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2_matches_numpy(W, inverse):
    import torch
    from paper_2205_04295_b300 import pty
    rng = np.random.default_rng(W)
    x = (rng.normal(size=(3, W, W)) + 1j * rng.normal(size=(3, W, W))).astype(np.complex64)
    t = torch.from_numpy(x).cuda()
    pty.fft2_(t, inverse=inverse)
    got = t.cpu().numpy().astype(np.complex128)
    xx = x.astype(np.complex128)
    want = np.fft.ifft2(xx) * W * W if inverse else np.fft.fft2(xx)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 2e-6, err


def test_fp32_peak_measurement_is_plausible():
    """The FMA-chain measurement lands between a third of and just above the
    nominal peak (148 SMs x 128 lanes x 2 flop x 2.032 GHz = 77.0 TFLOP/s;
    the clock may sit below its maximum)."""
    from paper_2205_04295_b300 import pty
    t = pty.measure_fp32_peak()
    assert 25.0 < t < 80.0
