"""pty_model_intensities_noalloc: the allocation-free variant of the model
intensity computation, for callers that may not allocate device memory (for
example code running inside another framework's memory pool, or a loop that
must never stall on the allocator).  Its output must equal the handle-based
pty_model_intensities within the tolerance of the other parity tests, on two
calls in a row (the shared fixed scratch keeps the previous call's contents).
Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from helpers import build, rel_l2
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def noalloc(O, P, pos, W, out):
    import torch
    from paper_2205_04295_b300 import pty
    Hy, Hx = O.shape
    M = P.shape[0]
    N = pos.shape[0]
    return pty.lib().pty_model_intensities_noalloc(
        O.data_ptr(), Hy, Hx, P.data_ptr(), M, W, pos.data_ptr(), N, out.data_ptr(),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# every FFT split the kernels take: 32 = 8x4, 64 = 8x8, 96 = 8x12, 128 = 16x8,
# 192 = 16x12, 256 = 16x16 (unequal splits use different lane counts per step)
@pytest.mark.parametrize("W,M,ny,nx,step", [(32, 2, 4, 4, 6.0), (64, 3, 4, 4, 10.0),
                                            (96, 2, 3, 3, 20.0), (128, 3, 3, 3, 24.0),
                                            (192, 2, 2, 3, 40.0), (256, 5, 2, 3, 48.0)])
def test_noalloc_matches_handle_path_on_two_calls(W, M, ny, nx, step):
    import torch
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=W, M=M, ny=ny, nx=nx, step=step, seed=21, photons=1e6)
    d = build(wl)
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    prob.run(1)                                   # a non-trivial object and probe
    ref = prob.model_intensities(device=True)
    O, P, pos = prob.object(), prob.probe(), prob.positions()
    for _ in range(2):
        out = torch.full_like(ref, -1.0)
        assert noalloc(O, P, pos, W, out) == pty.PTY_OK, pty.lib().pty_last_error()
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= TOL


def test_noalloc_rejects_patterns_beyond_its_scratch():
    import torch
    from paper_2205_04295_b300 import pty
    W, M = 256, 13                                # 13 * 256^2 * 8 B > 6 MiB
    O = torch.ones((300, 300), dtype=torch.complex64, device="cuda")
    P = torch.ones((M, W, W), dtype=torch.complex64, device="cuda")
    pos = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    out = torch.empty((1, W, W), dtype=torch.float32, device="cuda")
    assert noalloc(O, P, pos, W, out) == pty.PTY_EINVAL
    assert b"no-allocation scratch" in pty.lib().pty_last_error()


def test_noalloc_box_outside_object_is_nan_only_there():
    """A position whose crop box leaves the object yields a NaN pattern; the
    other patterns of the same call are unaffected."""
    import torch
    from oracle import model
    from paper_2205_04295_b300 import pty
    W, M = 64, 2
    wl = synth.tiny(W=W, M=M, ny=3, nx=3, step=10.0, seed=22)
    d = build(wl)
    pos = np.asarray(d["pos"], dtype=np.float32).copy()
    pos[4] = (wl.Hy - W + 3.0, 1.0)                  # box runs off the bottom edge
    O = torch.as_tensor(np.asarray(d["O_true"], dtype=np.complex64), device="cuda")
    P = torch.as_tensor(np.asarray(d["P_true"], dtype=np.complex64), device="cuda")
    pos_d = torch.as_tensor(pos, device="cuda")
    for _ in range(2):
        out = torch.zeros((len(pos), W, W), dtype=torch.float32, device="cuda")
        assert noalloc(O, P, pos_d, W, out) == pty.PTY_OK, pty.lib().pty_last_error()
        torch.cuda.synchronize()
        h = out.cpu().numpy()
        assert np.isnan(h[4]).all()
        keep = np.arange(len(pos)) != 4
        assert np.isfinite(h[keep]).all()
        ref = model.model_intensities(d["O_true"], d["P_true"], pos[keep])
        assert rel_l2(h[keep], ref) <= TOL


def test_noalloc_largest_accepted_mode_count():
    """256x256 with 12 modes: one pattern fills the whole fixed scratch
    (12 * 256^2 * 8 bytes = 6 MiB), so every pattern is its own chunk."""
    import torch
    from oracle import model
    from paper_2205_04295_b300 import pty
    W, M, N = 256, 12, 3
    rng = np.random.default_rng(23)
    Hy = Hx = 300
    O = (rng.uniform(0.5, 1.0, (Hy, Hx)) * np.exp(1j * rng.uniform(-1, 1, (Hy, Hx)))).astype(np.complex64)
    P = (rng.normal(size=(M, W, W)) + 1j * rng.normal(size=(M, W, W))).astype(np.complex64)
    pos = rng.uniform(0.0, Hy - W - 1.0, (N, 2)).astype(np.float32)
    ref = model.model_intensities(O, P, pos)
    Od, Pd, posd = (torch.as_tensor(a, device="cuda") for a in (O, P, pos))
    for _ in range(2):
        out = torch.full((N, W, W), -1.0, dtype=torch.float32, device="cuda")
        assert noalloc(Od, Pd, posd, W, out) == pty.PTY_OK, pty.lib().pty_last_error()
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= TOL
