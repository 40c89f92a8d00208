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


@pytest.mark.parametrize("W,M,ny,nx,step", [(64, 3, 4, 4, 10.0), (256, 5, 2, 3, 48.0)])
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
