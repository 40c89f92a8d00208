"""The CUDA forward model + adjoint against the FP64 oracle gradient (which is
itself pinned by central finite differences), through the C ABI and through
the torch.autograd.Function."""
import numpy as np
import pytest

from helpers import build, rel_l2, to_host
from oracle import grad, model
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu


def state(wl, d, seed=5):
    """A non-trivial point: the true object, the initial probe, fractional
    positions (supplied positions + a fractional offset away from kinks)."""
    rng = np.random.default_rng(seed)
    pos = np.floor(d["pos"].astype(np.float64)) + rng.uniform(0.2, 0.8, d["pos"].shape)
    return d["O_true"], d["P0"], pos.astype(np.float32)


def gpu_grad(wl, d, O, P, pos, delta=1.0):
    import torch
    from paper_2205_04295_b300 import pty
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (O, P, pos)]
    out = prob.loss_grad(*t, delta=delta)
    return prob, t, [to_host(x) for x in out]


@pytest.mark.parametrize("W,M,ny,nx,step", [(32, 2, 4, 4, 6.0), (64, 3, 4, 4, 20.0), (256, 5, 2, 2, 64.0)])
def test_gradient_matches_oracle(W, M, ny, nx, step):
    wl = synth.tiny(W=W, M=M, ny=ny, nx=nx, step=step, seed=41, photons=1e6)
    wl.Hy += 2
    wl.Hx += 2
    d = build(wl)
    O, P, pos = state(wl, d)
    prob, _, (L, gO, gP, gpos) = gpu_grad(wl, d, O, P, pos)
    Lo, gOo, gPo, gposo = grad.loss_and_grad(O, P, pos.astype(np.float64), d["I"], delta=1.0)
    assert abs(L[0] - Lo) <= 1e-5 * Lo
    assert rel_l2(gO, gOo) <= 1e-5
    assert rel_l2(gP, gPo) <= 1e-5
    assert rel_l2(gpos, gposo) <= 1e-4


def test_loss_only_and_repeatability():
    import torch
    wl = synth.tiny(W=64, M=2, ny=3, nx=3, step=12.0, seed=42, photons=1e6)
    wl.Hy += 2
    wl.Hx += 2
    d = build(wl)
    O, P, pos = state(wl, d)
    prob, t, (L, gO, gP, gpos) = gpu_grad(wl, d, O, P, pos)
    L2 = to_host(prob.loss(*t))
    np.testing.assert_array_equal(L, L2)
    again = [to_host(x) for x in prob.loss_grad(*t)]
    for a, b in zip((L, gO, gP, gpos), again):
        np.testing.assert_array_equal(a, b)


def test_autograd_function_and_descent_step():
    import torch
    from paper_2205_04295_b300.autograd import amplitude_loss
    wl = synth.tiny(W=64, M=2, ny=3, nx=3, step=12.0, seed=43, photons=1e6)
    wl.Hy += 2
    wl.Hx += 2
    d = build(wl)
    O, P, pos = state(wl, d)
    prob, t, (L, gO, gP, gpos) = gpu_grad(wl, d, O, P, pos)
    Ot, Pt, post = [x.clone().requires_grad_(True) for x in t]
    loss = amplitude_loss(prob, Ot, Pt, post)
    loss.backward()
    np.testing.assert_array_equal(to_host(Ot.grad), gO)
    np.testing.assert_array_equal(to_host(Pt.grad), gP)
    np.testing.assert_array_equal(to_host(post.grad), gpos)
    with torch.no_grad():
        step = 1e-4 * float(torch.linalg.vector_norm(Ot)) / float(torch.linalg.vector_norm(Ot.grad))
        O2 = Ot - step * Ot.grad
    assert float(amplitude_loss(prob, O2.contiguous(), Pt.detach(), post.detach())) < float(loss)


def test_error_on_position_outside():
    import torch
    from paper_2205_04295_b300 import pty
    wl = synth.tiny(W=32, M=1, ny=2, nx=2, step=6.0, seed=44)
    d = build(wl)
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    pos = torch.from_numpy(d["pos"]).cuda()
    pos[0, 0] = wl.Hy - wl.W + 0.5        # rows floor(y) .. floor(y) + W: outside
    with pytest.raises(pty.PtyError) as e:
        prob.loss(torch.from_numpy(d["O0"]).cuda(), torch.from_numpy(d["P0"]).cuda(), pos)
    assert e.value.code == pty.PTY_EDATA


def test_full_size_spiral_sampled_gradient():
    """256x256, 5 modes, 10^4 positions, 2800^2 object: one full gradient call
    in the benchmark's configuration, then sampled checks against the oracle:
    dL/dpos of 12 positions (each depends on its own patch only), and dL/dO on
    a 32x32 crop (the oracle sums the patches whose bilinear box covers it)."""
    import torch
    from paper_2205_04295_b300 import pty
    wl = synth.spiral_256()
    d = synth.build(wl, device="cuda")
    I = synth.counts_u16(d["I"])
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
    prob.set_data(I, torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["O0"]).cuda(),
                  torch.from_numpy(d["P0"]).cuda())
    O = torch.from_numpy(d["O_true"]).cuda()
    P = torch.from_numpy(d["P0"]).cuda()
    pos = torch.from_numpy(d["pos"]).cuda()
    L, gO, gP, gpos = [to_host(x) for x in prob.loss_grad(O, P, pos)]
    Ih = to_host(I.to(torch.int32))
    posd = d["pos"].astype(np.float64)
    rng = np.random.default_rng(0)
    for j in rng.choice(wl.N, 12, replace=False):
        _, _, _, gj = grad.loss_and_grad(d["O_true"], d["P0"], posd[j:j + 1], Ih[j:j + 1], delta=1.0)
        np.testing.assert_allclose(gpos[j], gj[0], rtol=2e-4, atol=2e-4 * np.abs(gj).max())
    y0, x0 = 1390, 1390
    fl = np.floor(posd)
    cover = np.nonzero((fl[:, 0] <= y0 + 31) & (fl[:, 0] + wl.W >= y0) &
                       (fl[:, 1] <= x0 + 31) & (fl[:, 1] + wl.W >= x0))[0]
    assert len(cover) > 20
    _, gOo, _, _ = grad.loss_and_grad(d["O_true"], d["P0"], posd[cover], Ih[cover], delta=1.0)
    assert rel_l2(gO[y0:y0 + 32, x0:x0 + 32], gOo[y0:y0 + 32, x0:x0 + 32]) <= 1e-5


def test_gradient_under_non_default_tilings():
    """Every buffer indexed by row block must fit the smallest row block."""
    wl = synth.tiny(W=64, M=3, ny=4, nx=4, step=20.0, seed=45, photons=1e6)
    wl.Hy += 2
    wl.Hx += 2
    d = build(wl)
    O, P, pos = state(wl, d)
    prob, t, ref = gpu_grad(wl, d, O, P, pos)
    for R, ppc, CB in ((1, 8, 4), (1, 1, 2), (2, 4, 16)):
        prob.set_tiling(R, ppc, CB, 0)
        got = [to_host(x) for x in prob.loss_grad(*t)]
        assert abs(got[0][0] - ref[0][0]) <= 1e-5 * abs(ref[0][0])
        for a, b in zip(got[1:], ref[1:]):
            assert rel_l2(a, b) <= 1e-5


def test_chunks_that_split_groups():
    """The per-patch passes take chunks of the group-ordered positions that
    need not end where a group ends (here 3 patches a chunk); the scatter
    into dL/dO then runs per group part.  dL/dO and dL/dpos are the same
    bits as with one chunk for all positions (each object pixel still takes
    its contributions group by group, in the same order); dL/dP differs only
    in how the probe partial sums are grouped."""
    wl = synth.tiny(W=64, M=2, ny=5, nx=5, step=10.0, seed=46, photons=1e6)
    wl.Hy += 2
    wl.Hx += 2
    d = build(wl)
    O, P, pos = state(wl, d)
    prob, t, ref = gpu_grad(wl, d, O, P, pos)
    assert len(prob.groups()) > 1
    tl = prob.tiling()
    prob.set_tiling(tl["R"], tl["ppc"], tl["CB"], 3 * (wl.M + 1) * wl.W * wl.W * 8, tl["ppcb"])
    L, gO, gP, gpos = [to_host(x) for x in prob.loss_grad(*t)]
    assert abs(L[0] - ref[0][0]) <= 1e-6 * abs(ref[0][0])
    np.testing.assert_array_equal(gO, ref[1])
    np.testing.assert_array_equal(gpos, ref[3])
    assert rel_l2(gP, ref[2]) <= 1e-6
    Lo, gOo, gPo, gposo = grad.loss_and_grad(O, P, pos.astype(np.float64), d["I"], delta=1.0)
    assert rel_l2(gO, gOo) <= 1e-5
    assert rel_l2(gP, gPo) <= 1e-5
