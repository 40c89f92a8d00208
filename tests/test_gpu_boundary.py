"""The handle's memory hooks and its state round trip, through the C ABI.

* PyTorch's caching allocator serves every device buffer of a handle through
  the alloc/free hooks of pty_problem_desc, and gets all of it back on
  pty_destroy; results are bitwise those of the library's own cudaMalloc.
* A host-side allocator that returns NULL at the k-th request, for every k,
  makes pty_init_problem fail with PTY_ENOMEM and release what it had taken
  (the failure is injected on the host; nothing faults on the GPU).
* Checkpoint / resume: 50 iterations, the state read out through the get
  calls and loaded into a fresh handle through the set calls, then 50 more,
  equals 100 iterations on one handle bitwise (with refinement, so the Adam
  moments and step count are part of the state)."""
import numpy as np
import pytest

from helpers import build
from paper_2205_04295_b300 import synth

pytestmark = pytest.mark.gpu


def small():
    wl = synth.tiny(W=64, M=2, ny=4, nx=4, step=10.0, seed=61, photons=1e6, jitter=1.0, err=1.5)
    return wl, build(wl)


def test_torch_allocator_serves_and_gets_back_every_buffer():
    import torch
    from paper_2205_04295_b300 import pty
    wl, d = small()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    al = pty.TorchAllocator()
    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, allocator=al)
    assert len(al.live) > 10
    held = sum(al.live.values())
    assert torch.cuda.memory_allocated() - base >= held
    prob.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    e1 = prob.run(3)
    O1, P1 = prob.object(False), prob.probe(False)
    prob.close()
    assert al.live == {}
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    ref = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, allocator="cuda")
    ref.set_data(d["I"], d["pos"], d["O0"], d["P0"])
    np.testing.assert_array_equal(ref.run(3), e1)
    np.testing.assert_array_equal(ref.object(False), O1)
    np.testing.assert_array_equal(ref.probe(False), P1)


def test_allocator_returning_null_gives_enomem_at_every_request():
    import torch
    from paper_2205_04295_b300 import pty
    wl, _ = small()
    probe = pty.TorchAllocator()
    pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, allocator=probe).close()
    total = probe.n_alloc
    assert total > 10
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for k in range(total):
        al = pty.TorchAllocator(fail_after=k)
        with pytest.raises(pty.PtyError) as ei:
            pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, allocator=al)
        assert ei.value.code == pty.PTY_ENOMEM, (k, str(ei.value))
        assert al.n_alloc == k and al.live == {}
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_checkpoint_resume_is_bitwise():
    from paper_2205_04295_b300 import pty
    wl, d = small()
    pg, rg = pty.rpie_params(), pty.refine_params(upsample=20, lr=0.5, start_iter=5)

    def fresh():
        p = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
        p.set_data(d["I"], d["pos"], d["O0"], d["P0"])
        return p

    straight = fresh()
    e_all = straight.refine(100, pg, rg)
    first = fresh()
    e_a = first.refine(50, pg, rg)
    O, P, pos = first.object(False), first.probe(False), first.positions(False)
    m, v, t, it = first.adam_state()
    first.close()
    second = fresh()
    second.set_object(O)
    second.set_probe(P)
    second.set_positions(pos)
    second.set_adam_state(m, v, t, it)
    e_b = second.refine(50, pg, rg)
    np.testing.assert_array_equal(np.concatenate([e_a, e_b]), e_all)
    np.testing.assert_array_equal(second.object(False), straight.object(False))
    np.testing.assert_array_equal(second.probe(False), straight.probe(False))
    np.testing.assert_array_equal(second.positions(False), straight.positions(False))
    m2, v2, t2, it2 = second.adam_state()
    ms, vs, ts, its = straight.adam_state()
    np.testing.assert_array_equal(m2, ms)
    np.testing.assert_array_equal(v2, vs)
    assert (t2, it2) == (ts, its) == (95, 100)
