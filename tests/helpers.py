"""Shared helpers of the parity tests: seeded inputs (from the generator
module), the oracle on the CPU, the library through its binding."""
import numpy as np

from paper_2205_04295_b300 import synth


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def build(wl, device="cpu"):
    d = synth.build(wl, device=device)
    I = d["I"]
    d["I"] = synth.counts_u16(I)
    return d


def to_host(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype == torch.uint16:
                x = x.to(torch.int32)
            return x.cpu().numpy()
    except ImportError:
        pass
    return np.asarray(x)
