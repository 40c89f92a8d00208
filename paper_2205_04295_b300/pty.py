"""Thin ctypes binding of libpty (include/pty.h): argument marshalling only.

Every step of the reconstruction runs in the library's CUDA kernels; this
module converts torch tensors / NumPy arrays to pointers, picks the memory
kind, and raises ``PtyError`` on a non-zero status.  Importing it fails
loudly when ``libpty.so`` has not been built: there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpty.so")

PTY_OK, PTY_EINVAL, PTY_ENOMEM, PTY_ECUDA, PTY_EDATA, PTY_ETIMEOUT, PTY_ESTATE = range(7)
MEM_HOST, MEM_DEVICE = 0, 1
FLAG_FP32_REGISTRATION = 1
ERR_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EDATA", 5: "ETIMEOUT", 6: "ESTATE"}

c_int, c_float, c_void_p, c_size_t = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
c_int_p = ctypes.POINTER(ctypes.c_int)
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class PtyError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERR_NAMES.get(code, code), msg))
        self.code = code


class ProblemDesc(ctypes.Structure):
    _fields_ = [("W", c_int), ("M", c_int), ("N", c_int), ("Hy", c_int), ("Hx", c_int),
                ("stream", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", c_void_p), ("scratch_bytes", c_size_t), ("flags", c_int)]


class RpieParams(ctypes.Structure):
    _fields_ = [("alpha_O", c_float), ("alpha_P", c_float), ("beta", c_float), ("gamma", c_float),
                ("eps", c_float), ("reg_eps", c_float), ("max_group", c_int),
                ("update_probe", c_int)]


class RefineParams(ctypes.Structure):
    _fields_ = [("upsample", c_int), ("lr", c_float), ("b1", c_float), ("b2", c_float),
                ("eps", c_float), ("start_iter", c_int), ("max_step", c_float),
                ("point", c_int)]


K_NAMES = ["rows_fwd", "cols", "rows_inv", "probe", "reduce", "refine", "grad", "other", "patch"]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 9), ("ms", ctypes.c_double * 9),
                ("patches", ctypes.c_longlong)]

    def as_dict(self):
        return {"launches": {k: int(self.launches[i]) for i, k in enumerate(K_NAMES)},
                "ms": {k: float(self.ms[i]) for i, k in enumerate(K_NAMES)},
                "patches": int(self.patches)}


class Tiling(ctypes.Structure):
    _fields_ = [("R", c_int), ("ppc", c_int), ("CB", c_int), ("scratch_bytes", c_size_t),
                ("ppcb", c_int), ("fused", c_int)]


class BatchSchedule(ctypes.Structure):
    _fields_ = [("split_rows", c_int), ("split_cols", c_int), ("split_probe", c_int),
                ("timeout_ms", c_int), ("ctas", c_int), ("stall_problem", c_int)]


def rpie_params(alpha_O=1.0, alpha_P=1.0, beta=1.0, gamma=0.1, eps=1.0, reg_eps=1e-12,
                max_group=0, update_probe=True):
    return RpieParams(alpha_O, alpha_P, beta, gamma, eps, reg_eps, max_group, int(update_probe))


def refine_params(upsample=20, lr=0.5, b1=0.9, b2=0.999, eps=1e-8, start_iter=0, max_step=0.0,
                  point="A"):
    """point: "A" (XCORR_A, object plane) or "B" (XCORR_B, detector plane)."""
    return RefineParams(upsample, lr, b1, b2, eps, start_iter, max_step,
                        {"A": 0, "B": 1}[point])


_SIGS = {
    "pty_last_error": (ctypes.c_char_p, []),
    "pty_abi_version": (c_int, []),
    "pty_init_problem": (c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(c_void_p)]),
    "pty_destroy": (c_int, [c_void_p]),
    "pty_set_data": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "pty_set_data_async": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "pty_orthogonalize_probe": (c_int, [c_void_p, c_void_p]),
    "pty_debug_stall_copies": (c_int, [c_void_p, c_int]),
    "pty_measure_fp32_peak": (c_int, [c_void_p]),
    "pty_hermitian_eig": (c_int, [c_int, c_void_p, c_void_p, c_void_p]),
    "pty_set_scan_order": (c_int, [c_void_p, c_void_p]),
    "pty_run_iterations": (c_int, [c_void_p, c_int, ctypes.POINTER(RpieParams), c_void_p]),
    "pty_refine_positions": (c_int, [c_void_p, c_int, ctypes.POINTER(RpieParams),
                                     ctypes.POINTER(RefineParams), c_void_p, c_void_p]),
    "pty_run_groups": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(RpieParams), c_void_p]),
    "pty_get_groups": (c_int, [c_void_p, c_int_p, c_void_p, c_void_p]),
    "pty_get_object": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_set_object": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_get_probe": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_set_probe": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_get_positions": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_set_positions": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_get_adam_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int_p, c_int_p, c_int]),
    "pty_set_adam_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int]),
    "pty_model_intensities": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_group_positions": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                    c_int_p]),
    "pty_fft2": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p]),
    "pty_profile": (c_int, [c_void_p, c_int]),
    "pty_set_tiling": (c_int, [c_void_p, ctypes.POINTER(Tiling)]),
    "pty_get_tiling": (c_int, [c_void_p, ctypes.POINTER(Tiling)]),
    "pty_batch_create": (c_int, [ctypes.POINTER(ProblemDesc), c_int, ctypes.POINTER(c_void_p)]),
    "pty_batch_problem": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p)]),
    "pty_batch_set_schedule": (c_int, [c_void_p, ctypes.POINTER(BatchSchedule)]),
    "pty_batch_run": (c_int, [c_void_p, c_int, ctypes.POINTER(RpieParams)]),
    "pty_batch_status": (c_int, [c_void_p, c_void_p]),
    "pty_batch_destroy": (c_int, [c_void_p]),
    "pty_loss": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "pty_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                              c_void_p, c_void_p, c_void_p]),
    "pty_get_refine_gaps": (c_int, [c_void_p, c_void_p, c_int]),
    "pty_model_intensities_noalloc": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int,
                                              c_void_p, c_int, c_void_p, c_void_p]),
    "pty_get_stats": (c_int, [c_void_p, ctypes.POINTER(Stats), c_int]),
}

_lib = None


def lib():
    """Load libpty.so once; raises ImportError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpty.so is not built (run python -m paper_2205_04295_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != PTY_OK:
        raise PtyError(rc, lib().pty_last_error().decode())


def measure_fp32_peak():
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    v = ctypes.c_double(0.0)
    check(lib().pty_measure_fp32_peak(ctypes.byref(v)))
    return v.value


# ------------------------------------------------------------ marshalling
def _ptr(x, dtype):
    """(pointer, mem_kind, keepalive) for a torch tensor or NumPy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != dtype[1]:
                raise TypeError("expected %s, got %s" % (dtype[1], x.dtype))
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype[0])
    return a.ctypes.data, MEM_HOST, a


def _dt(name):
    import torch
    return {"u16": (np.uint16, torch.uint16), "f32": (np.float32, torch.float32),
            "c64": (np.complex64, torch.complex64), "i32": (np.int32, torch.int32)}[name]


def _check_dev(O, P, pos):
    import torch
    for t, dt in ((O, torch.complex64), (P, torch.complex64), (pos, torch.float32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("expected contiguous CUDA tensors: O, P complex64, pos float32")


def group_positions(pos, W, max_group=0, order=None):
    """Greedy disjoint grouping on the host (a C-ABI call that needs no GPU).

    Returns a list of int32 arrays of position indices."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    N = len(pos)
    gptr = np.zeros(N + 1, np.int32)
    gpos = np.zeros(N, np.int32)
    ng = ctypes.c_int(0)
    od = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    check(lib().pty_group_positions(pos.ctypes.data, N, W, max_group,
                                    None if od is None else od.ctypes.data,
                                    gptr.ctypes.data, gpos.ctypes.data, ctypes.byref(ng)))
    return [gpos[gptr[g]:gptr[g + 1]].copy() for g in range(ng.value)]


def hermitian_eig(A):
    """Eigenvalues (decreasing) and eigenvectors (columns, largest entry of
    each real positive) of a Hermitian matrix, by the library's host solver."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    M = A.shape[0]
    w = np.zeros(M, np.float64)
    V = np.zeros((M, M), np.complex128)
    check(lib().pty_hermitian_eig(M, A.ctypes.data, w.ctypes.data, V.ctypes.data))
    return w, V


def fft2_(x, inverse=False):
    """In-place unnormalised 2-D DFT of a contiguous CUDA complex64 tensor (..., W, W)."""
    import torch
    assert x.is_cuda and x.dtype == torch.complex64 and x.is_contiguous()
    W = x.shape[-1]
    batch = x.numel() // (W * W)
    check(lib().pty_fft2(x.data_ptr(), W, batch, int(inverse),
                         torch.cuda.current_stream(x.device).cuda_stream))
    return x


class TorchAllocator:
    """The handle's device memory from PyTorch's caching allocator, through
    the alloc/free hooks of pty_problem_desc: the library's buffers then share
    torch's memory pool (no cudaMalloc, no implicit synchronisation on reuse)
    and are accounted in torch.cuda.memory_allocated().

    ``fail_after`` (test hook, host side): after that many successful
    allocations every further request returns NULL, which the library must
    report as PTY_ENOMEM.  ``live`` maps each outstanding pointer to its size.
    Keep the allocator referenced for as long as any handle it serves lives.
    """

    def __init__(self, device=None, fail_after=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device
        self.fail_after = fail_after
        self.n_alloc = 0
        self.live = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        if self.fail_after is not None and self.n_alloc >= self.fail_after:
            return None
        try:
            import torch
            p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
        except Exception:   # out of memory: the library returns PTY_ENOMEM
            return None
        self.n_alloc += 1
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, stream, ctx):
        if ptr is None:
            return
        self.live.pop(ptr, None)
        try:
            import torch
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:   # interpreter shutdown: torch is already gone
            pass

    def hooks(self):
        return self.alloc_fn, self.free_fn


def _hooks(allocator):
    """(alloc, free, keep-alive) for a desc: "torch" (default), "cuda" (the
    library's own cudaMalloc) or a TorchAllocator-like object."""
    if allocator == "cuda":
        return ALLOC_FN(), FREE_FN(), None
    if allocator == "torch":
        allocator = TorchAllocator()
    a, f = allocator.hooks()
    return a, f, allocator


class Problem:
    """One reconstruction problem (a pty_handle) on the current CUDA device.

    Device memory comes from PyTorch's caching allocator by default
    (``allocator="torch"``); ``"cuda"`` lets the library call cudaMalloc.
    ``fp32_registration`` takes the registration's fine-grid DFT on the FP32
    cores instead of the tensor cores."""

    def __init__(self, W, M, N, Hy, Hx, stream=None, scratch_bytes=0, allocator="torch",
                 fp32_registration=False):
        import torch
        self.W, self.M, self.N, self.Hy, self.Hx = W, M, N, Hy, Hx
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        af, ff, self._allocator = _hooks(allocator)
        d = ProblemDesc(W, M, N, Hy, Hx, c_void_p(stream.cuda_stream), af, ff,
                        None, scratch_bytes, FLAG_FP32_REGISTRATION if fp32_registration else 0)
        h = c_void_p()
        check(lib().pty_init_problem(ctypes.byref(d), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pty_destroy(self.h)  # synchronises: a pending stack is no longer read
            self.h = None
        self._pending_stack = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- data
    def set_data(self, I, pos, O0, P0, overlap=False):
        """Copy in the data.  overlap=True (pty_set_data_async): a host pattern
        stack is uploaded during the next run(), group by group, while earlier
        groups compute; pinned host memory makes the copies asynchronous.
        The stack is kept referenced here until the next set_data or close,
        and must not be modified before the run has finished on the GPU."""
        pI, k1, a1 = _ptr(I, _dt("u16"))
        pp, k2, a2 = _ptr(pos, _dt("f32"))
        pO, k3, a3 = _ptr(O0, _dt("c64"))
        pP, k4, a4 = _ptr(P0, _dt("c64"))
        if len({k1, k2, k3, k4}) != 1:
            raise ValueError("all of I, pos, O0, P0 must live in the same memory (host or device)")
        fn = lib().pty_set_data_async if overlap else lib().pty_set_data
        check(fn(self.h, pI, pp, pO, pP, k1))
        self._pending_stack = a1 if overlap else None

    def set_scan_order(self, order):
        if order is None:
            check(lib().pty_set_scan_order(self.h, None))
        else:
            o = np.ascontiguousarray(order, dtype=np.int32)
            check(lib().pty_set_scan_order(self.h, o.ctypes.data))

    # -- iterations
    def run(self, n_iter, params=None, errors=True):
        params = params or rpie_params()
        err = np.zeros(max(n_iter, 1), np.float32)
        check(lib().pty_run_iterations(self.h, n_iter, ctypes.byref(params),
                                       err.ctypes.data if errors else None))
        return err[:n_iter] if errors else None

    def refine(self, n_iter, params=None, rparams=None, errors=True, shifts=False):
        params = params or rpie_params()
        rparams = rparams or refine_params()
        err = np.zeros(max(n_iter, 1), np.float32)
        sh = np.zeros((self.N, 2), np.float32)
        check(lib().pty_refine_positions(self.h, n_iter, ctypes.byref(params), ctypes.byref(rparams),
                                         err.ctypes.data if errors else None,
                                         sh.ctypes.data if shifts else None))
        out = err[:n_iter] if errors else None
        return (out, sh) if shifts else out

    def run_groups(self, g0, g1, params=None):
        params = params or rpie_params()
        e = np.zeros(1, np.float32)
        check(lib().pty_run_groups(self.h, g0, g1, ctypes.byref(params), e.ctypes.data))
        return float(e[0])

    def groups(self):
        ng = ctypes.c_int(0)
        check(lib().pty_get_groups(self.h, ctypes.byref(ng), None, None))
        gptr = np.zeros(ng.value + 1, np.int32)
        gpos = np.zeros(self.N, np.int32)
        check(lib().pty_get_groups(self.h, ctypes.byref(ng), gptr.ctypes.data, gpos.ctypes.data))
        return [gpos[gptr[g]:gptr[g + 1]].copy() for g in range(ng.value)]

    # -- copies (device tensors out)
    def _get(self, fn, shape, dt, device=True):
        import torch
        if device:
            t = torch.empty(shape, dtype=dt[1], device="cuda")
            check(fn(self.h, t.data_ptr(), MEM_DEVICE))
            return t
        a = np.empty(shape, dtype=dt[0])
        check(fn(self.h, a.ctypes.data, MEM_HOST))
        return a

    def object(self, device=True):
        return self._get(lib().pty_get_object, (self.Hy, self.Hx), _dt("c64"), device)

    def probe(self, device=True):
        return self._get(lib().pty_get_probe, (self.M, self.W, self.W), _dt("c64"), device)

    def positions(self, device=True):
        return self._get(lib().pty_get_positions, (self.N, 2), _dt("f32"), device)

    def refine_gaps(self, device=False):
        return self._get(lib().pty_get_refine_gaps, (self.N,), _dt("f32"), device)

    def model_intensities(self, device=True):
        return self._get(lib().pty_model_intensities, (self.N, self.W, self.W), _dt("f32"), device)

    def set_object(self, O):
        p, k, a = _ptr(O, _dt("c64"))
        check(lib().pty_set_object(self.h, p, k))

    def set_probe(self, P):
        p, k, a = _ptr(P, _dt("c64"))
        check(lib().pty_set_probe(self.h, p, k))

    def set_positions(self, pos):
        p, k, a = _ptr(pos, _dt("f32"))
        check(lib().pty_set_positions(self.h, p, k))

    def adam_state(self):
        m = np.zeros((self.N, 2), np.float32)
        v = np.zeros((self.N, 2), np.float32)
        t, it = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().pty_get_adam_state(self.h, m.ctypes.data, v.ctypes.data, ctypes.byref(t),
                                       ctypes.byref(it), MEM_HOST))
        return m, v, t.value, it.value

    def loss(self, O, P, pos, delta=1.0):
        """Amplitude loss of the bilinear-crop forward model (device tensors)."""
        import torch
        _check_dev(O, P, pos)
        out = torch.empty(1, dtype=torch.float32, device=O.device)
        check(lib().pty_loss(self.h, O.data_ptr(), P.data_ptr(), pos.data_ptr(), float(delta),
                             out.data_ptr()))
        return out

    def loss_grad(self, O, P, pos, delta=1.0):
        """(loss, dL/dO, dL/dP, dL/dpos); complex gradients as dL/dRe + i dL/dIm."""
        import torch
        _check_dev(O, P, pos)
        out = torch.empty(1, dtype=torch.float32, device=O.device)
        gO, gP, gpos = torch.empty_like(O), torch.empty_like(P), torch.empty_like(pos)
        check(lib().pty_loss_grad(self.h, O.data_ptr(), P.data_ptr(), pos.data_ptr(), float(delta),
                                  out.data_ptr(), gO.data_ptr(), gP.data_ptr(), gpos.data_ptr()))
        return out, gO, gP, gpos

    def debug_stall_copies(self, on):
        """Test hook: make every staged copy's bounded wait run out (on=True)
        or restore normal operation (on=False)."""
        check(lib().pty_debug_stall_copies(self.h, int(bool(on))))

    def orthogonalize_probe(self):
        """Orthogonalise the probe modes in place; returns their powers
        (decreasing)."""
        w = np.zeros(self.M, np.float64)
        check(lib().pty_orthogonalize_probe(self.h, w.ctypes.data))
        return w

    def set_tiling(self, R=0, ppc=0, CB=0, scratch_bytes=0, ppcb=0, fused=0):
        """fused = S > 0: the single-kernel patch path (W <= 128), a cluster
        of S CTAs per patch; 0: the three passes."""
        check(lib().pty_set_tiling(self.h, ctypes.byref(Tiling(R, ppc, CB, scratch_bytes, ppcb,
                                                               fused))))

    def tiling(self):
        t = Tiling()
        check(lib().pty_get_tiling(self.h, ctypes.byref(t)))
        return {"R": t.R, "ppc": t.ppc, "CB": t.CB, "scratch_bytes": int(t.scratch_bytes),
                "ppcb": t.ppcb, "fused": t.fused}

    def profile(self, mode):
        check(lib().pty_profile(self.h, int(mode)))

    def stats(self, reset=False):
        st = Stats()
        check(lib().pty_get_stats(self.h, ctypes.byref(st), int(reset)))
        return st.as_dict()

    def set_adam_state(self, m, v, t, it):
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        check(lib().pty_set_adam_state(self.h, m.ctypes.data, v.ctypes.data, t, it, MEM_HOST))


class _Borrowed(Problem):
    """A Problem view of a handle owned by a Batch (never destroyed here)."""

    def __init__(self, h, W, M, N, Hy, Hx, stream):
        self.W, self.M, self.N, self.Hy, self.Hx = W, M, N, Hy, Hx
        self.stream = stream
        self.h = h

    def close(self):
        self.h = None


class Batch:
    """Many independent problems run by one persistent graph-captured launch."""

    def __init__(self, shapes, stream=None, scratch_bytes=0, allocator="torch"):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        n = len(shapes)
        af, ff, self._allocator = _hooks(allocator)
        arr = (ProblemDesc * n)()
        for i, (W, M, N, Hy, Hx) in enumerate(shapes):
            arr[i] = ProblemDesc(W, M, N, Hy, Hx, c_void_p(stream.cuda_stream), af, ff, None,
                                 scratch_bytes, 0)
        b = c_void_p()
        check(lib().pty_batch_create(arr, n, ctypes.byref(b)))
        self.b = b
        self.problems = []
        for i, shp in enumerate(shapes):
            h = c_void_p()
            check(lib().pty_batch_problem(b, i, ctypes.byref(h)))
            self.problems.append(_Borrowed(h, *shp, stream))

    def schedule(self, split_rows=4, split_cols=2, split_probe=4, timeout_ms=2000, ctas=0,
                 stall_problem=-1):
        sc = BatchSchedule(split_rows, split_cols, split_probe, timeout_ms, ctas, stall_problem)
        check(lib().pty_batch_set_schedule(self.b, ctypes.byref(sc)))

    def run(self, n_iter, params=None):
        params = params or rpie_params()
        check(lib().pty_batch_run(self.b, n_iter, ctypes.byref(params)))

    def status(self):
        st = np.zeros(len(self.problems), np.int32)
        check(lib().pty_batch_status(self.b, st.ctypes.data))
        return st

    def close(self):
        if getattr(self, "b", None):
            for p in self.problems:
                p.close()
            lib().pty_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
