"""ctypes binding of liblra.so (include/lra.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch
supplies device memory and the stream.  Importing this module does not load the
library; the first call does, and fails with an error when it was not built
(no CPU fallback).

Names follow the C ABI: lra_create / lra_sketch / lra_farpca_run / lra_result /
lra_copy_omega / lra_farpca_host / lra_last_error, wrapped by ``Farpca``.
"""
import ctypes
import os
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_int32, c_int64, c_uint32, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblra.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
GAUSSIAN, STD_BERNOULLI, SPARSE_SIGN, SPARSE_SIGN_IID, SPARSE_GAUSSIAN, BERNOULLI = range(6)
F64, F32 = 0, 1
FLAG_KEEP_Y = 1
FLAG_PROFILE = 2
FLAG_FP64_SIMT = 4
FLAG_NO_A_DIGITS = 8
FLAG_NO_GRAPHS = 16
FLAG_MIXED = 32
FLAG_POOL = 64
PHASES = ("omega", "sketch", "dense", "deflate", "project", "orth", "indicator", "cut")
MAX_B, MAX_P, MAX_ZETA = 64, 8, 256

EXPORTS = ("lra_create", "lra_destroy", "lra_capacity", "lra_sketch", "lra_farpca_run", "lra_result",
           "lra_farpca_host", "lra_farpca_host_prefetch", "lra_copy_omega", "lra_last_error", "lra_status_string",
           "lra_kernel_launches", "lra_version", "lra_phase_times", "lra_apply", "lra_svd", "lra_farpca_host_f32",
           "lra_workspace_bytes", "lra_device_bytes", "lra_server_create", "lra_server_submit",
           "lra_server_poll", "lra_server_pending", "lra_server_release", "lra_server_clock",
           "lra_server_destroy", "lra_batch_create", "lra_batch_run", "lra_batch_result",
           "lra_batch_steps", "lra_batch_device_bytes", "lra_batch_destroy", "lra_batch_set_tiling",
           "lra_batch_get_tiling", "lra_batch_tune", "lra_selftest_waits")


class Matrix(Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("lda", c_int64), ("dtype", c_int32),
                ("reserved", c_int32), ("data", c_void_p)]


class Params(Structure):
    _fields_ = [("eps", c_double), ("k", c_int64), ("b", c_int32), ("P", c_int32), ("kind", c_int32),
                ("zeta", c_int32), ("p", c_double), ("seed", c_uint64), ("max_blocks", c_int32),
                ("flags", c_uint32)]


class Result(Structure):
    _fields_ = [("status", c_int32), ("reserved", c_int32), ("rank", c_int64), ("blocks", c_int64),
                ("E", c_double), ("normA2", c_double), ("rel_err", c_double), ("Q", c_void_p),
                ("ldq", c_int64), ("B", c_void_p), ("ldb", c_int64), ("Y", c_void_p), ("ldy", c_int64)]


class SvdResult(Structure):
    _fields_ = [("status", c_int32), ("sweeps", c_int32), ("l", c_int64), ("r", c_int64),
                ("E_r", c_double), ("normA2", c_double), ("U", c_void_p), ("ldu", c_int64),
                ("sigma", c_void_p), ("V", c_void_p), ("ldv", c_int64)]


class ServerParams(Structure):
    _fields_ = [("hbm_budget", c_int64), ("slots", c_int32), ("flags", c_uint32)]


class Request(Structure):
    _fields_ = [("id", c_uint64), ("A", Matrix), ("params", Params), ("keep", c_int32),
                ("reserved", c_int32)]


class Completion(Structure):
    _fields_ = [("id", c_uint64), ("status", c_int32), ("reserved", c_int32), ("rank", c_int64),
                ("rel_err", c_double), ("t_submit", c_double), ("t_admit", c_double), ("t_start", c_double),
                ("t_done", c_double), ("bytes", c_int64), ("ctx", c_void_p)]


class BatchItem(Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("lda", c_int64), ("A", c_void_p), ("eps", c_double),
                ("seed", c_uint64)]


class BatchParams(Structure):
    _fields_ = [("b", c_int32), ("P", c_int32), ("zeta", c_int32), ("max_blocks", c_int32),
                ("flags", c_uint32)]


class BatchTiling(Structure):
    _fields_ = [("tn", c_int32 * 3), ("nn", c_int32 * 3)]


class BatchResult(Structure):
    _fields_ = [("status", c_int32), ("reserved", c_int32), ("rank", c_int64), ("E", c_double),
                ("normA2", c_double), ("rel_err", c_double), ("Q", c_void_p), ("ldq", c_int64),
                ("Bt", c_void_p), ("ldbt", c_int64)]


class LraError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_string(status), msg))
        self.status = status


_lib = None


def load(path=LIB_PATH):
    """Load liblra.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError("liblra.so not built at %s: run __graft_entry__.build() or "
                                "python -m paper_2506_03859_gb300.build" % path)
    lib = ctypes.CDLL(path)
    vp = c_void_p
    lib.lra_create.argtypes = [POINTER(vp), c_int64, c_int64, POINTER(Params), vp]
    lib.lra_create.restype = c_int32
    lib.lra_destroy.argtypes = [vp]
    lib.lra_destroy.restype = None
    lib.lra_capacity.argtypes = [vp]
    lib.lra_capacity.restype = c_int64
    lib.lra_sketch.argtypes = [vp, POINTER(Matrix), c_int64, c_int64, vp, c_int64]
    lib.lra_sketch.restype = c_int32
    lib.lra_farpca_run.argtypes = [vp, POINTER(Matrix)]
    lib.lra_farpca_run.restype = c_int32
    lib.lra_result.argtypes = [vp, POINTER(Result)]
    lib.lra_result.restype = c_int32
    lib.lra_farpca_host.argtypes = [vp, vp, c_int64, vp, c_int64, vp, c_int64, POINTER(Result)]
    lib.lra_farpca_host.restype = c_int32
    lib.lra_farpca_host_prefetch.argtypes = [vp, vp, c_int64, vp, vp, c_int64, vp, c_int64, POINTER(Result)]
    lib.lra_farpca_host_prefetch.restype = c_int32
    lib.lra_copy_omega.argtypes = [vp, c_int64, c_int64, vp, vp, vp]
    lib.lra_copy_omega.restype = c_int32
    lib.lra_last_error.argtypes = [vp]
    lib.lra_last_error.restype = c_char_p
    lib.lra_status_string.argtypes = [c_int32]
    lib.lra_status_string.restype = c_char_p
    lib.lra_kernel_launches.argtypes = []
    lib.lra_kernel_launches.restype = c_uint64
    lib.lra_version.argtypes = []
    lib.lra_version.restype = c_int32
    lib.lra_phase_times.argtypes = [vp, vp, vp, c_int32, c_int32]
    lib.lra_phase_times.restype = c_int32
    lib.lra_apply.argtypes = [vp, POINTER(Matrix), c_int32, vp, c_int64, c_int64, vp, c_int64]
    lib.lra_apply.restype = c_int32
    lib.lra_farpca_host_f32.argtypes = [vp, vp, c_int64, vp, c_int64, vp, c_int64, POINTER(Result)]
    lib.lra_farpca_host_f32.restype = c_int32
    lib.lra_workspace_bytes.argtypes = [c_int64, c_int64, POINTER(Params)]
    lib.lra_workspace_bytes.restype = c_int64
    lib.lra_device_bytes.argtypes = [vp]
    lib.lra_device_bytes.restype = c_int64
    lib.lra_selftest_waits.argtypes = [POINTER(c_int32)]
    lib.lra_selftest_waits.restype = c_int32
    lib.lra_server_create.argtypes = [POINTER(vp), POINTER(ServerParams)]
    lib.lra_server_create.restype = c_int32
    lib.lra_server_submit.argtypes = [vp, POINTER(Request)]
    lib.lra_server_submit.restype = c_int32
    lib.lra_server_poll.argtypes = [vp, POINTER(Completion), c_int64, c_int32]
    lib.lra_server_poll.restype = c_int64
    lib.lra_server_pending.argtypes = [vp]
    lib.lra_server_pending.restype = c_int64
    lib.lra_server_release.argtypes = [vp, vp]
    lib.lra_server_release.restype = c_int32
    lib.lra_server_clock.argtypes = [vp]
    lib.lra_server_clock.restype = c_double
    lib.lra_server_destroy.argtypes = [vp]
    lib.lra_server_destroy.restype = None
    lib.lra_batch_create.argtypes = [POINTER(vp), POINTER(BatchItem), c_int64, POINTER(BatchParams), vp]
    lib.lra_batch_create.restype = c_int32
    lib.lra_batch_run.argtypes = [vp]
    lib.lra_batch_run.restype = c_int32
    lib.lra_batch_result.argtypes = [vp, c_int64, POINTER(BatchResult)]
    lib.lra_batch_result.restype = c_int32
    lib.lra_batch_steps.argtypes = [vp]
    lib.lra_batch_steps.restype = c_int64
    lib.lra_batch_device_bytes.argtypes = [vp]
    lib.lra_batch_device_bytes.restype = c_int64
    lib.lra_batch_destroy.argtypes = [vp]
    lib.lra_batch_destroy.restype = None
    lib.lra_batch_set_tiling.argtypes = [vp, POINTER(BatchTiling)]
    lib.lra_batch_set_tiling.restype = c_int32
    lib.lra_batch_get_tiling.argtypes = [vp, POINTER(BatchTiling)]
    lib.lra_batch_get_tiling.restype = c_int32
    lib.lra_batch_tune.argtypes = [vp, c_int32, POINTER(BatchTiling), POINTER(c_double), POINTER(c_double)]
    lib.lra_batch_tune.restype = c_int32
    lib.lra_svd.argtypes = [vp, POINTER(SvdResult)]
    lib.lra_svd.restype = c_int32
    _lib = lib
    return lib


def status_string(s):
    return load().lra_status_string(int(s)).decode()


def kernel_launches():
    return int(load().lra_kernel_launches())


class _DeviceView:
    """A __cuda_array_interface__ over library-owned device memory (no copy)."""

    def __init__(self, ptr, shape, strides_elems, owner, itemsize=8):
        self._owner = owner
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": "<f%d" % itemsize, "data": (int(ptr), False),
            "strides": tuple(itemsize * s for s in strides_elems), "version": 3, "stream": None}


def _device_matrix(A, torch):
    if not (A.is_cuda and A.dtype in (torch.float64, torch.float32) and A.dim() == 2):
        raise TypeError("A must be a 2-D float64 or float32 CUDA tensor")
    m, n = A.shape
    if A.stride(0) != 1 or (n > 1 and A.stride(1) < m):
        raise ValueError("A must be column-major (stride(0) == 1, stride(1) >= m)")
    return Matrix(m, n, max(A.stride(1), m), F64 if A.dtype == torch.float64 else F32, 0,
                  A.data_ptr())


def column_major(t):
    """Copy a 2-D tensor into a fresh column-major tensor on the same device."""
    import torch
    out = torch.empty_strided(tuple(t.shape), (1, t.shape[0]), dtype=t.dtype, device=t.device)
    out.copy_(t)
    return out


class Farpca:
    """One library context (lra_create) for m x n inputs and fixed parameters."""

    def __init__(self, m, n, eps=0.0, k=0, b=20, P=1, kind=SPARSE_SIGN, zeta=8, p=0.0, seed=0,
                 max_blocks=0, keep_y=False, profile=False, fp64_simt=False, a_digits=True,
                 graphs=True, mixed=False, pool=False, stream=None):
        import torch
        self._torch = torch
        self._lib = load()
        self.m, self.n, self.b = m, n, b
        flags = ((FLAG_KEEP_Y if keep_y else 0) | (FLAG_PROFILE if profile else 0)
                 | (FLAG_FP64_SIMT if fp64_simt else 0) | (0 if a_digits else FLAG_NO_A_DIGITS)
                 | (0 if graphs else FLAG_NO_GRAPHS) | (FLAG_MIXED if mixed else 0)
                 | (FLAG_POOL if pool else 0))
        self.params = Params(eps, k, b, P, kind, zeta, p, seed & 0xFFFFFFFFFFFFFFFF, max_blocks, flags)
        self._ctx = c_void_p()
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        sptr = c_void_p(stream.cuda_stream if stream is not None else 0)
        s = self._lib.lra_create(byref(self._ctx), m, n, byref(self.params), sptr)
        if s != OK:
            raise LraError(s, "lra_create failed (invalid parameters or no device memory)")

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.lra_destroy(self._ctx)
            self._ctx = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s < 0:
            raise LraError(s, self._lib.lra_last_error(self._ctx).decode())
        return s

    def device_bytes(self):
        """lra_device_bytes: device memory this context has allocated."""
        return int(self._lib.lra_device_bytes(self._ctx))

    @property
    def capacity(self):
        return int(self._lib.lra_capacity(self._ctx))

    def run(self, A):
        """lra_farpca_run on a column-major float64 CUDA tensor; returns the status."""
        mat = _device_matrix(A, self._torch)
        return self._check(self._lib.lra_farpca_run(self._ctx, byref(mat)))

    def result(self):
        """lra_result: a dict with status, rank, blocks, E, normA2, rel_err and
        zero-copy torch views Q (m x rank), B (rank x n) and, if kept, Y."""
        r = Result()
        self._check(self._lib.lra_result(self._ctx, byref(r)))
        torch = self._torch
        out = dict(status=r.status, rank=r.rank, blocks=r.blocks, E=r.E, normA2=r.normA2,
                   rel_err=r.rel_err)
        l = r.rank
        if l > 0:
            out["Q"] = torch.as_tensor(_DeviceView(r.Q, (self.m, l), (1, r.ldq), self), device="cuda")
            out["B"] = torch.as_tensor(_DeviceView(r.B, (l, self.n), (1, r.ldb), self), device="cuda")
            if r.Y:
                out["Y"] = torch.as_tensor(_DeviceView(r.Y, (self.m, l), (1, r.ldy), self), device="cuda")
        return out

    def svd(self):
        """lra_svd: the SVD of the last run's Q B and its truncation.  A dict with
        status, sweeps, l, r, E_r, normA2 and zero-copy torch views U (m x l),
        sigma (l, descending) and V (n x l); views stay valid until the next
        svd / run on this context."""
        r = SvdResult()
        self._check(self._lib.lra_svd(self._ctx, byref(r)))
        torch = self._torch
        out = dict(status=r.status, sweeps=r.sweeps, l=r.l, r=r.r, E_r=r.E_r, normA2=r.normA2)
        l = r.l
        if l > 0:
            out["U"] = torch.as_tensor(_DeviceView(r.U, (self.m, l), (1, r.ldu), self), device="cuda")
            out["sigma"] = torch.as_tensor(_DeviceView(r.sigma, (l,), (1,), self), device="cuda")
            out["V"] = torch.as_tensor(_DeviceView(r.V, (self.n, l), (1, r.ldv), self), device="cuda")
        return out

    def apply(self, A, Y, trans=False, C=None):
        """lra_apply: C = op(A) Y (op(A) = A^T if trans) with the context's dense engine."""
        torch = self._torch
        mat = _device_matrix(A, torch)
        rows_c = self.n if trans else self.m
        N = Y.shape[1]
        if Y.stride(0) != 1:
            raise ValueError("Y must be column-major")
        if C is None:
            C = torch.empty_strided((rows_c, N), (1, rows_c), dtype=torch.float64, device=A.device)
        self._check(self._lib.lra_apply(self._ctx, byref(mat), 1 if trans else 0, c_void_p(Y.data_ptr()),
                                        max(Y.stride(1), Y.shape[0]), N, c_void_p(C.data_ptr()),
                                        max(C.stride(1), rows_c)))
        return C

    def phase_times(self, reset=True):
        """lra_phase_times: {phase: (ms, calls)} accumulated since the last reset."""
        import numpy as np
        ms = np.zeros(len(PHASES))
        calls = np.zeros(len(PHASES), dtype=np.int64)
        self._check(self._lib.lra_phase_times(self._ctx, ms.ctypes.data, calls.ctypes.data, len(PHASES),
                                              1 if reset else 0))
        return {name: (float(ms[i]), int(calls[i])) for i, name in enumerate(PHASES)}

    def sketch(self, A, j0, nblk, Y=None):
        """lra_sketch: Y = A [Omega_j0 .. Omega_{j0+nblk-1}] into a column-major m x nblk*b tensor."""
        torch = self._torch
        mat = _device_matrix(A, torch)
        if Y is None:
            Y = torch.empty_strided((self.m, nblk * self.b), (1, self.m), dtype=torch.float64,
                                    device=A.device)
        if Y.stride(0) != 1 or Y.shape[0] != self.m or Y.shape[1] < nblk * self.b:
            raise ValueError("Y must be column-major m x (nblk*b)")
        ldy = max(Y.stride(1), self.m)
        self._check(self._lib.lra_sketch(self._ctx, byref(mat), j0, nblk, c_void_p(Y.data_ptr()), ldy))
        return Y

    def copy_omega(self, j, cap=None):
        """lra_copy_omega: (counts[b], rows[b, cap], vals[b, cap]) as numpy arrays."""
        import numpy as np
        kind = self.params.kind
        if cap is None:
            cap = self.params.zeta if kind == SPARSE_SIGN else self.n
        counts = np.zeros(self.b, dtype=np.int32)
        rows = np.zeros((self.b, cap), dtype=np.int32)
        vals = np.zeros((self.b, cap), dtype=np.float64)
        self._check(self._lib.lra_copy_omega(self._ctx, j, cap, counts.ctypes.data, rows.ctypes.data,
                                             vals.ctypes.data))
        return counts, rows, vals

    def run_host(self, A_host, Q_host=None, B_host=None, next_A=None):
        """lra_farpca_host (float64 A) or lra_farpca_host_f32 (float32 A): A, Q, B in
        host memory (numpy, column-major; ideally pinned).  With next_A (float64, the
        same shape and layout; kept unchanged by the caller until it is solved),
        lra_farpca_host_prefetch: its copy to the device overlaps this solve.
        Returns the result dict (without device views)."""
        import numpy as np
        if A_host.dtype not in (np.float64, np.float32) or not A_host.flags.f_contiguous:
            raise ValueError("A_host must be a Fortran-ordered float64 or float32 array")
        r = Result()
        qp = c_void_p(Q_host.ctypes.data) if Q_host is not None else c_void_p(0)
        bp = c_void_p(B_host.ctypes.data) if B_host is not None else c_void_p(0)
        ldq = Q_host.shape[0] if Q_host is not None else 0
        ldb = B_host.shape[0] if B_host is not None else 0
        if next_A is not None:
            if (A_host.dtype != np.float64 or next_A.dtype != np.float64 or next_A.shape != A_host.shape
                    or not next_A.flags.f_contiguous):
                raise ValueError("prefetch takes float64 Fortran-ordered matrices of one shape")
            s = self._lib.lra_farpca_host_prefetch(self._ctx, c_void_p(A_host.ctypes.data), A_host.shape[0],
                                                   c_void_p(next_A.ctypes.data), qp, ldq, bp, ldb, byref(r))
            self._check(s)
            return dict(status=r.status, rank=r.rank, blocks=r.blocks, E=r.E, normA2=r.normA2,
                        rel_err=r.rel_err)
        fn = self._lib.lra_farpca_host if A_host.dtype == np.float64 else self._lib.lra_farpca_host_f32
        s = fn(self._ctx, c_void_p(A_host.ctypes.data), A_host.shape[0], qp, ldq, bp, ldb, byref(r))
        self._check(s)
        return dict(status=r.status, rank=r.rank, blocks=r.blocks, E=r.E, normA2=r.normA2,
                    rel_err=r.rel_err)


def params(eps=0.0, k=0, b=20, P=1, kind=SPARSE_SIGN, zeta=8, p=0.0, seed=0, max_blocks=0, flags=0):
    """An lra_params structure (the problem statement's arguments)."""
    return Params(eps, k, b, P, kind, zeta, p, seed & 0xFFFFFFFFFFFFFFFF, max_blocks, flags)


def workspace_bytes(m, n, prm):
    """lra_workspace_bytes: device bytes a context for these arguments allocates."""
    v = int(load().lra_workspace_bytes(m, n, byref(prm)))
    if v < 0:
        raise LraError(v, "invalid arguments")
    return v


def selftest_waits():
    """lra_selftest_waits: (status, which) after running both kinds of bounded
    device wait against conditions that never come true (expected:
    ERR_TIMEOUT and which == 3)."""
    which = c_int32(0)
    st = int(load().lra_selftest_waits(byref(which)))
    return st, int(which.value)


class KeptRun:
    """A completed request whose context the server kept (lra_request.keep):
    result() and svd() as for Farpca; release() returns its memory to the server."""

    def __init__(self, server, ctx, m, n):
        import torch
        self._server, self._ctx, self.m, self.n = server, c_void_p(ctx), m, n
        self._lib, self._torch = server._lib, torch

    def _check(self, s):
        if s < 0:
            raise LraError(s, self._lib.lra_last_error(self._ctx).decode())
        return s

    result = lambda self: Farpca.result(self)   # noqa: E731
    svd = lambda self: Farpca.svd(self)         # noqa: E731

    def release(self):
        if self._ctx:
            self._server._check(self._server._lib.lra_server_release(self._server._srv, self._ctx))
            self._ctx = None


class Server:
    """lra_server: admission by device-memory budget, `slots` requests at once."""

    def __init__(self, hbm_budget=0, slots=8, flags=0):
        self._lib = load()
        self._srv = c_void_p()
        self._check(self._lib.lra_server_create(byref(self._srv), byref(ServerParams(hbm_budget, slots, flags))))
        self._shapes = {}
        self._keep = {}

    def _check(self, s):
        if s < 0:
            raise LraError(s, "server call failed")
        return s

    def submit(self, A, prm, rid, keep=False):
        """Queue a request on a column-major float64/float32 CUDA tensor A (kept
        alive by the caller until its completion is polled)."""
        import torch
        req = Request(rid, _device_matrix(A, torch), prm, 1 if keep else 0, 0)
        self._check(self._lib.lra_server_submit(self._srv, byref(req)))
        self._shapes[rid] = tuple(A.shape)

    def poll(self, max_items=256, wait=False):
        """Completions since the last poll: dicts with id, status, rank, rel_err,
        t_submit, t_start, t_done, bytes and, for kept requests, `run` (KeptRun)."""
        buf = (Completion * max_items)()
        k = int(self._lib.lra_server_poll(self._srv, buf, max_items, 1 if wait else 0))
        self._check(k)
        out = []
        for c in buf[:k]:
            d = dict(id=c.id, status=c.status, rank=c.rank, rel_err=c.rel_err, t_submit=c.t_submit,
                     t_admit=c.t_admit, t_start=c.t_start, t_done=c.t_done, bytes=c.bytes)
            m, n = self._shapes.pop(c.id, (0, 0))
            if c.ctx:
                d["run"] = KeptRun(self, c.ctx, m, n)
            out.append(d)
        return out

    def pending(self):
        return int(self._lib.lra_server_pending(self._srv))

    def clock(self):
        return float(self._lib.lra_server_clock(self._srv))

    def close(self):
        if self._srv:
            self._lib.lra_server_destroy(self._srv)
            self._srv = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """lra_batch: many independent FP32 problems (fixed-zeta sparse sign Omega),
    run together by one graph launch.  `mats`: column-major float32 CUDA tensors
    (kept alive by the caller); `eps`, `seeds`: one per matrix."""

    def __init__(self, mats, eps, seeds, b=16, P=1, zeta=4, max_blocks=0, stream=None, graph=True):
        import torch
        self._lib, self._torch = load(), torch
        items = (BatchItem * len(mats))()
        self.shapes = []
        for k, A in enumerate(mats):
            if not (A.is_cuda and A.dtype == torch.float32 and A.dim() == 2 and A.stride(0) == 1):
                raise TypeError("batch matrices must be column-major float32 CUDA tensors")
            m, n = A.shape
            items[k] = BatchItem(m, n, max(A.stride(1), m), A.data_ptr(), float(eps[k]),
                                 int(seeds[k]) & 0xFFFFFFFFFFFFFFFF)
            self.shapes.append((m, n))
        self._b = c_void_p()
        st = c_void_p(stream.cuda_stream) if stream is not None else c_void_p(0)
        s = self._lib.lra_batch_create(byref(self._b), items, len(mats), byref(BatchParams(b, P, zeta, max_blocks, 0 if graph else FLAG_NO_GRAPHS)),
                                       st)
        if s < 0:
            raise LraError(s, "lra_batch_create")

    def run(self):
        s = self._lib.lra_batch_run(self._b)
        if s < 0:
            raise LraError(s, "lra_batch_run")

    def steps(self):
        return int(self._lib.lra_batch_steps(self._b))

    def tiling(self):
        """lra_batch_get_tiling: {"tn": [3 ints], "nn": [3 ints]}."""
        t = BatchTiling()
        s = self._lib.lra_batch_get_tiling(self._b, byref(t))
        if s < 0:
            raise LraError(s, "lra_batch_get_tiling")
        return {"tn": list(t.tn), "nn": list(t.nn)}

    def set_tiling(self, tn, nn):
        """lra_batch_set_tiling: columns (tn) and rows (nn) per thread by shape class."""
        t = BatchTiling((c_int32 * 3)(*tn), (c_int32 * 3)(*nn))
        s = self._lib.lra_batch_set_tiling(self._b, byref(t))
        if s < 0:
            raise LraError(s, "lra_batch_set_tiling")

    def tune(self, reps=2):
        """lra_batch_tune: the autotuner; returns the tiling it left in place with its
        time and the time of the tiling before (ms per run)."""
        t, best, base = BatchTiling(), c_double(), c_double()
        s = self._lib.lra_batch_tune(self._b, reps, byref(t), byref(best), byref(base))
        if s < 0:
            raise LraError(s, "lra_batch_tune")
        return {"tn": list(t.tn), "nn": list(t.nn), "ms": best.value, "base_ms": base.value}

    def device_bytes(self):
        return int(self._lib.lra_batch_device_bytes(self._b))

    def result(self, i):
        """Problem i: status, rank, E, normA2, rel_err and float32 views Q (m x rank)
        and Bt (n x rank, = B^T)."""
        r = BatchResult()
        s = self._lib.lra_batch_result(self._b, i, byref(r))
        if s < 0:
            raise LraError(s, "lra_batch_result")
        m, n = self.shapes[i]
        out = dict(status=r.status, rank=r.rank, E=r.E, normA2=r.normA2, rel_err=r.rel_err)
        if r.rank > 0:
            torch = self._torch
            out["Q"] = torch.as_tensor(_DeviceView(r.Q, (m, r.rank), (1, r.ldq), self, 4), device="cuda")
            out["Bt"] = torch.as_tensor(_DeviceView(r.Bt, (n, r.rank), (1, r.ldbt), self, 4), device="cuda")
        return out

    def close(self):
        if self._b:
            self._lib.lra_batch_destroy(self._b)
            self._b = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sketch_noalloc(A, j0, nblk, b, kind, zeta=8, p=0.0, seed=0, Y=None, stream=None):
    """lra_sketch_noalloc: the sparse sketch without a context or any device
    allocation by the library (Y is allocated here, by the caller's side, when
    not given).  Returns Y (column-major m x nblk*b)."""
    import torch
    lib = load()
    lib.lra_sketch_noalloc.argtypes = [POINTER(Matrix), POINTER(Params), c_int64, c_int64, c_void_p,
                                       c_int64, c_void_p]
    lib.lra_sketch_noalloc.restype = c_int32
    mat = _device_matrix(A, torch)
    m = A.shape[0]
    if Y is None:
        Y = torch.empty_strided((m, nblk * b), (1, m), dtype=torch.float64, device=A.device)
    else:
        # the library writes m x nblk*b doubles, column-major with ld = Y.stride(1)
        if Y.dtype != torch.float64 or Y.device != A.device or Y.dim() != 2:
            raise ValueError("Y must be a 2-D float64 tensor on A's device")
        if tuple(Y.shape) != (m, nblk * b):
            raise ValueError("Y must be m x nblk*b = %d x %d" % (m, nblk * b))
        if Y.stride(0) != 1 or (nblk * b > 1 and Y.stride(1) < m):
            raise ValueError("Y must be column-major (stride(0) == 1, stride(1) >= m)")
    prm = Params(0.0, 0, b, 0, kind, zeta, p, seed & 0xFFFFFFFFFFFFFFFF, 0, 0)
    if stream is None:
        stream = torch.cuda.current_stream()
    s = lib.lra_sketch_noalloc(byref(mat), byref(prm), j0, nblk, c_void_p(Y.data_ptr()),
                               max(Y.stride(1), m), c_void_p(stream.cuda_stream))
    if s != OK:
        raise LraError(s, "lra_sketch_noalloc failed")
    return Y
