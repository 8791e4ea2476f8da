"""GB300 (sm_103a) library for dense linear algebra over F2.

Thin Python binding of the C ABI in include/gf2.h (libgf2.so, built in-tree
by ``__graft_entry__.build()`` or ``paper_1209_5198_gb300._build.build()``).
It only marshals arguments: every step of the computation runs in the CUDA
kernels of the library.  PyTorch provides device memory and streams.

The functions named like the C entry points (``gf2_mmm``, ``gf2_decompose``,
``gf2_rank``, ``gf2_decompose_host``) take ``Mat`` views of int64 CUDA
tensors holding column blocks: a tensor of shape (ceil(cols/64), ld), word
(i, q) at [q, i], bit t = column 64q+t (Section 3 of the paper).

There is no CPU fallback: if libgf2.so is missing or CUDA is unavailable the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GF2_COUNT_OPS=1 in the environment selects the op-counting build of the
# same ABI (libgf2_count.so, ``_build.build(counting=True)``): its kernels
# count their word operations for ``op_counts``; it is never the default
COUNTING = os.environ.get("GF2_COUNT_OPS") == "1"
# GF2_TRACE=1 selects the trace build (libgf2_trace.so,
# ``_build.build(trace=True)``): its decomposition kernels stamp a device
# timeline for ``trace_read``; it is never the default either
TRACING = os.environ.get("GF2_TRACE") == "1" and not COUNTING
LIB_PATH = os.path.join(_HERE, "libgf2_count.so" if COUNTING else "libgf2_trace.so" if TRACING else "libgf2.so")

GF2_OK = 0
GF2_MMM_TABLES = 2
GF2_MMM_TENSOR = 4
GF2_ERR_ARG = 1
GF2_ERR_SHAPE = 2
GF2_ERR_PADDING = 3
GF2_ERR_NOMEM = 4
GF2_ERR_CUDA = 5
GF2_ERR_TIMEOUT = 6
GF2_ERR_UNSUPPORTED = 7
GF2_NOCHECK = 1
GF2_SERVE_SERIAL = 1
KCLASS = {"panel": 0, "next": 1, "update": 2, "layout": 3, "solve": 4, "factor": 5}


class Gf2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


class _CMat(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64)]


_lib = None


def load() -> ctypes.CDLL:
    """Open libgf2.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    S = ctypes.c_size_t
    M = ctypes.POINTER(_CMat)
    lib.gf2_status_string.restype = ctypes.c_char_p
    lib.gf2_status_string.argtypes = [ctypes.c_int]
    lib.gf2_version.restype = ctypes.c_int
    lib.gf2_release_workspace.restype = ctypes.c_int
    lib.gf2_mmm_workspace_bytes.restype = S
    lib.gf2_mmm_workspace_bytes.argtypes = [I64, I64, I64, ctypes.c_uint]
    lib.gf2_mmm.restype = ctypes.c_int
    lib.gf2_mmm.argtypes = [M, M, M, ctypes.c_int, ctypes.c_uint, P, S, P]
    lib.gf2_batched_autotune.restype = ctypes.c_int
    lib.gf2_batched_autotune.argtypes = [I64, ctypes.POINTER(I64), P, P]
    lib.gf2_batched_set_c8_from.restype = ctypes.c_int
    lib.gf2_batched_set_c8_from.argtypes = [I64]
    lib.gf2_batched_c8_from.restype = I64
    lib.gf2_mmm_autotune.restype = ctypes.c_int
    lib.gf2_mmm_autotune.argtypes = [I64, ctypes.POINTER(I64), P]
    lib.gf2_tensor_peak.restype = ctypes.c_int
    lib.gf2_tensor_peak.argtypes = [I64, ctypes.POINTER(ctypes.c_double), P]
    lib.gf2_fp_decompose_workspace_bytes.restype = S
    lib.gf2_fp_decompose_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_fp_is_prime.restype = ctypes.c_int
    lib.gf2_fp_is_prime.argtypes = [ctypes.c_uint32]
    lib.gf2_fp_decompose.restype = ctypes.c_int
    lib.gf2_fp_decompose.argtypes = [P, I64, I64, I64, ctypes.c_uint32, P, P, P, P, I64, P, I64, ctypes.c_uint, P, S, P]
    lib.gf2_mmm_set_strassen_cutoff.restype = ctypes.c_int
    lib.gf2_mmm_set_strassen_cutoff.argtypes = [I64]
    lib.gf2_mmm_strassen_cutoff.restype = I64
    lib.gf2_decompose_workspace_bytes.restype = S
    lib.gf2_decompose_workspace_bytes.argtypes = [I64, I64, ctypes.c_int]
    lib.gf2_decompose.restype = ctypes.c_int
    lib.gf2_decompose.argtypes = [M, P, P, P, M, M, ctypes.c_uint, P, S, P]
    lib.gf2_nullspace_workspace_bytes.restype = S
    lib.gf2_nullspace_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_nullspace.restype = ctypes.c_int
    lib.gf2_nullspace.argtypes = [M, P, I64, M, P, S, P]
    lib.gf2_rref_workspace_bytes.restype = S
    lib.gf2_rref_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_rref.restype = ctypes.c_int
    lib.gf2_rref.argtypes = [M, P, P, S, P]
    lib.gf2_rank_workspace_bytes.restype = S
    lib.gf2_rank_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_rank.restype = ctypes.c_int
    lib.gf2_rank.argtypes = [M, ctypes.POINTER(I64), ctypes.c_uint, P, S, P]
    lib.gf2_decompose_host_workspace_bytes.restype = S
    lib.gf2_decompose_host_workspace_bytes.argtypes = [I64, I64, ctypes.c_int]
    lib.gf2_decompose_host.restype = ctypes.c_int
    lib.gf2_decompose_host.argtypes = [I64, I64, P, I64, P, P, P, P, P, ctypes.c_uint, P, S, P]
    lib.gf2_decompose_batched_workspace_bytes.restype = S
    lib.gf2_decompose_batched_workspace_bytes.argtypes = [ctypes.c_int, P, P, ctypes.c_int]
    lib.gf2_decompose_batched.restype = ctypes.c_int
    lib.gf2_decompose_batched.argtypes = [ctypes.c_int, P, P, P, P, P, P, ctypes.c_uint, P, S, P]
    lib.gf2_solve_workspace_bytes.restype = S
    lib.gf2_solve_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_solve.restype = ctypes.c_int
    lib.gf2_solve.argtypes = [M, M, P, P, P, M, M, P, ctypes.c_uint, P, S, P]
    lib.gf2_server_create.restype = ctypes.c_int
    lib.gf2_server_create.argtypes = [I64, I64, I64, ctypes.c_int, ctypes.c_uint, ctypes.POINTER(P)]
    lib.gf2_server_submit.restype = ctypes.c_int
    lib.gf2_server_submit.argtypes = [P, P, ctypes.c_int]
    lib.gf2_server_poll.restype = ctypes.c_int
    lib.gf2_server_poll.argtypes = [P, P, ctypes.c_int, I64, ctypes.POINTER(ctypes.c_int)]
    lib.gf2_server_clock_us.restype = ctypes.c_double
    lib.gf2_server_clock_us.argtypes = [P]
    lib.gf2_server_stats_read.restype = ctypes.c_int
    lib.gf2_server_stats_read.argtypes = [P, P]
    lib.gf2_server_destroy.restype = ctypes.c_int
    lib.gf2_server_destroy.argtypes = [P]
    lib.gf2_launch_count.restype = ctypes.c_int64
    lib.gf2_op_counts.restype = ctypes.c_int
    lib.gf2_op_counts.argtypes = [P, ctypes.c_int, ctypes.c_int]
    O = ctypes.POINTER(Opts)
    F = ctypes.POINTER(_CFactors)
    lib.gf2_opts_check.restype = ctypes.c_int
    lib.gf2_opts_check.argtypes = [O]
    T = ctypes.POINTER(TuneEntry)
    lib.gf2_tune_device_key.restype = ctypes.c_int
    lib.gf2_tune_device_key.argtypes = [ctypes.c_char_p, I64]
    lib.gf2_tune_put.restype = ctypes.c_int
    lib.gf2_tune_put.argtypes = [T]
    lib.gf2_tune_lookup.restype = ctypes.c_int
    lib.gf2_tune_lookup.argtypes = [ctypes.c_char_p, ctypes.c_int32, I64, I64, T, ctypes.POINTER(ctypes.c_int)]
    lib.gf2_tune_count.restype = I64
    lib.gf2_tune_clear.restype = ctypes.c_int
    lib.gf2_tune_save.restype = ctypes.c_int
    lib.gf2_tune_save.argtypes = [ctypes.c_char_p]
    lib.gf2_tune_load.restype = ctypes.c_int
    lib.gf2_tune_load.argtypes = [ctypes.c_char_p]
    lib.gf2_decompose_autotune.restype = ctypes.c_int
    lib.gf2_decompose_autotune.argtypes = [I64, I64, ctypes.c_int, T, P]
    lib.gf2_mmm_workspace_bytes_ex.restype = S
    lib.gf2_mmm_workspace_bytes_ex.argtypes = [I64, I64, I64, ctypes.c_uint, O]
    lib.gf2_mmm_ex.restype = ctypes.c_int
    lib.gf2_mmm_ex.argtypes = [M, M, M, ctypes.c_int, ctypes.c_uint, O, P, S, P]
    lib.gf2_decompose_ex.restype = ctypes.c_int
    lib.gf2_decompose_ex.argtypes = [M, P, P, P, M, M, ctypes.c_uint, O, P, S, P]
    lib.gf2_rank_ex.restype = ctypes.c_int
    lib.gf2_rank_ex.argtypes = [M, ctypes.POINTER(ctypes.c_int64), ctypes.c_uint, O, P, S, P]
    lib.gf2_decompose_batched_workspace_bytes_ex.restype = S
    lib.gf2_decompose_batched_workspace_bytes_ex.argtypes = [ctypes.c_int, P, P, ctypes.c_int, O]
    lib.gf2_decompose_batched_ex.restype = ctypes.c_int
    lib.gf2_decompose_batched_ex.argtypes = [ctypes.c_int, M, P, P, P, M, M, ctypes.c_uint, O, P, S, P]
    for name, args in (("gf2_factors_alloc", [F, I64, I64, ctypes.c_uint]), ("gf2_factors_free", [F]),
                       ("gf2_factors_decompose", [F, M, ctypes.c_uint, O, P]),
                       ("gf2_factors_rank", [F, ctypes.POINTER(ctypes.c_int64), P]),
                       ("gf2_factors_solve", [F, M, M, P, ctypes.c_uint, P]), ("gf2_factors_rref", [F, M, P]),
                       ("gf2_factors_nullspace", [F, M, P])):
        getattr(lib, name).restype = ctypes.c_int
        getattr(lib, name).argtypes = args
    lib.gf2_debug_set_wait_limit.restype = ctypes.c_int
    lib.gf2_debug_set_wait_limit.argtypes = [ctypes.c_int64]
    lib.gf2_trace_read.restype = ctypes.c_int
    lib.gf2_trace_read.argtypes = [P, ctypes.c_int64, ctypes.c_int]
    lib.gf2_timing_enable.argtypes = [ctypes.c_int]
    lib.gf2_timing_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().gf2_status_string(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != GF2_OK:
        raise Gf2Error(status, where)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


class Opts(ctypes.Structure):
    """gf2_opts of include/gf2.h: per-call options, 0 = automatic in every field."""
    _fields_ = [("panel_w", ctypes.c_int32), ("table_c", ctypes.c_int32), ("tile_words", ctypes.c_int32),
                ("backend", ctypes.c_int32), ("schedule", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("strassen_cutoff", ctypes.c_int64), ("batched_c8_from", ctypes.c_int64)]


class TuneEntry(ctypes.Structure):
    """gf2_tune_entry of include/gf2.h: the autotuner's choice for one
    (device, shape bucket)."""
    _fields_ = [("device", ctypes.c_char * 64), ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("bucket_n", ctypes.c_int64), ("bucket_m", ctypes.c_int64), ("opts", Opts), ("ms", ctypes.c_double)]


GF2_TUNE_DECOMPOSE = 0

BACKEND_AUTO, BACKEND_TABLES, BACKEND_TENSOR = 0, 1, 2
SCHEDULE_AUTO, SCHEDULE_STREAMS, SCHEDULE_PERSISTENT, SCHEDULE_SPLIT = 0, 1, 2, 3
GF2_FACTORS_RANK_ONLY = 1


def _opts(o):
    return None if o is None else ctypes.byref(o)


class Mat:
    """A rows x cols matrix over F2 in column blocks on the GPU.

    ``t`` is an int64 tensor of shape (ceil(cols/64), ld), ld >= rows.
    """

    def __init__(self, t: torch.Tensor, rows: int, cols: int):
        mu = (cols + 63) // 64
        if t.dtype != torch.int64 or t.dim() != 2 or t.shape[0] < mu or (mu and t.shape[1] < rows):
            raise ValueError("expected an int64 tensor of shape (ceil(cols/64), ld >= rows)")
        if not t.is_contiguous():
            raise ValueError("column-block tensor must be contiguous")
        self.t, self.rows, self.cols = t, int(rows), int(cols)

    @property
    def ld(self) -> int:
        return int(self.t.shape[1]) if self.t.dim() == 2 and self.t.shape[1] else max(self.rows, 1)

    def c(self) -> _CMat:
        return _CMat(self.t.data_ptr() if self.t.numel() else None, self.rows, self.cols, self.ld)

    @staticmethod
    def empty(rows: int, cols: int, device="cuda", ld: int | None = None) -> "Mat":
        ld = max(rows, 1) if ld is None else ld
        return Mat(torch.zeros(((cols + 63) // 64, ld), dtype=torch.int64, device=device), rows, cols)

    @staticmethod
    def from_rowmajor(words: np.ndarray, cols: int, device="cuda", ld: int | None = None) -> "Mat":
        """Row-major uint64 words (rows, ceil(cols/64)) -> column blocks on the device."""
        words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
        rows = words.shape[0]
        ld = max(rows, 1) if ld is None else ld
        host = np.zeros(((cols + 63) // 64, ld), dtype=np.uint64)
        host[:, :rows] = words[:, : (cols + 63) // 64].T
        return Mat(torch.from_numpy(host.view(np.int64)).to(device), rows, cols)

    def to_rowmajor(self) -> np.ndarray:
        """Column blocks on the device -> row-major uint64 words on the host."""
        host = self.t.cpu().numpy().view(np.uint64)
        return np.ascontiguousarray(host[: (self.cols + 63) // 64, : self.rows].T)


class _CFactors(ctypes.Structure):
    """gf2_factors of include/gf2.h."""
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("rank", ctypes.c_int64),
                ("perm", ctypes.c_void_p), ("pivcols", ctypes.c_void_p), ("rank_dev", ctypes.c_void_p),
                ("L", _CMat), ("E", _CMat), ("flags", ctypes.c_uint32), ("impl", ctypes.c_void_p)]


class _DeviceView:
    """__cuda_array_interface__ of library-owned device memory, so that torch
    can view it without a copy (valid while its owner lives)."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2, "strides": None}


def _view(ptr, shape, typestr, dtype) -> torch.Tensor:
    if not ptr or 0 in shape:
        return torch.zeros(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceView(ptr, shape, typestr), device="cuda")


class Factors:
    """A gf2_factors handle: the factors of one n x m decomposition in device
    memory the library owns (perm, pivcols, rank, L, E and the block form),
    with the scratch of its calls.  The tensors it hands out are views of
    that memory, valid until close()."""

    def __init__(self, n: int, m: int, rank_only: bool = False):
        self._f = _CFactors()
        _check(load().gf2_factors_alloc(ctypes.byref(self._f), n, m, GF2_FACTORS_RANK_ONLY if rank_only else 0),
               "gf2_factors_alloc")
        self.n, self.m = int(n), int(m)

    def close(self) -> None:
        if self._f.impl:
            _check(load().gf2_factors_free(ctypes.byref(self._f)), "gf2_factors_free")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def decompose(self, A: Mat, opts: Opts | None = None, flags: int = 0, stream=None) -> "Factors":
        a = A.c()
        _check(load().gf2_factors_decompose(ctypes.byref(self._f), ctypes.byref(a), flags, _opts(opts),
                                            _stream(stream)), "gf2_factors_decompose")
        return self

    def rank(self, stream=None) -> int:
        r = ctypes.c_int64(0)
        _check(load().gf2_factors_rank(ctypes.byref(self._f), ctypes.byref(r), _stream(stream)), "gf2_factors_rank")
        return int(r.value)

    @property
    def perm(self) -> torch.Tensor:
        return _view(self._f.perm, (self.n,), "<i4", torch.int32)

    @property
    def pivcols(self) -> torch.Tensor:
        return _view(self._f.pivcols, (min(self.n, self.m),), "<i4", torch.int32)

    def _mat(self, c: _CMat) -> Mat | None:
        if not c.w and c.rows and c.cols:
            return None
        t = _view(c.w, ((c.cols + 63) // 64, c.ld), "<i8", torch.int64)
        return Mat(t, c.rows, c.cols)

    @property
    def L(self) -> Mat | None:
        return self._mat(self._f.L)

    @property
    def E(self) -> Mat | None:
        return self._mat(self._f.E)

    def solve(self, B: Mat, stream=None) -> dict:
        """A X = B with the handle's factors: X (m x nrhs Mat) and the
        consistency mask (synchronises the stream)."""
        X = Mat.empty(self.m, B.cols, B.t.device)
        ok = torch.zeros(1, dtype=torch.int64, device=B.t.device)
        b, x = B.c(), X.c()
        _check(load().gf2_factors_solve(ctypes.byref(self._f), ctypes.byref(b), ctypes.byref(x), ok.data_ptr(), 0,
                                        _stream(stream)), "gf2_factors_solve")
        return dict(X=X, consistent=int(ok.cpu().numpy().view(np.uint64)[0]))

    def rref(self, stream=None) -> Mat:
        """The reduced row echelon form of E, in a new Mat (E is unchanged)."""
        R = Mat.empty(min(self.n, self.m), self.m)
        r = R.c()
        _check(load().gf2_factors_rref(ctypes.byref(self._f), ctypes.byref(r), _stream(stream)), "gf2_factors_rref")
        return R

    def nullspace(self, stream=None) -> Mat:
        """The null-space basis (m x (m - rank)); synchronises once for the rank."""
        N = Mat.empty(self.m, self.m - self.rank(stream))
        nn = N.c()
        _check(load().gf2_factors_nullspace(ctypes.byref(self._f), ctypes.byref(nn), _stream(stream)),
               "gf2_factors_nullspace")
        return N


def opts_check(o: Opts | None) -> int:
    """gf2_opts_check: the status an _ex call with these options returns first."""
    return int(load().gf2_opts_check(_opts(o)))


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------- C ABI

def gf2_mmm(A: Mat, B: Mat, C: Mat, accumulate: bool = False, flags: int = 0, workspace=None, stream=None) -> None:
    """C = A*B (or C ^= A*B) over F2.  Asynchronous on ``stream``."""
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_mmm_workspace_bytes(A.rows, A.cols, B.cols, flags), C.t.device)
    a, b, c = A.c(), B.c(), C.c()
    _check(lib.gf2_mmm(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(bool(accumulate)), flags,
                       workspace.data_ptr(), workspace.numel(), _stream(stream)), "gf2_mmm")


def gf2_decompose(A: Mat, perm: torch.Tensor, pivcols: torch.Tensor, rank: torch.Tensor,
                  L: Mat | None = None, E: Mat | None = None, flags: int = 0, workspace=None, stream=None) -> None:
    """P*A = L*E: fills perm (int32 [n]), pivcols (int32 [min(n,m)]), rank (int64 [1])
    and, when given, L (n x min(n,m)) and E (min(n,m) x m)."""
    lib = load()
    want = L is not None or E is not None
    if workspace is None:
        workspace = _workspace(lib.gf2_decompose_workspace_bytes(A.rows, A.cols, int(want)), A.t.device)
    a = A.c()
    l = L.c() if L is not None else None
    e = E.c() if E is not None else None
    _check(lib.gf2_decompose(ctypes.byref(a), _ptr(perm), _ptr(pivcols), _ptr(rank),
                             ctypes.byref(l) if l is not None else None, ctypes.byref(e) if e is not None else None,
                             flags, workspace.data_ptr(), workspace.numel(), _stream(stream)), "gf2_decompose")


def gf2_mmm_ex(A: Mat, B: Mat, C: Mat, opts: Opts | None, accumulate: bool = False, flags: int = 0, workspace=None,
               stream=None) -> None:
    """gf2_mmm with per-call options (backend, Strassen cutoff)."""
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_mmm_workspace_bytes_ex(A.rows, A.cols, B.cols, flags, _opts(opts)), C.t.device)
    a, b, c = A.c(), B.c(), C.c()
    _check(lib.gf2_mmm_ex(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(accumulate), flags, _opts(opts),
                          workspace.data_ptr(), workspace.numel(), _stream(stream)), "gf2_mmm_ex")


def gf2_decompose_ex(A: Mat, perm: torch.Tensor, pivcols: torch.Tensor, rank: torch.Tensor, L: Mat | None,
                     E: Mat | None, opts: Opts | None, flags: int = 0, workspace=None, stream=None) -> None:
    """gf2_decompose with per-call options (panel width, table size, tile)."""
    lib = load()
    want = L is not None or E is not None
    if workspace is None:
        workspace = _workspace(lib.gf2_decompose_workspace_bytes(A.rows, A.cols, int(want)), A.t.device)
    a = A.c()
    l = L.c() if L is not None else None
    e = E.c() if E is not None else None
    _check(lib.gf2_decompose_ex(ctypes.byref(a), _ptr(perm), _ptr(pivcols), _ptr(rank),
                                ctypes.byref(l) if l is not None else None, ctypes.byref(e) if e is not None else None,
                                flags, _opts(opts), workspace.data_ptr(), workspace.numel(), _stream(stream)),
           "gf2_decompose_ex")


def gf2_rank_ex(A: Mat, opts: Opts | None, flags: int = 0, workspace=None, stream=None) -> int:
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_rank_workspace_bytes(A.rows, A.cols), A.t.device)
    r = ctypes.c_int64(-1)
    a = A.c()
    _check(lib.gf2_rank_ex(ctypes.byref(a), ctypes.byref(r), flags, _opts(opts), workspace.data_ptr(),
                           workspace.numel(), _stream(stream)), "gf2_rank_ex")
    return int(r.value)


def gf2_rref(E: Mat, pivcols: torch.Tensor, workspace=None, stream=None) -> None:
    """E (an echelon factor from gf2_decompose, with its pivot columns) ->
    its reduced row echelon form, in place."""
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_rref_workspace_bytes(E.rows, E.cols), E.t.device)
    e = E.c()
    _check(lib.gf2_rref(ctypes.byref(e), _ptr(pivcols), workspace.data_ptr(), workspace.numel(), _stream(stream)),
           "gf2_rref")


def gf2_rank(A: Mat, flags: int = 0, workspace=None, stream=None) -> int:
    """rank(A); synchronises the stream."""
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_rank_workspace_bytes(A.rows, A.cols), A.t.device)
    out = ctypes.c_int64(0)
    a = A.c()
    _check(lib.gf2_rank(ctypes.byref(a), ctypes.byref(out), flags, workspace.data_ptr(), workspace.numel(),
                        _stream(stream)), "gf2_rank")
    return int(out.value)


def gf2_decompose_host(n: int, m: int, A_host: np.ndarray, perm_host: np.ndarray, pivcols_host: np.ndarray,
                       rank_host: np.ndarray, L_host: np.ndarray | None = None, E_host: np.ndarray | None = None,
                       flags: int = 0, workspace=None, stream=None, device="cuda") -> None:
    """End-to-end decomposition from host buffers (column blocks, lda = A_host.shape[1])."""
    lib = load()
    want = L_host is not None or E_host is not None
    if workspace is None:
        workspace = _workspace(lib.gf2_decompose_host_workspace_bytes(n, m, int(want)), device)
    ptr = lambda a: None if a is None else a.ctypes.data
    lda = A_host.shape[1] if A_host.ndim == 2 else max(n, 1)
    _check(lib.gf2_decompose_host(n, m, ptr(A_host), lda, ptr(perm_host), ptr(pivcols_host), ptr(rank_host),
                                  ptr(L_host), ptr(E_host), flags, workspace.data_ptr(), workspace.numel(),
                                  _stream(stream)), "gf2_decompose_host")


def gf2_decompose_batched(As: list, perms: list, pivcols: list, ranks: torch.Tensor,
                          Ls: list | None = None, Es: list | None = None, flags: int = 0, workspace=None,
                          stream=None) -> None:
    """Decomposes every matrix of As in one launch (outputs as gf2_decompose;
    ranks: int64 [len(As)] on the device).  Synchronises the stream."""
    lib = load()
    count = len(As)
    if count == 0:
        return
    ns = (ctypes.c_int64 * count)(*[a.rows for a in As])
    ms = (ctypes.c_int64 * count)(*[a.cols for a in As])
    want = Ls is not None
    if workspace is None:
        workspace = _workspace(lib.gf2_decompose_batched_workspace_bytes(count, ns, ms, int(want)), ranks.device)
    A_arr = (_CMat * count)(*[a.c() for a in As])
    P_arr = (ctypes.c_void_p * count)(*[_ptr(p) for p in perms])
    V_arr = (ctypes.c_void_p * count)(*[_ptr(p) for p in pivcols])
    L_arr = (_CMat * count)(*[x.c() for x in Ls]) if want else None
    E_arr = (_CMat * count)(*[x.c() for x in Es]) if want else None
    _check(lib.gf2_decompose_batched(count, A_arr, P_arr, V_arr, _ptr(ranks), L_arr, E_arr, flags,
                                     workspace.data_ptr(), workspace.numel(), _stream(stream)),
           "gf2_decompose_batched")


def gf2_solve(L: Mat, E: Mat, perm: torch.Tensor, pivcols: torch.Tensor, rank: torch.Tensor, B: Mat, X: Mat,
              consistent: torch.Tensor, flags: int = 0, workspace=None, stream=None) -> None:
    """A X = B from the factors gf2_decompose wrote (B: n x nrhs, X: m x nrhs,
    nrhs <= 64; consistent: int64 [1] on the device).  Synchronises the stream."""
    lib = load()
    n, m = B.rows, X.rows
    if workspace is None:
        workspace = _workspace(lib.gf2_solve_workspace_bytes(n, m), B.t.device)
    l, e, b, x = L.c(), E.c(), B.c(), X.c()
    _check(lib.gf2_solve(ctypes.byref(l), ctypes.byref(e), _ptr(perm), _ptr(pivcols), _ptr(rank), ctypes.byref(b),
                         ctypes.byref(x), _ptr(consistent), flags, workspace.data_ptr(), workspace.numel(),
                         _stream(stream)), "gf2_solve")


# ----------------------------------------------------------------- helpers

def decompose(A: Mat, factors: bool = True, flags: int = 0, stream=None) -> dict:
    """Allocates the outputs and runs gf2_decompose; returns tensors on the device."""
    n, m = A.rows, A.cols
    k = min(n, m)
    dev = A.t.device
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    piv = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    rank = torch.zeros(1, dtype=torch.int64, device=dev)
    L = Mat.empty(n, k, dev) if factors else None
    E = Mat.empty(k, m, dev) if factors else None
    gf2_decompose(A, perm, piv, rank, L, E, flags=flags, stream=stream)
    return dict(perm=perm[:n], pivcols=piv[:k], rank=rank, L=L, E=E)


def decompose_batched(As: list, factors: bool = True, flags: int = 0, stream=None) -> list:
    """Allocates the outputs and runs gf2_decompose_batched; returns one dict
    per matrix as decompose() does (rank as an int64 tensor view)."""
    if not As:
        return []
    dev = As[0].t.device
    perms = [torch.empty(max(a.rows, 1), dtype=torch.int32, device=dev) for a in As]
    pivs = [torch.empty(max(min(a.rows, a.cols), 1), dtype=torch.int32, device=dev) for a in As]
    ranks = torch.zeros(len(As), dtype=torch.int64, device=dev)
    Ls = [Mat.empty(a.rows, min(a.rows, a.cols), dev) for a in As] if factors else None
    Es = [Mat.empty(min(a.rows, a.cols), a.cols, dev) for a in As] if factors else None
    gf2_decompose_batched(As, perms, pivs, ranks, Ls, Es, flags=flags, stream=stream)
    out = []
    for i, a in enumerate(As):
        k = min(a.rows, a.cols)
        out.append(dict(perm=perms[i][:a.rows], pivcols=pivs[i][:k], rank=ranks[i:i + 1],
                        L=Ls[i] if factors else None, E=Es[i] if factors else None))
    return out


def gf2_nullspace(R: Mat, pivcols: torch.Tensor, rank: int, N: Mat, workspace=None, stream=None) -> None:
    """N (m x (m - rank)) <- the null-space basis read off the reduced row
    echelon form R and its pivot columns."""
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.gf2_nullspace_workspace_bytes(R.cols, rank), N.t.device)
    r, nn = R.c(), N.c()
    _check(lib.gf2_nullspace(ctypes.byref(r), _ptr(pivcols), int(rank), ctypes.byref(nn), workspace.data_ptr(),
                             workspace.numel(), _stream(stream)), "gf2_nullspace")


def nullspace(A: Mat, stream=None) -> Mat:
    """A basis of {x : A x = 0} as the columns of an m x (m - rank) Mat:
    decompose, reduce E, read the basis off (synchronises once for the rank)."""
    out = decompose(A, stream=stream)
    R = rref(out, stream=stream)
    r = int(out["rank"].item())
    N = Mat.empty(A.cols, A.cols - r, A.t.device)
    gf2_nullspace(R, out["pivcols"], r, N, stream=stream)
    return N


def rref(factors: dict, stream=None) -> Mat:
    """The reduced row echelon form of the E factor of decompose() (in place;
    returns it)."""
    gf2_rref(factors["E"], factors["pivcols"], stream=stream)
    return factors["E"]


def solve(factors: dict, B: Mat, m: int, stream=None) -> dict:
    """Solves A X = B with the output of decompose(); returns X (Mat, m x nrhs)
    and the consistency mask (int)."""
    X = Mat.empty(m, B.cols, B.t.device)
    ok = torch.zeros(1, dtype=torch.int64, device=B.t.device)
    gf2_solve(factors["L"], factors["E"], factors["perm"], factors["pivcols"], factors["rank"], B, X, ok,
              stream=stream)
    return dict(X=X, consistent=int(ok.cpu().numpy().view(np.uint64)[0]))


def mmm(A: Mat, B: Mat, flags: int = 0, stream=None) -> Mat:
    C = Mat.empty(A.rows, B.cols, A.t.device)
    gf2_mmm(A, B, C, flags=flags, stream=stream)
    return C


STRASSEN_OFF = 1 << 62


def mmm_autotune(max_dim: int = 32768, stream=None) -> int:
    """Times M4RM against one Strassen-Winograd level on this device and sets
    the product's Strassen cutoff (returned; STRASSEN_OFF when never faster)."""
    out = ctypes.c_int64(0)
    _check(load().gf2_mmm_autotune(int(max_dim), ctypes.byref(out), _stream(stream)), "gf2_mmm_autotune")
    return int(out.value)


def tune_device_key() -> str:
    """The current device's key in the autotuner's table."""
    buf = ctypes.create_string_buffer(64)
    _check(load().gf2_tune_device_key(buf, 64), "gf2_tune_device_key")
    return buf.value.decode()


def tune_put(entry: TuneEntry) -> None:
    _check(load().gf2_tune_put(ctypes.byref(entry)), "gf2_tune_put")


def tune_lookup(device: str, n: int, m: int, kind: int = GF2_TUNE_DECOMPOSE):
    """The entry of (device, kind) for the shape bucket of n x m, or None."""
    out, found = TuneEntry(), ctypes.c_int(0)
    _check(load().gf2_tune_lookup(device.encode(), kind, int(n), int(m), ctypes.byref(out), ctypes.byref(found)),
           "gf2_tune_lookup")
    return out if found.value else None


def tune_count() -> int:
    return int(load().gf2_tune_count())


def tune_clear() -> None:
    _check(load().gf2_tune_clear(), "gf2_tune_clear")


def tune_save(path: str) -> None:
    _check(load().gf2_tune_save(os.fsencode(path)), "gf2_tune_save")


def tune_load(path: str) -> None:
    _check(load().gf2_tune_load(os.fsencode(path)), "gf2_tune_load")


def decompose_autotune(n: int, m: int, factors: bool = True, stream=None) -> TuneEntry:
    """Times the decomposition's speed-only options on this device for an
    n x m matrix, records the fastest for its shape bucket (used by later
    calls with automatic options) and returns it."""
    out = TuneEntry()
    _check(load().gf2_decompose_autotune(int(n), int(m), int(bool(factors)), ctypes.byref(out), _stream(stream)),
           "gf2_decompose_autotune")
    return out


def fp_decompose(A: torch.Tensor, p: int, factors: bool = True, flags: int = 0, workspace=None, stream=None) -> dict:
    """P A = L E over the prime field F_p (gf2_fp_decompose): A is an n x m
    int32 CUDA tensor of residues (row-major, rows contiguous).  Returns perm,
    pivcols, rank (int64 tensor; -1 when a bounded device wait gave up) and,
    with factors, L (n x k) and E (k x m) as int32 tensors of residues."""
    if A.dtype != torch.int32 or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("expected a 2-d int32 tensor with contiguous rows")
    n, m = A.shape
    k = min(n, m)
    dev = A.device
    lib = load()
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    piv = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    rank = torch.zeros(1, dtype=torch.int64, device=dev)
    L = torch.empty((n, k), dtype=torch.int32, device=dev) if factors else None
    E = torch.empty((k, m), dtype=torch.int32, device=dev) if factors else None
    if workspace is None:
        workspace = _workspace(lib.gf2_fp_decompose_workspace_bytes(n, m), dev)
    _check(lib.gf2_fp_decompose(A.data_ptr() if A.numel() else None, max(A.stride(0), m), n, m, int(p), perm.data_ptr(),
                                piv.data_ptr(), rank.data_ptr(), _ptr(L), max(k, 1), _ptr(E), max(m, 1), flags,
                                workspace.data_ptr(), workspace.numel(), _stream(stream)), "gf2_fp_decompose")
    return dict(perm=perm[:n], pivcols=piv[:k], rank=rank, L=L, E=E)


def fp_is_prime(p: int) -> bool:
    return bool(load().gf2_fp_is_prime(int(p)))


def tensor_peak(iters: int = 4096, stream=None) -> float:
    """Dense TFLOP/s of the tensor pipe for the tensor backend's MMA shape
    (tcgen05 kind::f8f6f4, 128 x 256 x 32) from shared memory, one CTA per SM."""
    out = ctypes.c_double(0)
    _check(load().gf2_tensor_peak(int(iters), ctypes.byref(out), _stream(stream)), "gf2_tensor_peak")
    return float(out.value)


def batched_autotune(max_dim: int = 4096, stream=None, times: dict | None = None) -> int:
    """Times the batched kernel with 4- and 8-bit tables on this device and
    sets the size from which matrices take the 8-bit tables (returned).
    `times`, when given, receives {d: (ms with 4-bit, ms with 8-bit)}."""
    out = ctypes.c_int64(0)
    dims = []
    d = 128
    while d <= min(int(max_dim), 4096):
        dims.append(d)
        d *= 2
    buf = (ctypes.c_float * (2 * max(1, len(dims))))()
    _check(load().gf2_batched_autotune(int(max_dim), ctypes.byref(out), buf, _stream(stream)), "gf2_batched_autotune")
    if times is not None:
        for i, d in enumerate(dims):
            times[d] = (float(buf[2 * i]), float(buf[2 * i + 1]))
    return int(out.value)


def set_batched_c8_from(dim: int) -> None:
    _check(load().gf2_batched_set_c8_from(int(dim)), "gf2_batched_set_c8_from")


def batched_c8_from() -> int:
    return int(load().gf2_batched_c8_from())


def set_strassen_cutoff(cutoff: int) -> None:
    _check(load().gf2_mmm_set_strassen_cutoff(int(cutoff)), "gf2_mmm_set_strassen_cutoff")


def strassen_cutoff() -> int:
    return int(load().gf2_mmm_strassen_cutoff())


# ------------------------------------------------------------- diagnostics

def launch_count() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(load().gf2_launch_count())


# the counters of gf2_op_counts, in the order of GF2_OP_* (include/gf2.h)
OPS = ("updates", "yrows", "lookups8", "lookups4", "table8", "table4", "mmm_lookups", "mmm_table", "mmm_adds")


def op_counts(reset: bool = False) -> dict:
    """Word-operation counters of the op-counting build (GF2_COUNT_OPS=1):
    synchronises the device, returns {name: count} and optionally zeroes
    them.  The release build raises Gf2Error(GF2_ERR_UNSUPPORTED)."""
    out = (ctypes.c_uint64 * len(OPS))()
    _check(load().gf2_op_counts(ctypes.cast(out, ctypes.c_void_p), len(OPS), int(reset)), "gf2_op_counts")
    return {k: int(v) for k, v in zip(OPS, out)}


def set_wait_limit(polls: int) -> None:
    """gf2_debug_set_wait_limit: polls after which a bounded device wait gives
    up (0: the defaults); for tests that make a wait run out."""
    _check(load().gf2_debug_set_wait_limit(int(polls)), "gf2_debug_set_wait_limit")


TRACE_PANELS = 4096
TRACE_SLOTS = ("panel_start", "panel_loaded", "panel_loop", "panel_end", "next_start", "next_end", "rest_start",
               "rest_end", "panel_uinv", "panel_t", "panel_tinv", "panel_zp", "panel_entry")


def trace_read(reset: bool = False) -> dict:
    """The trace build's device timeline (GF2_TRACE=1): {slot: int64 array of
    nanosecond stamps per panel, 0 = none}; see gf2_trace_read.  The release
    build raises Gf2Error(GF2_ERR_UNSUPPORTED)."""
    out = np.zeros(len(TRACE_SLOTS) * TRACE_PANELS, dtype=np.uint64)
    _check(load().gf2_trace_read(ctypes.c_void_p(out.ctypes.data), out.size, int(reset)), "gf2_trace_read")
    v = out.astype(np.int64).reshape(len(TRACE_SLOTS), TRACE_PANELS)
    return {k: v[i] for i, k in enumerate(TRACE_SLOTS)}


def timing(on: bool) -> None:
    """Bracket every launch with CUDA events on its stream (grouped by class)."""
    lib = load()
    lib.gf2_timing_reset()
    lib.gf2_timing_enable(int(bool(on)))


def timing_read() -> dict:
    """{class: (total device ms, launches)} since timing was switched on."""
    lib = load()
    out = {}
    for name, cls in KCLASS.items():
        ms = ctypes.c_double(0)
        cnt = ctypes.c_int64(0)
        _check(lib.gf2_timing_read(cls, ctypes.byref(ms), ctypes.byref(cnt)), "gf2_timing_read")
        out[name] = (ms.value, cnt.value)
    return out


# ------------------------------------------------------------- serving

# gf2_request / gf2_completion / gf2_server_stats of include/gf2.h, as numpy
# record types (C layout: align=True)
REQUEST_DTYPE = np.dtype([("id", "<u8"), ("matrix", "<u8"), ("n", "<i8"), ("m", "<i8"), ("A", "<u8"),
                          ("lda", "<i8"), ("nrhs", "<i4"), ("B", "<u8"), ("X", "<u8"), ("arrival_us", "<f8")],
                         align=True)
COMPLETION_DTYPE = np.dtype([("id", "<u8"), ("status", "<i4"), ("hit", "<i4"), ("rank", "<i8"),
                             ("consistent", "<u8"), ("arrival_us", "<f8"), ("admit_us", "<f8"),
                             ("done_us", "<f8")], align=True)
STATS_FIELDS = ("completed", "hits", "misses", "evictions", "solve_launches", "batched_decompositions",
                "plain_decompositions", "max_batch", "resident_bytes", "arena_bytes", "admitted_in_flight",
                "overlapped_launches")


class Server:
    """The serving engine (gf2_server_*): rank / solve requests on resident
    factors, continuous batching on the GPU (or, with ``serial=True``, one
    request at a time through gf2_decompose and gf2_solve).

    Requests are REQUEST_DTYPE records whose A, B, X fields are HOST
    addresses; those buffers must stay alive until the request completes.
    """

    def __init__(self, device_bytes: int, max_n: int, max_m: int, max_batch: int = 1024, serial: bool = False):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.gf2_server_create(int(device_bytes), int(max_n), int(max_m), int(max_batch),
                                     GF2_SERVE_SERIAL if serial else 0, ctypes.byref(h)), "gf2_server_create")
        self._h = h
        self._lib = lib

    def submit(self, requests: np.ndarray) -> None:
        requests = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
        _check(self._lib.gf2_server_submit(self._h, requests.ctypes.data, len(requests)), "gf2_server_submit")

    def poll(self, max_count: int = 4096, wait_us: int = 0) -> np.ndarray:
        out = np.zeros(max_count, dtype=COMPLETION_DTYPE)
        got = ctypes.c_int(0)
        _check(self._lib.gf2_server_poll(self._h, out.ctypes.data, max_count, int(wait_us), ctypes.byref(got)),
               "gf2_server_poll")
        return out[: got.value]

    def wait_all(self, count: int, timeout_s: float = 600.0) -> np.ndarray:
        """Completions until `count` have arrived (raises after timeout_s)."""
        import time
        parts, have = [], 0
        t_end = time.monotonic() + timeout_s
        while have < count:
            if time.monotonic() > t_end:
                raise TimeoutError(f"{have} of {count} requests completed")
            c = self.poll(4096, 20000)
            parts.append(c)
            have += len(c)
        return np.concatenate(parts) if parts else np.zeros(0, dtype=COMPLETION_DTYPE)

    def clock_us(self) -> float:
        return float(self._lib.gf2_server_clock_us(self._h))

    def stats(self) -> dict:
        raw = (ctypes.c_int64 * len(STATS_FIELDS))()
        _check(self._lib.gf2_server_stats_read(self._h, ctypes.byref(raw)), "gf2_server_stats_read")
        return dict(zip(STATS_FIELDS, list(raw)))

    def close(self) -> None:
        if self._h:
            _check(self._lib.gf2_server_destroy(self._h), "gf2_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def host_colblocks(rowmajor: np.ndarray, cols: int, pinned: bool = True) -> torch.Tensor:
    """Row-major words -> column blocks (ceil(cols/64), rows) in a host int64
    tensor (pinned by default), for the serving requests' A."""
    words = np.ascontiguousarray(np.asarray(rowmajor, dtype=np.uint64))
    mu = (cols + 63) // 64
    t = torch.empty((mu, words.shape[0]), dtype=torch.int64, pin_memory=pinned)
    t.numpy().view(np.uint64)[:] = words[:, :mu].T
    return t
