"""Plain CPU oracle for the F2 decomposition (ctypes wrapper of f2_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports
it.  All matrices here are numpy arrays of uint64 words in ROW-MAJOR packing
(shape (rows, ceil(cols/64)), bit t of word q = column 64q+t).

Which passage of the paper each function follows is stated in f2_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "f2_oracle.c")
_LIB = os.path.join(_HERE, "libf2oracle.so")
_lib = None

_P64 = ctypes.POINTER(ctypes.c_uint64)
_P32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile f2_oracle.c into libf2oracle.so next to it (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def load_library(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    lib.f2o_ple.argtypes = [_I64, _I64, _P64, _I64, _P32, _P32, _PI64, _P64, _I64, _P64, _I64, _I64, ctypes.c_int]
    lib.f2o_blockdecomp.argtypes = [_I64, _I64, ctypes.c_int, _P64, _I64, _P32, _P32, _PI64, _P32, _P64]
    lib.f2o_mmm.argtypes = [_I64, _I64, _I64, _P64, _I64, _P64, _I64, _P64, _I64, ctypes.c_int, ctypes.c_int]
    lib.f2o_rref.argtypes = [_I64, _I64, _P64, _I64, _P64, _I64, _P32, _PI64]
    lib.f2o_solve.argtypes = [_I64, _I64, _P64, _I64, ctypes.c_int, _P64, _P64, _P64]
    lib.f2o_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


def _w(a):
    return a.ctypes.data_as(_P64) if a is not None else None


def _i32(a):
    return a.ctypes.data_as(_P32) if a is not None else None


def _words(a: np.ndarray, cols: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    mu = (cols + 63) // 64
    if a.ndim != 2 or a.shape[1] < mu:
        raise ValueError("expected a (rows, ceil(cols/64)) uint64 array")
    if a.shape[1] == 0:
        a = np.zeros((a.shape[0], 1), dtype=np.uint64)
    return a


def max_threads() -> int:
    return int(_load().f2o_max_threads())


def ple(A: np.ndarray, m: int, want_L: bool = True, want_E: bool = True,
        col_limit: int = -1, nthreads: int = 1) -> dict:
    """P*A = L*E by bit-level elimination with the paper's pivot rule.

    Returns dict(perm, pivcols, rank, L, E): perm int32 (n,), pivcols int32
    (rank,), L words (n, ceil(min(n,m)/64)), E words (min(n,m), ceil(m/64)).
    """
    lib = _load()
    n = A.shape[0]
    A = _words(A, m)
    kmax = min(n, m)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    piv = np.zeros(max(kmax, 1), dtype=np.int32)
    rank = ctypes.c_int64(0)
    lw = max((kmax + 63) // 64, 1)
    L = np.zeros((max(n, 1), lw), dtype=np.uint64) if want_L else None
    E = np.zeros((max(kmax, 1), A.shape[1]), dtype=np.uint64) if want_E else None
    rc = lib.f2o_ple(n, m, _w(A), A.shape[1], _i32(perm), _i32(piv), ctypes.byref(rank),
                     _w(L), lw, _w(E), A.shape[1], col_limit, nthreads)
    if rc:
        raise RuntimeError(f"f2o_ple failed ({rc})")
    r = rank.value
    out = dict(perm=perm[:n], pivcols=piv[:r].copy(), rank=r)
    out["L"] = L[:n, : (kmax + 63) // 64] if want_L else None
    out["E"] = E[:kmax, : (m + 63) // 64] if want_E else None
    return out


def blockdecomp(A: np.ndarray, m: int, b: int) -> dict:
    """The paper's iterative block algorithm (Procedure buildZ) with word size b.

    Returns dict(perm, pivcols, rank, rblock, Wb) where Wb is the final
    in-place storage of Figure 1 as b-bit column blocks, shape (ceil(m/b), n).
    """
    lib = _load()
    n = A.shape[0]
    A = _words(A, m)
    mub = (m + b - 1) // b
    perm = np.zeros(max(n, 1), dtype=np.int32)
    piv = np.zeros(max(min(n, m), 1), dtype=np.int32)
    rb = np.zeros(max(mub, 1), dtype=np.int32)
    Wb = np.zeros(max(mub * n, 1), dtype=np.uint64)
    rank = ctypes.c_int64(0)
    rc = lib.f2o_blockdecomp(n, m, b, _w(A), A.shape[1], _i32(perm), _i32(piv), ctypes.byref(rank),
                             _i32(rb), _w(Wb))
    if rc:
        raise RuntimeError(f"f2o_blockdecomp failed ({rc})")
    r = rank.value
    return dict(perm=perm[:n], pivcols=piv[:r].copy(), rank=r, rblock=rb[:mub],
                Wb=Wb[: mub * n].reshape(mub, n))


def mmm(A: np.ndarray, B: np.ndarray, k: int, m: int, C: np.ndarray | None = None,
        nthreads: int = 1) -> np.ndarray:
    """C = A*B over F2 (or C ^= A*B if C is given); A is n x k, B is k x m."""
    lib = _load()
    n = A.shape[0]
    A = _words(A, k)
    B = _words(B, m) if B.shape[0] else np.zeros((0, max((m + 63) // 64, 1)), dtype=np.uint64)
    mu = max((m + 63) // 64, 1)
    acc = C is not None
    out = np.ascontiguousarray(C.copy() if acc else np.zeros((max(n, 1), mu), dtype=np.uint64))
    if out.shape[1] < mu:
        out = np.concatenate([out, np.zeros((out.shape[0], mu - out.shape[1]), dtype=np.uint64)], axis=1)
    rc = lib.f2o_mmm(n, k, m, _w(A), A.shape[1], _w(B), B.shape[1], _w(out), out.shape[1], int(acc), nthreads)
    if rc:
        raise RuntimeError(f"f2o_mmm failed ({rc})")
    return out[:n, : (m + 63) // 64]


def rref(A: np.ndarray, m: int) -> dict:
    """Reduced row echelon form: dict(R (rank rows), pivcols, rank)."""
    lib = _load()
    n = A.shape[0]
    A = _words(A, m)
    R = np.zeros((max(n, 1), A.shape[1]), dtype=np.uint64)
    piv = np.zeros(max(n, 1), dtype=np.int32)
    rank = ctypes.c_int64(0)
    rc = lib.f2o_rref(n, m, _w(A), A.shape[1], _w(R), A.shape[1], _i32(piv), ctypes.byref(rank))
    if rc:
        raise RuntimeError(f"f2o_rref failed ({rc})")
    r = rank.value
    return dict(R=R[:r, : (m + 63) // 64], pivcols=piv[:r].copy(), rank=r)


def solve(A: np.ndarray, m: int, B: np.ndarray, nrhs: int) -> dict:
    """A X = B for nrhs <= 64 packed right-hand sides (B: one word per row).

    Returns dict(X (m,) words with free variables 0, consistent bit mask).
    """
    lib = _load()
    n = A.shape[0]
    A = _words(A, m)
    B = np.ascontiguousarray(np.asarray(B, dtype=np.uint64).reshape(-1))
    X = np.zeros(max(m, 1), dtype=np.uint64)
    ok = ctypes.c_uint64(0)
    Bp = B if B.size else np.zeros(1, dtype=np.uint64)
    rc = lib.f2o_solve(n, m, _w(A), A.shape[1], nrhs, _w(Bp), _w(X), ctypes.byref(ok))
    if rc:
        raise RuntimeError(f"f2o_solve failed ({rc})")
    return dict(X=X[:m], consistent=ok.value)


def rank(A: np.ndarray, m: int, nthreads: int = 1) -> int:
    return ple(A, m, want_L=False, want_E=False, nthreads=nthreads)["rank"]


def _unpack(words: np.ndarray, cols: int) -> np.ndarray:
    """Row-major uint64 words -> bool (rows, cols), bit t of word q = column 64q+t."""
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    if cols == 0 or words.shape[0] == 0:
        return np.zeros((words.shape[0], cols), dtype=bool)
    by = words.view(np.uint8).reshape(words.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :cols].astype(bool)


def _pack(bits: np.ndarray) -> np.ndarray:
    """bool (rows, cols) -> row-major uint64 words (rows, max(1, ceil(cols/64)))."""
    rows, cols = bits.shape
    mu = max(1, (cols + 63) // 64)
    padded = np.zeros((rows, 64 * mu), dtype=np.uint8)
    padded[:, :cols] = bits
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint64).reshape(rows, mu)


def nullspace(A: np.ndarray, m: int) -> dict:
    """A basis of {x : A x = 0}, read off the reduced row echelon form as in
    the textbook: for the j-th free (non-pivot) column f_j, in increasing
    order, basis vector j has x[f_j] = 1, x[pivcols[t]] = R[t][f_j] and every
    other entry 0.  Returns dict(N row-major words (m, ceil(nul/64)) with row
    i = variable i and bit j = basis vector j, nul, rank)."""
    red = rref(A, m)
    r, piv = red["rank"], red["pivcols"].astype(np.int64)
    Rb = _unpack(red["R"], m)
    free = np.setdiff1d(np.arange(m), piv)
    nul = m - r
    Nb = np.zeros((m, nul), dtype=bool)
    Nb[free, np.arange(nul)] = True
    if r and nul:
        Nb[piv, :] = Rb[:, free]
    return dict(N=_pack(Nb), nul=nul, rank=r)


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))
