"""gf2_rank_noalloc: the rank entry point for callers that may not allocate
device memory at call time (a fixed device-memory budget reserved at
start-up, or a framework that owns every device buffer).  Its scratch is a
static array inside the library; this file runs last so that a failure here
comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


def rank_noalloc(A: "gf2.Mat") -> int:
    lib = gf2.load()
    lib.gf2_rank_noalloc.restype = ctypes.c_int
    lib.gf2_rank_noalloc.argtypes = [ctypes.POINTER(gf2._CMat), ctypes.c_void_p, ctypes.c_void_p]
    out = torch.full((1,), -7, dtype=torch.int64, device=A.t.device)
    a = A.c()
    st = lib.gf2_rank_noalloc(ctypes.byref(a), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if st:
        raise gf2.Gf2Error(st, "gf2_rank_noalloc")
    torch.cuda.synchronize()
    return int(out.item())


def test_noalloc_rank_matches_gf2_rank_on_two_calls_in_a_row():
    # two different matrices back to back: the second call must not see the
    # first call's contents of the shared scratch
    cases = []
    X, Y = f2gen.fixed_rank_factors(1500, 1400, 700, 61)
    cases.append(gf2.mmm(gf2.Mat.from_rowmajor(X, 700), gf2.Mat.from_rowmajor(Y, 1400)))
    cases.append(gf2.Mat.from_rowmajor(f2gen.uniform(4096, 4096, 62), 4096))
    got = [rank_noalloc(A) for A in cases]
    want = [gf2.gf2_rank(A) for A in cases]
    assert got == want
    assert got[0] == 700
    # and the oracle's rank of the same inputs
    assert got == [oracle.rank(A.to_rowmajor(), A.cols, nthreads=oracle.max_threads()) for A in cases]
    # and once more in the other order
    assert [rank_noalloc(A) for A in reversed(cases)] == list(reversed(want))


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    lib = gf2.load()
    lib.gf2_rank_noalloc.restype = ctypes.c_int
    lib.gf2_rank_noalloc.argtypes = [ctypes.POINTER(gf2._CMat), ctypes.c_void_p, ctypes.c_void_p]
    big = gf2._CMat(1, 4097, 100, 4097)
    assert lib.gf2_rank_noalloc(ctypes.byref(big), ctypes.c_void_p(8), None) == gf2.GF2_ERR_UNSUPPORTED


def test_noalloc_rank_of_a_wide_matrix():
    # fewer rows than columns: this entry point decomposes the matrix itself
    # (gf2_rank goes through the transpose); both must give the known rank
    X, Y = f2gen.fixed_rank_factors(700, 4096, 333, 63)
    A = gf2.mmm(gf2.Mat.from_rowmajor(X, 333), gf2.Mat.from_rowmajor(Y, 4096))
    got = rank_noalloc(A)
    assert got == 333
    assert got == gf2.gf2_rank(A)
    assert got == oracle.rank(A.to_rowmajor(), 4096)


def test_noalloc_reports_padding_bits():
    # a bit beyond the last column (m = 100: bits 36..63 of word 1 are padding)
    words = f2gen.uniform(100, 100, 64)
    words[17, 1] |= np.uint64(1) << np.uint64(40)
    A = gf2.Mat.from_rowmajor(words, 100)
    with pytest.raises(gf2.Gf2Error) as e:
        rank_noalloc(A)
    assert e.value.status == gf2.GF2_ERR_PADDING
    # the next call on a clean matrix is unaffected
    clean = gf2.Mat.from_rowmajor(f2gen.uniform(100, 100, 65), 100)
    assert rank_noalloc(clean) == gf2.gf2_rank(clean)
