"""Parity of the null-space basis (gf2_nullspace, read off the reduced row
echelon form) with the oracle's, bit for bit, and of gf2_rank's transposed
route for wide matrices (n < m) with the oracle's rank."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


def fixed_rank(n, m, r, seed):
    X, Y = f2gen.fixed_rank_factors(n, m, r, seed)
    return oracle.mmm(X, Y, r, m, nthreads=oracle.max_threads()), m


NULL_CASES = {
    "wide-300x1000": lambda: (f2gen.uniform(300, 1000, f2gen.BASE_SEED, 51), 1000),
    "wide-64x4096": lambda: (f2gen.uniform(64, 4096, f2gen.BASE_SEED, 52), 4096),
    "ragged-777x2111": lambda: (f2gen.uniform(777, 2111, 53), 2111),
    "square-1024": lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
    "tall-2000x500": lambda: (f2gen.uniform(2000, 500, 54), 500),
    "rank-600-1024": lambda: fixed_rank(1024, 1024, 600, 55),
    "rank-1-300x700": lambda: fixed_rank(300, 700, 1, 56),
    "sparse2-1000": lambda: (f2gen.sparse_rows(1000, 1000, 2, 57), 1000),
    "zero-50x200": lambda: (np.zeros((50, 4), dtype=np.uint64), 200),
    "one-row": lambda: (f2gen.uniform(1, 700, 58), 700),
    "one-col": lambda: (np.ones((5, 1), dtype=np.uint64), 1),
}


@pytest.mark.parametrize("name", sorted(NULL_CASES))
def test_nullspace_matches_oracle(name):
    A, m = NULL_CASES[name]()
    N = gf2.nullspace(gf2.Mat.from_rowmajor(A, m))
    torch.cuda.synchronize()
    ref = oracle.nullspace(A, m)
    assert N.cols == ref["nul"] and N.rows == m
    if ref["nul"]:
        assert np.array_equal(N.to_rowmajor(), ref["N"]), "basis differs"


def test_nullspace_annihilates_large():
    """8192 x 32768 Bernoulli(1/2): nullity 24576; A N = 0 by the library's
    product, checked on the host, and the rows at the free columns form the
    identity (so the columns are independent)."""
    n, m = 8192, 32768
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 59)
    M = gf2.Mat.from_rowmajor(A, m)
    N = gf2.nullspace(M)
    assert N.cols == m - n  # full row rank with overwhelming probability
    P = gf2.mmm(M, N)
    torch.cuda.synchronize()
    assert not P.t.any().item()
    out = gf2.decompose(M)
    piv = out["pivcols"][: n].cpu().numpy()
    free = np.setdiff1d(np.arange(m), piv)
    rows = np.random.default_rng(3).choice(free.size, 64, replace=False)
    Nh = N.to_rowmajor()
    for j in rows:
        w = Nh[free[j]]
        assert w[j // 64] == np.uint64(1) << np.uint64(j % 64) and np.count_nonzero(w) == 1


def test_nullspace_errors():
    lib = gf2.load()
    R = gf2.Mat.empty(10, 100)
    piv = torch.arange(10, dtype=torch.int32, device="cuda")
    bad = gf2.Mat.empty(100, 80)  # should be 100 x 90
    r, b = R.c(), bad.c()
    assert lib.gf2_nullspace(gf2.ctypes.byref(r), piv.data_ptr(), 10, gf2.ctypes.byref(b), None, 0, None) == gf2.GF2_ERR_SHAPE
    assert lib.gf2_nullspace(gf2.ctypes.byref(r), piv.data_ptr(), 11, gf2.ctypes.byref(b), None, 0, None) == gf2.GF2_ERR_ARG
    assert lib.gf2_nullspace(None, None, 0, None, None, 0, None) == gf2.GF2_ERR_ARG


RANK_WIDE = {
    "100x5000": lambda: (f2gen.uniform(100, 5000, 61), 5000),
    "777x2111": lambda: (f2gen.uniform(777, 2111, 62), 2111),
    "1x700": lambda: (f2gen.uniform(1, 700, 63), 700),
    "500x3000-rank-37": lambda: fixed_rank(500, 3000, 37, 64),
    "64x65": lambda: (f2gen.uniform(64, 65, 65), 65),
    "1000x1001-rank-990": lambda: fixed_rank(1000, 1001, 990, 66),
    "sparse-300x2000": lambda: (f2gen.sparse_rows(300, 2000, 3, 67), 2000),
}


@pytest.mark.parametrize("name", sorted(RANK_WIDE))
def test_rank_of_wide_matrices_through_the_transpose(name):
    A, m = RANK_WIDE[name]()
    n = A.shape[0]
    M = gf2.Mat.from_rowmajor(A, m, ld=n + 5)
    # rows past n in the buffer are not part of A: fill them with ones
    M.t[:, n:] = -1
    assert gf2.gf2_rank(M) == oracle.rank(A, m)


def test_rank_of_wide_matrix_padding_error():
    A = f2gen.uniform(100, 300, 68)
    M = gf2.Mat.from_rowmajor(A, 300)
    M.t[-1, 7] |= 1 << 50  # column 64*4 + 50 = 306 >= 300
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.gf2_rank(M)
    assert e.value.status == gf2.GF2_ERR_PADDING
    assert gf2.gf2_rank(M, flags=gf2.GF2_NOCHECK) >= 0  # unchecked: no error
