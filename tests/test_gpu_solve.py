"""Parity of the CUDA solve A X = B (forward substitution with L, consistency,
back substitution with E, free variables 0) with the oracle's Gauss-Jordan
solve, bit for bit (X and the consistency mask), through the C ABI."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


def make_rhs(A_rm, n, m, nrhs, n_consistent, seed):
    """B: the first n_consistent right-hand sides are A*X0 (solvable), the rest
    are random (solvable only when they fall in the column space)."""
    X0 = f2gen.rhs_from_solution(nrhs, m, seed)
    B = oracle.mmm(A_rm, X0, m, nrhs).reshape(-1) if m > 0 else np.zeros(n, dtype=np.uint64)
    R = f2gen.uniform(n, nrhs, seed, 77).reshape(-1)
    keep = np.uint64(0) if n_consistent == 0 else np.uint64((1 << n_consistent) - 1)
    return (B & keep) | (R & ~keep & np.uint64((1 << nrhs) - 1 if nrhs < 64 else (1 << 64) - 1))


def gpu_solve(A_rm, m, B_words, nrhs):
    n = A_rm.shape[0]
    A = gf2.Mat.from_rowmajor(A_rm, m, ld=n + 5)
    fac = gf2.decompose(A, factors=True)
    B = gf2.Mat.from_rowmajor(B_words.reshape(-1, 1), nrhs, ld=n + 2)
    out = gf2.solve(fac, B, m)
    X = out["X"].to_rowmajor().reshape(-1)
    # B is an input: untouched
    assert np.array_equal(B.to_rowmajor().reshape(-1), B_words)
    return X, out["consistent"]


def check(A_rm, m, nrhs, n_consistent, seed):
    n = A_rm.shape[0]
    Bw = make_rhs(A_rm, n, m, nrhs, n_consistent, seed)
    X, ok = gpu_solve(A_rm, m, Bw, nrhs)
    ref = oracle.solve(A_rm, m, Bw, nrhs)
    assert ok == ref["consistent"], (hex(ok), hex(ref["consistent"]))
    assert np.array_equal(X, ref["X"]), "X differs"
    # the consistent columns really solve the system
    full = (1 << nrhs) - 1 if nrhs < 64 else (1 << 64) - 1
    if n_consistent:
        assert ok & ((1 << n_consistent) - 1) == (1 << n_consistent) - 1
    AX = oracle.mmm(A_rm, X.reshape(-1, 1), m, nrhs).reshape(-1) if m > 0 else np.zeros(n, dtype=np.uint64)
    mask = np.uint64(ok & full)
    assert np.array_equal(AX & mask, Bw & mask)


CASES = {
    "tiny-1x1": (lambda: (np.ones((1, 1), dtype=np.uint64), 1), 1, 1),
    "tiny-5x7": (lambda: (f2gen.uniform(5, 7, 11), 7), 3, 2),
    "exact-64x64": (lambda: (f2gen.uniform(64, 64, 12), 64), 64, 40),
    "ragged-300x333": (lambda: (f2gen.uniform(300, 333, 13), 333), 17, 10),
    "tall-700x200": (lambda: (f2gen.uniform(700, 200, 14), 200), 64, 32),
    "wide-200x700": (lambda: (f2gen.uniform(200, 700, 15), 700), 64, 20),
    "square-1024": (lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024), 64, 64),
    "square-2048": (lambda: (f2gen.uniform(2048, 2048, 16), 2048), 33, 16),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_solve_matches_oracle(name):
    make, nrhs, ncons = CASES[name]
    A, m = make()
    check(A, m, nrhs, ncons, 900 + len(name))


@pytest.mark.parametrize("n,m,r", [(500, 600, 300), (640, 640, 576), (1000, 900, 899), (129, 130, 1)])
def test_solve_rank_deficient(n, m, r):
    X, Y = f2gen.fixed_rank_factors(n, m, r, 31 + r)
    A = oracle.mmm(X, Y, r, m)
    check(A, m, 64, 48, 5 + n)


def test_solve_sparse_low_rank():
    # two nonzeros per row: rank-deficient, many column blocks with few pivots
    A = f2gen.sparse_rows(1500, 1500, 2, 21)
    check(A, 1500, 64, 30, 8)


def test_solve_zero_matrix():
    n, m = 200, 150
    A = np.zeros((n, (m + 63) // 64), dtype=np.uint64)
    check(A, m, 64, 64, 3)  # only B = 0 is consistent: A*X0 = 0


def test_solve_identity_returns_rhs():
    n = 300
    A = np.zeros((n, (n + 63) // 64), dtype=np.uint64)
    for i in range(n):
        A[i, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    Bw = f2gen.uniform(n, 64, 44).reshape(-1)
    X, ok = gpu_solve(A, n, Bw, 64)
    assert ok == (1 << 64) - 1
    assert np.array_equal(X, Bw)


def test_solve_repeatable():
    A = f2gen.uniform(400, 450, 51)
    Bw = make_rhs(A, 400, 450, 64, 64, 52)
    X1, ok1 = gpu_solve(A, 450, Bw, 64)
    X2, ok2 = gpu_solve(A, 450, Bw, 64)
    assert ok1 == ok2 and np.array_equal(X1, X2)


def test_solve_padding_error():
    A = f2gen.uniform(100, 100, 61)
    Ad = gf2.Mat.from_rowmajor(A, 100)
    fac = gf2.decompose(Ad)
    Bw = np.zeros(100, dtype=np.uint64)
    Bw[7] = np.uint64(1) << np.uint64(20)  # bit 20 of a 5-column right-hand side
    B = gf2.Mat.from_rowmajor(Bw.reshape(-1, 1), 5)
    with pytest.raises(gf2.Gf2Error) as ei:
        gf2.solve(fac, B, 100)
    assert ei.value.status == 3  # GF2_ERR_PADDING


@pytest.mark.slow
def test_solve_8192_sampled():
    """A serving-size system: n = m = 8192, 64 right-hand sides.  The GPU
    solution is checked by A X = B on the consistent columns (all of them,
    B = A X0) and against the oracle's solve."""
    n = 8192
    A = f2gen.uniform(n, n, f2gen.BASE_SEED, 5)
    check(A, n, 64, 64, 99)
