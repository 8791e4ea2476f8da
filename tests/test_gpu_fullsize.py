"""Parity at the benchmark's full sizes (n = m = 32768, the 65536 and
rectangular scale configurations, the fixed-rank products), in the launch
configuration the benchmark times.

Every decomposition here is compared element by element with a COMPLETE run
of the oracle on the same input: rank, pivot columns, perm, L and E.  The
factors are unique given the pivot rule (Lemma 4.1 and Section 4), so any
difference is an error.  (The oracle's multithreaded elimination takes a few
seconds at 32768 and under a minute at 65536 on the host cores.)  On top:
  * P*A = L*E by Freivalds' test with 64 random vectors packed one word per
    row (a wrong factor passes with probability at most 2^-64);
  * the unit lower-triangular / row-echelon invariants of every row;
  * the exact rank of products X*Y of known rank r (built on the CPU);
  * solves and products checked against the definition A X = B, C = A B.
Every input is built on the CPU from the seeded generators."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402

N = 32768
NTHREADS = oracle.max_threads()


def matvec_parity(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Bits of M x over F2 (M row-major words, x packed words) as a 0/1 array."""
    acc = np.zeros(M.shape[0], dtype=np.uint64)
    for q in range(M.shape[1]):  # column by column keeps the temporaries small
        acc += np.bitwise_count(M[:, q] & x[q]).astype(np.uint64)
    return (acc & np.uint64(1)).astype(np.uint8)


def pack(bits: np.ndarray, words: int) -> np.ndarray:
    out = f2gen.pack_bits(bits.reshape(1, -1)).reshape(-1)
    if out.size < words:
        out = np.concatenate([out, np.zeros(words - out.size, dtype=np.uint64)])
    return out[:words]


def freivalds64(A, perm, L, E, m, seed):
    """P A X == L (E X) for a random m x 64 bit matrix X (64 vectors, one
    word per row): a wrong factor passes with probability at most 2^-64."""
    X = f2gen.uniform(m, 64, seed, 64)
    kmax = E.shape[0]
    AX = oracle.mmm(A, X, m, 64, nthreads=NTHREADS)[perm]
    EX = oracle.mmm(E, X, m, 64, nthreads=NTHREADS)
    LEX = oracle.mmm(L, EX, kmax, 64, nthreads=NTHREADS)
    assert np.array_equal(AX, LEX), "P*A*X != L*(E*X)"


def matches_full_oracle(A, m, perm, piv, r, L, E):
    """The oracle's complete decomposition of the same input, element by
    element."""
    ref = oracle.ple(A, m, want_L=True, want_E=True, nthreads=NTHREADS)
    assert r == ref["rank"]
    assert np.array_equal(piv[:r], ref["pivcols"])
    assert (piv[r:] == -1).all()
    assert np.array_equal(perm, ref["perm"]), "perm differs"
    assert np.array_equal(L, ref["L"]), "L differs"
    assert np.array_equal(E, ref["E"]), "E differs"
    return ref


def check_shapes(perm, piv, r, L, E, n, m):
    """perm a permutation; pivcols increasing; E row echelon with its leading
    ones at pivcols and zero rows from r on; L unit lower trapezoidal with
    zero columns from r on."""
    assert np.array_equal(np.sort(perm), np.arange(n)), "perm is not a permutation"
    p = piv[:r].astype(np.int64)
    assert (np.diff(p) > 0).all() and (p >= 0).all() and (p < m).all()
    assert (piv[r:] == -1).all()
    rows = np.arange(r)
    word, bit = p // 64, (p % 64).astype(np.uint64)
    assert ((E[rows, word] >> bit) & np.uint64(1) == 1).all()
    assert not (E[rows, word] & ((np.uint64(1) << bit) - np.uint64(1))).any()
    for q in range(E.shape[1]):  # words before the leading word are zero
        assert not E[:r][word > q, q].any()
    assert not E[r:].any()
    t = np.arange(r)
    tw, tb = t // 64, (t % 64).astype(np.uint64)
    assert ((L[t, tw] >> tb) & np.uint64(1) == 1).all()
    above = ~((np.uint64(2) << tb) - np.uint64(1))
    assert not (L[t, tw] & above).any()
    for q in range(L.shape[1]):  # words after the diagonal word are zero
        assert not L[:r][tw < q, q].any()
    # columns >= r
    if r < L.shape[1] * 64:
        q0 = r // 64
        if r % 64:
            assert not (L[:, q0] & ~((np.uint64(1) << np.uint64(r % 64)) - np.uint64(1))).any()
            q0 += 1
        assert not L[:, q0:].any()


def gpu_factors(A_rm, m):
    n = A_rm.shape[0]
    A = gf2.Mat.from_rowmajor(A_rm, m)
    out = gf2.decompose(A, factors=True)
    torch.cuda.synchronize()
    r = int(out["rank"].item())
    return (out["perm"].cpu().numpy(), out["pivcols"].cpu().numpy(), r,
            out["L"].to_rowmajor(), out["E"].to_rowmajor(), out)


def test_full_size_decomposition_32768():
    A = f2gen.uniform(N, N, f2gen.BASE_SEED, 1, 0)  # the benchmark's input
    perm, piv, r, L, E, _ = gpu_factors(A, N)
    assert r >= N - 8  # a Bernoulli(1/2) square matrix has rank n - O(1)
    check_shapes(perm, piv, r, L, E, N, N)
    matches_full_oracle(A, N, perm, piv, r, L, E)
    freivalds64(A, perm, L, E, N, 77)


@pytest.mark.parametrize("n,m", [(65536, 65536), (16384, 65536), (65536, 16384)])
def test_full_size_scale_configurations(n, m):
    """The largest square and the two rectangular scale configurations."""
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 2, n // 1024 + m // 1024)
    perm, piv, r, L, E, _ = gpu_factors(A, m)
    assert r >= min(n, m) - 8 if n == m else r == min(n, m)
    check_shapes(perm, piv, r, L, E, n, m)
    matches_full_oracle(A, m, perm, piv, r, L, E)
    freivalds64(A, perm, L, E, m, 83)


@pytest.mark.parametrize("n,r", [(16384, 8192), (16384, 16384 - 64), (32768, 16384), (32768, 32768 - 64)])
def test_full_size_fixed_rank(n, r):
    """Fixed-rank products X*Y (the scale configuration's r = n/2 and n - 64):
    the known rank and the complete oracle decomposition."""
    X, Y = f2gen.fixed_rank_factors(n, n, r, 500 + r)
    A = oracle.mmm(X, Y, r, n, nthreads=NTHREADS)
    perm, piv, rk, L, E, _ = gpu_factors(A, n)
    assert rk == r
    check_shapes(perm, piv, rk, L, E, n, n)
    matches_full_oracle(A, n, perm, piv, rk, L, E)
    freivalds64(A, perm, L, E, n, 78)


def test_full_size_solve_32768():
    A = f2gen.uniform(N, N, f2gen.BASE_SEED, 1, 0)
    nrhs = 8
    X0 = f2gen.rhs_from_solution(nrhs, N, 79)
    # B = A X0 on the CPU, one right-hand side at a time
    B = np.zeros(N, dtype=np.uint64)
    for cidx in range(nrhs):
        xc = pack(((X0[:, 0] >> np.uint64(cidx)) & np.uint64(1)).astype(np.uint8), A.shape[1])
        B |= matvec_parity(A, xc).astype(np.uint64) << np.uint64(cidx)
    Ad = gf2.Mat.from_rowmajor(A, N)
    fac = gf2.decompose(Ad, factors=True)
    Bd = gf2.Mat.from_rowmajor(B.reshape(-1, 1), nrhs)
    out = gf2.solve(fac, Bd, N)
    assert out["consistent"] == (1 << nrhs) - 1
    X = out["X"].to_rowmajor().reshape(-1)
    for cidx in range(nrhs):
        xc = pack(((X >> np.uint64(cidx)) & np.uint64(1)).astype(np.uint8), A.shape[1])
        bc = ((B >> np.uint64(cidx)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(matvec_parity(A, xc), bc)


@pytest.mark.parametrize("strassen", [False, True])
def test_full_size_product_16384(strassen):
    """C = A B at 16384 against the oracle's product, element by element,
    with M4RM alone and with two Strassen-Winograd levels (cutoff 8192 ->
    4096)."""
    n = 16384
    Ah = f2gen.uniform(n, n, 80)
    Bh = f2gen.uniform(n, n, 81)
    old = gf2.strassen_cutoff()
    try:
        gf2.set_strassen_cutoff(8192 if strassen else gf2.STRASSEN_OFF)
        C = gf2.mmm(gf2.Mat.from_rowmajor(Ah, n), gf2.Mat.from_rowmajor(Bh, n)).to_rowmajor()
    finally:
        gf2.set_strassen_cutoff(old)
    assert np.array_equal(C, oracle.mmm(Ah, Bh, n, n, nthreads=NTHREADS))
