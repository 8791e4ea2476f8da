"""The Strassen-Winograd schedule of the product's recursion (seven
products, fifteen additions per level, run as an accumulate schedule over
F2: every product is either written into a temporary X or XORed into a
quadrant of C), checked on the CPU against the plain product over F2 for
random matrices, one and two levels deep, with and without accumulation.
The schedule below is the one the library's host recursion issues, step by
step (sub-products by the same recursion, the leaves by plain products)."""
import numpy as np


def f2(a):
    return a & 1


def rec(C, A, B, acc, levels, plant=None):
    """C (+)= A B over F2, in place, with `levels` Strassen-Winograd levels
    (`plant` names one step to get wrong, for the planted-mistake test)."""
    if levels == 0:
        P = f2(A.astype(np.int64) @ B.astype(np.int64)).astype(np.uint8)
        if acc:
            C ^= P
        else:
            C[:] = P
        return
    if not acc:
        C[:] = 0
    n2, k2, m2 = A.shape[0] // 2, A.shape[1] // 2, B.shape[1] // 2
    A11, A12, A21, A22 = A[:n2, :k2], A[:n2, k2:], A[n2:, :k2], A[n2:, k2:]
    B11, B12, B21, B22 = B[:k2, :m2], B[:k2, m2:], B[k2:, :m2], B[k2:, m2:]
    C11, C12, C21, C22 = C[:n2, :m2], C[:n2, m2:], C[n2:, :m2], C[n2:, m2:]
    S1 = A21 ^ A22
    S2 = S1 ^ A11
    S3 = A11 ^ A21
    S4 = A12 ^ S2
    T1 = B12 ^ B11
    T2 = B22 ^ T1
    T3 = B22 ^ B12
    T4 = T2 if plant == "T4" else T2 ^ B21
    X = np.zeros((n2, m2), dtype=np.uint8)
    rec(X, A11, B11, False, levels - 1)        # X = P1
    C11 ^= X
    rec(C11, A12, B21, True, levels - 1)       # C11 += P2
    rec(X, S2, T2, True, levels - 1)           # X = P1 + P6 (U2)
    C12 ^= X
    C21 ^= X
    C22 ^= X
    rec(X, S3, T3, False, levels - 1)          # X = P7
    C21 ^= X
    C22 ^= X
    rec(X, S1, T1, False, levels - 1)          # X = P5
    C12 ^= X
    if plant != "P5 into C22":
        C22 ^= X
    rec(C12, S4, B22, True, levels - 1)        # C12 += P3
    rec(C21, A22, T4, True, levels - 1)        # C21 += P4


def test_schedule_equals_the_product_over_f2():
    rng = np.random.default_rng(1209)
    for levels, (n, k, m) in ((1, (8, 6, 10)), (2, (16, 12, 8)), (2, (32, 32, 32)), (3, (24, 16, 40))):
        for acc in (False, True):
            A = rng.integers(0, 2, size=(n, k), dtype=np.uint8)
            B = rng.integers(0, 2, size=(k, m), dtype=np.uint8)
            C0 = rng.integers(0, 2, size=(n, m), dtype=np.uint8)
            want = f2(A.astype(np.int64) @ B.astype(np.int64)).astype(np.uint8)
            if acc:
                want ^= C0
            C = C0.copy()
            rec(C, A, B, acc, levels)
            assert np.array_equal(C, want), (levels, n, k, m, acc)


def test_a_planted_mistake_is_caught():
    """A dropped term (B21 in T4) or a dropped addition (P5 into C22) breaks
    the check: the test tells the right schedule from plausible wrong ones."""
    rng = np.random.default_rng(5198)
    A = rng.integers(0, 2, size=(16, 16), dtype=np.uint8)
    B = rng.integers(0, 2, size=(16, 16), dtype=np.uint8)
    want = f2(A.astype(np.int64) @ B.astype(np.int64)).astype(np.uint8)
    for plant in ("T4", "P5 into C22"):
        C = np.zeros((16, 16), dtype=np.uint8)
        rec(C, A, B, False, 1, plant=plant)
        assert not np.array_equal(C, want), plant
