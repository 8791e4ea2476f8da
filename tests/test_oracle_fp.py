"""Pins of the F_p oracle (oracle/fp.py) against what the mathematics fixes,
none of which re-runs the oracle's own elimination:
  * at p = 2 it equals the F2 oracle (f2_oracle.c, another implementation
    of the same pivot rule) factor for factor;
  * on every 2 x 2, 2 x 3, 3 x 2 and 3 x 3 matrix over F_3 (and a sample of
    3 x 4 over F_5) the rank is log_p of the size of the enumerated row
    space, and the pivot columns are the columns where the enumerated rank
    of the column prefix grows (the column rank profile);
  * P A = L E mod p, L unit lower trapezoidal, E row echelon with nonzero
    leading entries at the pivot columns, on large primes too;
  * products X Y of full-rank factors of rank r have rank r;
  * planted mistakes (a wrong inverse, the last qualifying row instead of the
    first, a dropped exchange of the stored multipliers, a dropped
    elimination) fail these pins."""
import itertools

import numpy as np
import pytest

import f2gen
import oracle
from oracle import fp


def span_size(rows: np.ndarray, p: int) -> int:
    """Number of distinct vectors in the row space, by enumerating every
    combination of the rows."""
    n, m = rows.shape
    seen = set()
    for coeffs in itertools.product(range(p), repeat=n):
        v = tuple((np.array(coeffs, dtype=np.int64) @ rows) % p) if n else (0,) * m
        seen.add(v)
    return len(seen)


def brute_rank(A: np.ndarray, p: int) -> int:
    s = span_size(A, p)
    r = 0
    while p ** r < s:
        r += 1
    assert p ** r == s
    return r


def matmul_p(A: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """A B mod p with Python integers (no overflow for any p)."""
    return (A.astype(object) @ B.astype(object)) % p


def check_factors(A, out, p):
    n, m = A.shape
    k = min(n, m)
    r = out["rank"]
    L, E, perm, piv = out["L"], out["E"], out["perm"], out["pivcols"]
    assert L.shape == (n, k) and E.shape == (k, m) and len(piv) == r
    assert sorted(perm.tolist()) == list(range(n))
    PA = A[perm] % p
    assert np.array_equal(matmul_p(L, E, p).astype(np.int64), PA)
    for t in range(r):
        assert L[t, t] == 1 and not L[t, t + 1:].any() and not L[:t, t].any()
        c = piv[t]
        assert E[t, c] != 0 and not E[t, :c].any()
        if t:
            assert piv[t] > piv[t - 1]
    assert not E[r:].any() and not L[:, r:].any()


def test_p2_equals_the_f2_oracle():
    for n, m, seed in ((64, 64, 1), (130, 70, 2), (70, 130, 3), (200, 200, 4)):
        words = f2gen.uniform(n, m, 900, seed)
        bits = f2gen.unpack_bits(words, m).astype(np.int64)
        ref = oracle.ple(words, m)
        got = fp.ple(bits, 2)
        r = ref["rank"]
        assert got["rank"] == r
        assert np.array_equal(got["perm"], ref["perm"])
        assert np.array_equal(got["pivcols"], ref["pivcols"][:r])
        assert np.array_equal(got["L"][:, :r], f2gen.unpack_bits(ref["L"], min(n, m))[:, :r])
        assert np.array_equal(got["E"][:r], f2gen.unpack_bits(ref["E"], m)[:r])


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_every_small_matrix_over_f3(shape):
    n, m = shape
    p = 3
    for entries in itertools.product(range(p), repeat=n * m):
        A = np.array(entries, dtype=np.int64).reshape(n, m)
        out = fp.ple(A, p)
        assert out["rank"] == brute_rank(A, p)
        prof = [c for c in range(m) if brute_rank(A[:, :c + 1], p) > (brute_rank(A[:, :c], p) if c else 0)]
        assert out["pivcols"].tolist() == prof
        check_factors(A, out, p)


def test_sample_over_f5():
    p = 5
    for seed in range(40):
        A = f2gen.fp_uniform(3, 4, p, 901, seed)
        if seed % 4 == 0:
            A[2] = (A[0] + 2 * A[1]) % p  # rank deficient
        out = fp.ple(A, p)
        assert out["rank"] == brute_rank(A, p)
        check_factors(A, out, p)


@pytest.mark.parametrize("p", [3, 7, 251, 65521, 1000003, 2147483647])
def test_invariants_and_fixed_rank(p):
    for n, m, r in ((40, 30, 30), (30, 40, 12), (60, 60, 59), (50, 50, 1)):
        X, Y = f2gen.fp_fixed_rank_factors(n, m, r, p, 902, n)
        A = matmul_p(X, Y, p).astype(np.int64)
        out = fp.ple(A, p)
        assert out["rank"] == r
        check_factors(A, out, p)
    A = f2gen.fp_uniform(45, 37, p, 903)
    check_factors(A, fp.ple(A, p), p)


def test_inverse():
    for p in (2, 3, 5, 65521, 2147483647):
        for b in (1, 2, p - 1, p // 2 + 1):
            if 0 < b < p:
                assert (fp.inverse(b, p) * b) % p == 1
    with pytest.raises(ZeroDivisionError):
        fp.inverse(0, 7)


PLANTED = {
    # a wrong inverse: beta itself
    "inverse": ("inv = inverse(beta, p)", "inv = beta % p"),
    # the last qualifying row instead of the first
    "last_row": ("i = t + int(rows[0])", "i = t + int(rows[-1])"),
    # the exchange forgets the multipliers already stored
    "no_L_exchange": ("L[[t, i], :t] = L[[i, t], :t]", "pass"),
    # a dropped elimination term: the pivot row's own entries
    "no_elimination": ("W[below, :] = (W[below, :] - (mult[:, None] * W[t, :][None, :]) % p) % p", "pass"),
}


def planted_module(kind):
    """A copy of oracle/fp.py with one mistake planted in its source."""
    src = open(fp.__file__).read()
    old, new = PLANTED[kind]
    assert src.count(old) == 1
    ns = {}
    exec(compile(src.replace(old, new), f"planted_{kind}", "exec"), ns)
    return ns


def pins_hold(ple) -> bool:
    try:
        for p, seed in ((7, 1), (2, 2), (65521, 3)):
            A = f2gen.fp_uniform(14, 12, p, 904, seed)
            check_factors(A, ple(A, p), p)
        words = f2gen.uniform(40, 40, 905)
        bits = f2gen.unpack_bits(words, 40).astype(np.int64)
        got, ref = ple(bits, 2), oracle.ple(words, 40)
        assert np.array_equal(got["perm"], ref["perm"])
        assert np.array_equal(got["E"][:ref["rank"]], f2gen.unpack_bits(ref["E"], 40)[:ref["rank"]])
        return True
    except AssertionError:
        return False


def test_pins_hold_for_the_oracle():
    assert pins_hold(fp.ple)


@pytest.mark.parametrize("kind", sorted(PLANTED))
def test_planted_mistakes_fail_the_pins(kind):
    assert not pins_hold(planted_module(kind)["ple"])
