"""Operation counts of the method: the paper's cost formulas and the exact
counts of the blocked decomposition and of the Four Russians product.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the op-counting tests
compare these numbers with the counters of the library's op-counting build
(gf2_op_counts).  Nothing here is called by the library.

Units: operations on b-bit words (the paper's Xor_b; the library has b = 64),
table size c bits.  Everything is exact integer (or Fraction) arithmetic.

Formulas (Section 6, the Four Russians product and Strassen's recursion;
Section 7, the complexity estimate):
  C(b, c, n)  = (b/c)(2^c - 1 + n): the M4RM product of an n x b matrix by a
                b x b matrix -- b/c tables of 2^c - 1 entries, one XOR each,
                then b/c lookups for each of the n rows;
  M(n)        = (n^2 (2^c - 1) + n^3) / (b c): the M4RM product of two n x n
                matrices;
  S(n)        = 11 n^2 / (2b) + 7 S(n/2): Strassen's recursion with the
                paper's 22 additions of n/2 x n/2 matrices per level;
  cost_full   = sum_{k=1..M} (b/c)(M-k+1)(2^c - 1 + (N-k) b), n = bN, m = bM:
                the M4RM work of the decomposition of a full-rank n x m
                matrix, n >= m, leading term n^3 / (3 b c) for n = m;
  cost_1      = sum_{k=1..M} (b/c)(M-k+1)(2^c - 1 + N b): rank 1, leading
                term n^3 / (2 b c).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def m4rm_cost(b: int, c: int, n) -> Fraction:
    """C(b, c, n) = (b/c)(2^c - 1 + n) (Section 6)."""
    return Fraction(b, c) * (2 ** c - 1 + n)


def best_table_size(b: int, lo: float = 1.0, hi: float = 16.0) -> float:
    """The real c in [lo, hi] minimising C(b, c, b) (Section 6, the remark on
    the choice of c): golden-section search on the continuous function, which
    is unimodal there."""
    f = lambda c: (b / c) * (2.0 ** c - 1.0 + b)  # noqa: E731
    g = (5 ** 0.5 - 1) / 2
    a, d = lo, hi
    x1, x2 = d - g * (d - a), a + g * (d - a)
    for _ in range(200):
        if f(x1) < f(x2):
            d, x2 = x2, x1
            x1 = d - g * (d - a)
        else:
            a, x1 = x1, x2
            x2 = a + g * (d - a)
    return (a + d) / 2


def m4rm_square(n: int, b: int, c: int) -> Fraction:
    """M(n) = (n^2 (2^c - 1) + n^3) / (b c) (Section 6)."""
    return Fraction(n * n * (2 ** c - 1) + n ** 3, b * c)


def strassen_one_level(n: int, b: int, c: int) -> Fraction:
    """One level of Strassen's recursion over M4RM: 11 n^2 / (2b) + 7 M(n/2)
    (Section 6; n even)."""
    return Fraction(11 * n * n, 2 * b) + 7 * m4rm_square(Fraction(n, 2), b, c)


def strassen_crossover(b: int, c: int) -> int:
    """44 c + 6 (2^c - 1): from this n on one level of Strassen costs no more
    than M4RM (Section 6; independent of b)."""
    return 44 * c + 6 * (2 ** c - 1)


def strassen_cost(n: int, b: int, c: int, cutoff: int) -> Fraction:
    """S(n) = 11 n^2 / (2b) + 7 S(n/2) while n >= cutoff (and n even), M(n) below."""
    if n < cutoff or n % 2:
        return m4rm_square(n, b, c)
    return Fraction(11 * n * n, 2 * b) + 7 * strassen_cost(n // 2, b, c, cutoff)


def cost_full(N: int, M: int, b: int, c: int) -> Fraction:
    """The paper's M4RM cost of the full-rank decomposition, N >= M blocks of b (Section 7)."""
    return sum((Fraction(b, c) * (M - k + 1) * (2 ** c - 1 + (N - k) * b) for k in range(1, M + 1)), Fraction(0))


def cost_rank1(N: int, M: int, b: int, c: int) -> Fraction:
    """The paper's M4RM cost when rank(A) = 1 (Section 7)."""
    return sum((Fraction(b, c) * (M - k + 1) * (2 ** c - 1 + N * b) for k in range(1, M + 1)), Fraction(0))


def m4rm_product(n: int, k: int, m: int, b: int, c: int) -> tuple[int, int]:
    """(table entries, lookups) of the M4RM product of an n x k by a k x m
    matrix, k and m multiples of b, c | b: for each slice of b rows of B and
    each word column, b/c tables of 2^c - 1 entries, and b/c lookups for each
    of the n rows -- the rectangular form (m/c)(2^c - 1 + n) per slice
    (Section 7) summed over the k/b slices."""
    assert k % b == 0 and m % b == 0 and b % c == 0
    per = (k // b) * (m // b) * (b // c)
    return per * (2 ** c - 1), per * n


def _bits(words: np.ndarray, ncols: int) -> np.ndarray:
    """Row-major uint64 words (rows, ceil(ncols/64)) -> bool matrix (rows, ncols)."""
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    rows = words.shape[0]
    if ncols == 0:
        return np.zeros((rows, 0), dtype=bool)
    by = words.view(np.uint8).reshape(rows, -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :ncols].astype(bool)


def block_counts(L: np.ndarray, pivcols: np.ndarray, n: int, m: int, b: int = 64) -> dict:
    """Exact work of the blocked decomposition (b-column blocks) from its PLE
    factors P A = L E (the oracle's ``ple``), per block j with r_j pivots
    starting at pivot R_j:
      yrows   = sum over blocks with r_j > 0 of n - R_j - r_j: the rows below
                the block's pivots, whose multipliers y = d Z are formed
                (Y = D Z, Section 4);
      nzrows  = those rows whose multiplier is nonzero: their L entries in the
                block's pivot columns are not all zero (y = 0 exactly when the
                row's word d in block j is 0, and L holds d's coordinates);
      updates = sum_j nzrows_j (mu - j - 1): (panel, row, word) triples of the
                trailing update A(j+1) = E + Y C (eq. (Aj) of Section 4) on
                the mu - j - 1 words after block j.
    Also the per-block lists r and nzrows."""
    mu = (m + b - 1) // b
    piv = np.asarray(pivcols, dtype=np.int64)
    r = int(piv.size)
    Lb = _bits(L, r)
    R = 0
    yrows = updates = 0
    rs, nzs = [], []
    for j in range(mu):
        rj = int(np.count_nonzero((piv >= b * j) & (piv < b * (j + 1))))
        below = Lb[R + rj:, R:R + rj]
        nz = int(np.count_nonzero(below.any(axis=1))) if rj else 0
        if rj:
            yrows += n - R - rj
        updates += nz * (mu - j - 1)
        rs.append(rj)
        nzs.append(nz)
        R += rj
    return {"yrows": yrows, "updates": updates, "r": rs, "nzrows": nzs}


def full_rank_counts(N: int, M: int, b: int) -> dict:
    """block_counts of a full-rank n x m matrix, n = bN >= m = bM, whose rows
    below each block's pivots all have nonzero multipliers: the (N-k) b rows
    below block k take y (Y = D Z) and update the M - k words after it.  With
    the tables, the paper's cost_full is (b/c) [yrows + updates + sum_k
    (M-k+1)(2^c - 1)]."""
    return {"yrows": sum((N - k) * b for k in range(1, M + 1)),
            "updates": sum((M - k) * (N - k) * b for k in range(1, M + 1))}
