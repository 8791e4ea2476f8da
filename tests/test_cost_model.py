"""Pins of oracle/cost.py, the operation counts of the method (Section 6:
the Four Russians product and Strassen's recursion; Section 7: the
complexity estimate of the decomposition).  CPU only.

What pins what:
  - the table-size minima the paper prints (tests/golden/m4rm_table_size.txt);
  - the Strassen crossover 44c + 6(2^c - 1), derived from the two cost
    formulas, checked against them with exact arithmetic for every even n;
  - closed forms of the decomposition sums (the substitution i = M - k + 1
    and sums of powers) and their leading terms n^3/(3bc), n^3/(2bc);
  - the exact per-block counts from the PLE factors against a brute-force
    block elimination written here with Python integers.
"""
from __future__ import annotations

import os
import random
from fractions import Fraction

import numpy as np
import pytest

import f2gen
import oracle
from oracle import cost

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "m4rm_table_size.txt")


def golden_minima():
    out = []
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            out.append((int(line[0]), line[1]))
    return out


@pytest.mark.parametrize("b,printed", golden_minima())
def test_best_table_size_matches_the_printed_minima(b, printed):
    digits = len(printed.split(".")[1]) if "." in printed else 0
    assert abs(cost.best_table_size(b) - float(printed)) <= 0.5 * 10 ** -digits + 1e-9


def test_m4rm_cost_is_tables_plus_lookups():
    # C(b, c, n) per slice and word column = b/c tables of 2^c - 1 entries + (b/c) n lookups
    for b, c, n, k, m in ((64, 8, 1024, 1024, 1024), (64, 4, 300, 640, 128), (32, 4, 96, 64, 96)):
        tables, lookups = cost.m4rm_product(n, k, m, b, c)
        assert Fraction(tables + lookups) == cost.m4rm_cost(b, c, n) * (k // b) * (m // b)
        assert lookups == n * k * m // (b * c)
    assert cost.m4rm_product(1024, 1024, 1024, 64, 8) == (16 * 16 * 8 * 255, 1024 ** 3 // 512)


@pytest.mark.parametrize("b", [32, 64, 128])
def test_strassen_crossover_follows_from_the_costs(b):
    for c in range(1, 11):
        x = cost.strassen_crossover(b, c)
        assert x % 2 == 0
        for n in range(2, 3 * x + 2, 2):
            cheaper = cost.strassen_one_level(n, b, c) <= cost.m4rm_square(n, b, c)
            assert cheaper == (n >= x), (b, c, n, x)
        # equality exactly at the crossover
        assert cost.strassen_one_level(x, b, c) == cost.m4rm_square(x, b, c)


def test_strassen_recursion():
    b, c = 64, 8
    n = 4096
    one = cost.strassen_cost(n, b, c, n)  # one level: cutoff n
    assert one == Fraction(11 * n * n, 2 * b) + 7 * cost.m4rm_square(n // 2, b, c)
    two = cost.strassen_cost(n, b, c, n // 2)
    assert two == Fraction(11 * n * n, 2 * b) + 7 * (Fraction(11 * (n // 2) ** 2, 2 * b) + 7 * cost.m4rm_square(n // 4, b, c))
    assert cost.strassen_cost(n, b, c, 2 * n) == cost.m4rm_square(n, b, c)


def test_strassen_additions_of_this_schedule():
    """The test-side model of the library's schedule (not the oracle's):
    16 explicit additions of half-size matrices per level, 4 more fused."""
    from tests.schedule_model import strassen_additions
    b = 64
    n = 1024
    one = strassen_additions(n, n, n, b, 1)
    h = (n // 2) * (n // 2) // b  # words of one n/2 x n/2 matrix
    assert one == 16 * h
    # 16 explicit + 4 fused accumulations = 20 additions, fewer than the paper's 22
    assert one + 4 * h == 20 * h and 20 * h < Fraction(11 * n * n, 2 * b)
    assert strassen_additions(n, n, n, b, 2) == 16 * h + 7 * 16 * (h // 4)
    # rectangular: A halves n/2 x k/2, B halves k/2 x m/2, C halves n/2 x m/2
    assert strassen_additions(256, 512, 1024, b, 1) == 4 * 128 * 4 + 4 * 256 * 8 + 8 * 128 * 8


@pytest.mark.parametrize("b,c", [(64, 8), (32, 4), (64, 4), (128, 6)])
def test_cost_full_closed_form(b, c):
    for M in (1, 2, 3, 7, 16, 33):
        for N in (M, M + 1, 2 * M + 5):
            # i = M - k + 1 runs 1..M and N - k = N - M - 1 + i
            s1 = Fraction(M * (M + 1), 2)
            s2 = Fraction(M * (M + 1) * (2 * M + 1), 6)
            closed = Fraction(b, c) * ((2 ** c - 1) * s1 + b * ((N - M - 1) * s1 + s2))
            assert cost.cost_full(N, M, b, c) == closed
            assert cost.cost_rank1(N, M, b, c) == Fraction(b, c) * (2 ** c - 1 + N * b) * s1


def test_leading_terms():
    b, c = 64, 8
    prev_full = prev_1 = None
    for M in (64, 256, 1024):
        n = b * M
        full = cost.cost_full(M, M, b, c) * 3 * b * c / Fraction(n) ** 3
        one = cost.cost_rank1(M, M, b, c) * 2 * b * c / Fraction(n) ** 3
        # exact: cost_full = n^3/(3bc) - n b/(3c) + (2^c - 1) M (M + 1) b / (2c)
        assert cost.cost_full(M, M, b, c) == Fraction(n ** 3, 3 * b * c) - Fraction(n * b, 3 * c) + Fraction((2 ** c - 1) * M * (M + 1) * b, 2 * c)
        if prev_full is not None:
            assert abs(full - 1) < abs(prev_full - 1) and abs(one - 1) < abs(prev_1 - 1)
        prev_full, prev_1 = full, one
    assert abs(float(full) - 1) < 0.02 and abs(float(one) - 1) < 0.02


@pytest.mark.parametrize("b,c", [(64, 8), (64, 4), (32, 4)])
def test_full_rank_counts_split_the_paper_cost(b, c):
    # cost_full = (b/c) [rows taking y + trailing word updates + table entries]
    for M in (1, 4, 9):
        for N in (M, M + 3):
            fr = cost.full_rank_counts(N, M, b)
            tables = sum((M - k + 1) * (2 ** c - 1) for k in range(1, M + 1))
            assert cost.cost_full(N, M, b, c) == Fraction(b, c) * (fr["yrows"] + fr["updates"] + tables)


def brute_block_counts(A_rows: list[int], n: int, m: int, b: int) -> dict:
    """Plain bit-level elimination with the first-row pivot rule, rows as
    Python integers (bit t = column t), counting per block of b columns the
    rows below its pivots and those whose word in the block was nonzero when
    the block started."""
    rows = list(enumerate(A_rows))  # (identity, bits) in current order
    mu = (m + b - 1) // b
    t = 0
    yrows = updates = 0
    rs, nzs = [], []
    for j in range(mu):
        d = {ident: (v >> (b * j)) & ((1 << b) - 1) for ident, v in rows[t:]}
        t0 = t
        for col in range(b * j, min(b * (j + 1), m)):
            i = next((i for i in range(t, n) if (rows[i][1] >> col) & 1), None)
            if i is None:
                continue
            rows[t], rows[i] = rows[i], rows[t]
            pv = rows[t][1]
            for i2 in range(t + 1, n):
                if (rows[i2][1] >> col) & 1:
                    rows[i2] = (rows[i2][0], rows[i2][1] ^ pv)
            t += 1
        rj = t - t0
        nz = sum(1 for ident, _ in rows[t:] if d[ident]) if rj else 0
        if rj:
            yrows += n - t
        updates += nz * (mu - j - 1)
        rs.append(rj)
        nzs.append(nz)
    return {"yrows": yrows, "updates": updates, "r": rs, "nzrows": nzs}


def as_ints(A: np.ndarray) -> list[int]:
    return [sum(int(w) << (64 * q) for q, w in enumerate(row)) for row in A]


@pytest.mark.parametrize("b", [8, 16, 64])
def test_block_counts_against_brute_force(b):
    rnd = random.Random(5198)
    cases = []
    for seed, (n, m) in enumerate(((40, 40), (70, 33), (33, 70), (97, 130), (64, 64), (1, 9))):
        cases.append((f2gen.uniform(n, m, f2gen.BASE_SEED, 300 + seed), n, m))
    # rank-deficient products and a sparse matrix
    for seed, (n, m, r) in enumerate(((60, 50, 13), (90, 120, 40), (128, 128, 70))):
        X, Y = f2gen.fixed_rank_factors(n, m, r, 400 + seed)
        cases.append((oracle.mmm(X, Y, r, m), n, m))
    sp = np.zeros((50, 1), dtype=np.uint64)
    for i in range(50):
        if rnd.random() < 0.5:
            sp[i, 0] = np.uint64(1) << np.uint64(rnd.randrange(40))
    cases.append((sp, 50, 40))
    for A, n, m in cases:
        ref = oracle.ple(A, m)
        got = cost.block_counts(ref["L"], ref["pivcols"][:ref["rank"]], n, m, b)
        want = brute_block_counts(as_ints(A), n, m, b)
        assert got == want, (n, m, b)


def test_block_counts_full_rank_tall_matches_paper_sum():
    # a tall Bernoulli(1/2) matrix has full column rank and every row below a
    # block's pivots a nonzero word in it, with overwhelming probability; the
    # counts are then the paper's full-rank sums
    n, m, b = 512, 256, 64
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 77)
    ref = oracle.ple(A, m)
    assert ref["rank"] == m
    got = cost.block_counts(ref["L"], ref["pivcols"][:ref["rank"]], n, m, b)
    fr = cost.full_rank_counts(n // b, m // b, b)
    assert got["yrows"] == fr["yrows"] and got["updates"] == fr["updates"]
