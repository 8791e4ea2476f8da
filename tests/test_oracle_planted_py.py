"""The pins of the oracle's Python parts catch plausible mistakes: each case
plants one mistake (a dropped term, an off-by-one, a wrong operand) in a copy
of oracle/cost.py or of oracle.nullspace, loads the copy, and checks that
the pins of tests/test_cost_model.py and tests/test_oracle_nullspace.py
reject it.  The committed oracle is never modified."""
import inspect
import itertools
import os
import types
from fractions import Fraction

import numpy as np
import pytest

import f2gen
import oracle
from oracle import cost
from tests import test_cost_model as cm

COST_SRC = open(cost.__file__).read()

COST_MUTATIONS = {
    "counts-include-own-pivots": ("below = Lb[R + rj:, R:R + rj]", "below = Lb[R:, R:R + rj]"),
    "updates-include-own-block": ("updates += nz * (mu - j - 1)", "updates += nz * (mu - j)"),
    "yrows-include-pivots": ("yrows += n - R - rj", "yrows += n - R"),
    "cost-full-extra-row-block": ("(2 ** c - 1 + (N - k) * b)", "(2 ** c - 1 + (N - k + 1) * b)"),
    "cost-rank1-table-off-by-one": ("(2 ** c - 1 + N * b)", "(2 ** c + N * b)"),
    "strassen-additions-doubled": ("Fraction(11 * n * n, 2 * b) + 7 * m4rm_square", "Fraction(11 * n * n, b) + 7 * m4rm_square"),
    "m4rm-square-table-off-by-one": ("n * n * (2 ** c - 1) + n ** 3", "n * n * (2 ** c) + n ** 3"),
    "table-size-wrong-rows": ("(b / c) * (2.0 ** c - 1.0 + b)", "(b / c) * (2.0 ** c - 1.0 + 2 * b)"),
    "product-table-off-by-one": ("return per * (2 ** c - 1), per * n", "return per * (2 ** c), per * n"),
    "full-rank-counts-extra-word": ("\"updates\": sum((M - k) * (N - k) * b", "\"updates\": sum((M - k + 1) * (N - k) * b"),
}


def load_cost(src):
    mod = types.ModuleType("cost_planted")
    exec(compile(src, "cost_planted", "exec"), mod.__dict__)
    return mod


def cost_pins_pass(m) -> bool:
    try:
        # the printed table-size minima
        for b, printed in cm.golden_minima():
            digits = len(printed.split(".")[1]) if "." in printed else 0
            assert abs(m.best_table_size(b) - float(printed)) <= 0.5 * 10 ** -digits + 1e-9
        # tables + lookups of the product, and the n k m / (b c) lookups
        for b, c, n, k, mm in ((64, 8, 1024, 1024, 1024), (32, 4, 96, 64, 96)):
            t, lk = m.m4rm_product(n, k, mm, b, c)
            assert Fraction(t + lk) == m.m4rm_cost(b, c, n) * (k // b) * (mm // b)
            assert lk == n * k * mm // (b * c)
        assert m.m4rm_product(1024, 1024, 1024, 64, 8) == (16 * 16 * 8 * 255, 1024 ** 3 // 512)
        # the crossover follows from the cost formulas
        for b in (32, 64):
            for c in (2, 4, 8):
                x = m.strassen_crossover(b, c)
                for nn in range(2, 2 * x + 2, 2):
                    assert (m.strassen_one_level(nn, b, c) <= m.m4rm_square(nn, b, c)) == (nn >= x)
        # closed forms of the decomposition sums
        for b, c in ((64, 8), (32, 4)):
            for M in (1, 3, 7):
                for N in (M, M + 2):
                    s1 = Fraction(M * (M + 1), 2)
                    s2 = Fraction(M * (M + 1) * (2 * M + 1), 6)
                    assert m.cost_full(N, M, b, c) == Fraction(b, c) * ((2 ** c - 1) * s1 + b * ((N - M - 1) * s1 + s2))
                    assert m.cost_rank1(N, M, b, c) == Fraction(b, c) * (2 ** c - 1 + N * b) * s1
                    fr = m.full_rank_counts(N, M, b)
                    tables = sum((M - k + 1) * (2 ** c - 1) for k in range(1, M + 1))
                    assert m.cost_full(N, M, b, c) == Fraction(b, c) * (fr["yrows"] + fr["updates"] + tables)
        # the per-block counts against brute force
        for seed, (n, mm) in enumerate(((40, 40), (70, 33), (33, 70))):
            A = f2gen.uniform(n, mm, f2gen.BASE_SEED, 300 + seed)
            ref = oracle.ple(A, mm)
            for b in (8, 16):
                got = m.block_counts(ref["L"], ref["pivcols"][:ref["rank"]], n, mm, b)
                assert got == cm.brute_block_counts(cm.as_ints(A), n, mm, b)
        return True
    except AssertionError:
        return False


def test_committed_cost_model_passes_its_pins():
    assert cost_pins_pass(cost)


@pytest.mark.parametrize("name", sorted(COST_MUTATIONS))
def test_planted_cost_mistake_is_caught(name):
    old, new = COST_MUTATIONS[name]
    assert COST_SRC.count(old) == 1, f"mutation anchor for {name} not found once"
    assert not cost_pins_pass(load_cost(COST_SRC.replace(old, new)))


NULL_SRC = inspect.getsource(oracle.nullspace)
NULL_MUTATIONS = {
    "identity-dropped": ("Nb[free, np.arange(nul)] = True", "Nb[free, np.arange(nul)] = False"),
    "pivot-rows-reversed": ("Nb[piv, :] = Rb[:, free]", "Nb[piv[::-1], :] = Rb[:, free]"),
    "pivot-rows-missing": ("Nb[piv, :] = Rb[:, free]", "pass"),
    "nullity-off-by-one": ("nul = m - r\n", "nul = max(m - r - 1, 0)\n"),
}


def load_nullspace(src):
    ns = dict(oracle.__dict__)
    exec(compile(src, "nullspace_planted", "exec"), ns)
    return ns["nullspace"]


def nullspace_pins_pass(f) -> bool:
    try:
        for seed in range(25):
            rng = np.random.default_rng(seed)
            n, m = int(rng.integers(1, 6)), int(rng.integers(2, 9))
            Ab = rng.random((n, m)) < 0.5
            res = f(oracle._pack(Ab), m)
            nul = res["nul"]
            Nb = oracle._unpack(res["N"], nul).astype(np.int64) if nul else np.zeros((m, 0), dtype=np.int64)
            sols = {x for x in itertools.product((0, 1), repeat=m) if not ((Ab.astype(np.int64) @ np.array(x)) % 2).any()}
            assert len(sols) == 2 ** nul
            span = {tuple(((Nb @ np.array(co, dtype=np.int64)) % 2).tolist()) for co in itertools.product((0, 1), repeat=nul)}
            assert span == sols
        return True
    except (AssertionError, IndexError, ValueError):
        return False


def test_committed_nullspace_passes_its_pins():
    assert nullspace_pins_pass(oracle.nullspace)


@pytest.mark.parametrize("name", sorted(NULL_MUTATIONS))
def test_planted_nullspace_mistake_is_caught(name):
    old, new = NULL_MUTATIONS[name]
    assert NULL_SRC.count(old) == 1, f"mutation anchor for {name} not found once"
    assert not nullspace_pins_pass(load_nullspace(NULL_SRC.replace(old, new)))
