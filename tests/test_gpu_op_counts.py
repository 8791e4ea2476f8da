"""The work the kernels do against the cost model (oracle/cost.py): the
op-counting build of the library (libgf2_count.so, compiled with
-DGF2_COUNT_OPS) counts word operations in its kernels; these tests compare
the counts with the exact counts of the method derived from the oracle's
factors, and those with the paper's formulas (Section 6: the Four Russians
product and Strassen's recursion; Section 7: the complexity estimate).

  - every (panel, row, word) triple of the trailing update is applied once:
    GF2_OP_UPDATES equals the count from the PLE factors, with and without
    the pair-of-panels update;
  - the rows taking y = d Z equal the rows below each panel's pivots;
  - lookups: b/c per updated word (8 for the c = 8 tables of the wide update,
    16 for the c = 4 tables of the look-ahead);
  - table entries: at least one set of b/c tables of 2^c - 1 entries per
    panel and trailing word (each CTA builds its own copy);
  - the product: n k m / (b c) lookups for dense A, the tables once per row
    block of the launch shape, and the Strassen level's additions.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import f2gen
import oracle
from tests.schedule_model import strassen_additions
from oracle import cost

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
B, C8, C4 = 64, 8, 4
ROWS_PER_CTA = (512, 1024, 1536, 3072)  # the product kernel's launch shapes: 256 U rows, U = 2, 4, 6, 12


@pytest.fixture(scope="module")
def counting_lib():
    from paper_1209_5198_gb300 import _build
    return _build.build(counting=True)


def decompose_cases():
    cases = [("tall 2048x1024", f2gen.uniform(2048, 1024, f2gen.BASE_SEED, 901), 2048, 1024),
             ("ragged 1000x777", f2gen.uniform(1000, 777, f2gen.BASE_SEED, 902), 1000, 777),
             ("wide 512x2048", f2gen.uniform(512, 2048, f2gen.BASE_SEED, 903), 512, 2048)]
    X, Y = f2gen.fixed_rank_factors(1024, 1024, 600, 904)
    cases.append(("rank 600 of 1024", oracle.mmm(X, Y, 600, 1024), 1024, 1024))
    return cases


def mmm_cases():
    A = f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 911)
    Bm = f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 912)
    A2 = f2gen.uniform(1000, 700, f2gen.BASE_SEED, 913)
    B2 = f2gen.uniform(700, 333, f2gen.BASE_SEED, 914)
    off = 1 << 62
    return [("1024^3 M4RM", A, Bm, 1024, 1024, 1024, 2, off),            # GF2_MMM_TABLES: no recursion
            ("1000x700x333 M4RM", A2, B2, 1000, 700, 333, 0, off),
            ("1024^3 one Strassen level", A, Bm, 1024, 1024, 1024, 0, 1024)]


def run_child(tmp_path, jobs, pairs: bool):
    arrays = {}
    for i, job in enumerate(jobs):
        arrays[f"kind_{i}"] = np.array(job[0])
        arrays[f"A_{i}"] = job[1]
        arrays[f"dims_{i}"] = np.array(job[3], dtype=np.int64)
        if job[2] is not None:
            arrays[f"B_{i}"] = job[2]
    jp = os.path.join(tmp_path, f"jobs_{int(pairs)}.npz")
    op = os.path.join(tmp_path, f"out_{int(pairs)}.json")
    np.savez(jp, **arrays)
    env = dict(os.environ, GF2_COUNT_OPS="1", GF2_PAIRS="1" if pairs else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "op_count_child.py"), jp, op],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.load(open(op))


@pytest.mark.parametrize("pairs", [True, False])
def test_decomposition_work_matches_the_model(counting_lib, tmp_path, pairs):
    cases = decompose_cases()
    res = run_child(tmp_path, [("decompose", A, None, (n, m)) for _, A, n, m in cases], pairs)
    for (name, A, n, m), got in zip(cases, res):
        ref = oracle.ple(A, m)
        r = ref["rank"]
        assert got["rank"] == r and got["pivcols"] == ref["pivcols"][:r].tolist(), name
        model = cost.block_counts(ref["L"], ref["pivcols"][:r], n, m, B)
        cnt = got["counts"]
        assert cnt["updates"] == model["updates"], (name, cnt, model)
        assert cnt["yrows"] == model["yrows"], (name, cnt, model)
        mu = (m + B - 1) // B
        # every panel with pivots builds b/c tables of 2^c - 1 entries for
        # each of its trailing words at least once (per CTA that needs them)
        table_sets = cnt["table8"] / ((B // C8) * (2 ** C8 - 1)) + cnt["table4"] / ((B // C4) * (2 ** C4 - 1))
        need = sum(mu - j - 1 for j in range(mu) if model["r"][j] > 0)
        assert table_sets >= need, (name, table_sets, need)
        assert cnt["mmm_lookups"] == cnt["mmm_table"] == cnt["mmm_adds"] == 0
        # b/c lookups per updated word, when every panel that updates has
        # more than 56 pivots (then both table sets are whole: 8 and 16)
        if all(rj > 56 for j, rj in enumerate(model["r"]) if rj and j < mu - 1):
            assert cnt["lookups8"] % (B // C8) == 0 and cnt["lookups4"] % (B // C4) == 0
            assert cnt["lookups8"] // (B // C8) + cnt["lookups4"] // (B // C4) == cnt["updates"], (name, cnt)
        if name.startswith("tall"):
            # full column rank, every row below a panel's pivots nonzero in
            # it: the paper's full-rank sums of Section 7
            fr = cost.full_rank_counts(n // B, m // B, B)
            assert r == m and model["updates"] == fr["updates"] and model["yrows"] == fr["yrows"]


def test_product_work_matches_the_model(counting_lib, tmp_path):
    cases = mmm_cases()
    res = run_child(tmp_path, [("mmm", A, Bm, (n, k, m, flags, cut)) for _, A, Bm, n, k, m, flags, cut in cases], True)
    for (name, A, Bm, n, k, m, flags, cut), got in zip(cases, res):
        Cref = oracle.mmm(A, Bm, k, m)
        assert np.array_equal(np.array(got["C"], dtype=np.uint64).reshape(Cref.shape), Cref), name
        cnt = got["counts"]
        mw, kw = (m + 63) // 64, (k + 63) // 64
        per_word = (B // C8) * (2 ** C8 - 1)
        if cut > n:
            # lookups: b/c per (row, word of C, slice of B) with a nonzero word of A
            assert cnt["mmm_lookups"] == np.count_nonzero(A) * mw * (B // C8), name
            # tables: once per slice and word column for each row block
            once = kw * mw * per_word
            assert cnt["mmm_table"] % once == 0 and cnt["mmm_table"] // once in {-(-n // rpc) for rpc in ROWS_PER_CTA}, name
            assert cnt["mmm_adds"] == 0
            if k % 64 == 0 and m % 64 == 0 and np.count_nonzero(A) == A.size:
                t, lk = cost.m4rm_product(n, k, m, B, C8)
                assert cnt["mmm_lookups"] == lk and cnt["mmm_table"] % t == 0
        else:
            # one level: the explicit additions of the schedule, and the seven
            # half-size products' lookups over their left operands
            assert cnt["mmm_adds"] == strassen_additions(n, k, m, B, 1), name
            n2, k2 = n // 2, (k // 64) // 2
            A11, A12, A21, A22 = A[:n2, :k2], A[:n2, k2:], A[n2:, :k2], A[n2:, k2:]
            S1 = A21 ^ A22
            S2 = S1 ^ A11
            S3 = A11 ^ A21
            S4 = A12 ^ S2
            lefts = (A11, A12, S2, S3, S1, S4, A22)
            assert cnt["mmm_lookups"] == sum(np.count_nonzero(L) for L in lefts) * (mw // 2) * (B // C8), name
