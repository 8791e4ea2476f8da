"""Pins of oracle.nullspace (the basis of {x : A x = 0} read off the reduced
row echelon form): on tiny matrices, brute force over every x in F2^m -- the
solution set has 2^(m - r) elements and is exactly the span of the basis;
on larger ones, A N = 0 by numpy integer products and the identity block at
the free columns (so the columns are independent and there are m - r of
them)."""
import itertools

import numpy as np
import pytest

import f2gen
import oracle


def bits(words, cols):
    return oracle._unpack(words, cols).astype(np.int64)


@pytest.mark.parametrize("seed", range(40))
def test_nullspace_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 7)), int(rng.integers(1, 10))
    density = rng.choice([0.2, 0.5, 0.8])
    Ab = rng.random((n, m)) < density
    A = oracle._pack(Ab)
    res = oracle.nullspace(A, m)
    Nb = bits(res["N"], res["nul"]) if res["nul"] else np.zeros((m, 0), dtype=np.int64)
    sols = {x for x in itertools.product((0, 1), repeat=m) if not ((Ab.astype(np.int64) @ np.array(x)) % 2).any()}
    assert len(sols) == 2 ** res["nul"]
    span = set()
    for coef in itertools.product((0, 1), repeat=res["nul"]):
        span.add(tuple(((Nb @ np.array(coef, dtype=np.int64)) % 2).tolist()) if res["nul"] else tuple([0] * m))
    assert span == sols


@pytest.mark.parametrize("n,m,r", [(100, 300, None), (300, 100, None), (200, 250, 77), (64, 64, 1), (50, 200, 0)])
def test_nullspace_annihilates(n, m, r):
    if r is None:
        A = f2gen.uniform(n, m, f2gen.BASE_SEED, 500 + n)
    elif r == 0:
        A = np.zeros((n, (m + 63) // 64), dtype=np.uint64)
    else:
        X, Y = f2gen.fixed_rank_factors(n, m, r, 600 + n)
        A = oracle.mmm(X, Y, r, m)
    res = oracle.nullspace(A, m)
    rk = oracle.rank(A, m)
    assert res["nul"] == m - rk
    Nb = bits(res["N"], res["nul"])
    assert not ((bits(A, m) @ Nb) % 2).any()
    # the rows at the free columns form the identity
    piv = oracle.rref(A, m)["pivcols"]
    free = np.setdiff1d(np.arange(m), piv)
    assert np.array_equal(Nb[free], np.eye(res["nul"], dtype=np.int64))
