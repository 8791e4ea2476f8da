"""Parity of the CUDA decomposition with the oracle, bit for bit (perm,
pivcols, rank, L, E), on seeded synthetic inputs: the paper's dense random
workload, ragged and rectangular shapes, known-rank products, sparse
low-rank matrices and degenerate cases."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

from tests.gpu_util import assert_same_decomposition, gpu_decompose  # noqa: E402


def eye(n, m):
    w = np.zeros((n, (m + 63) // 64), dtype=np.uint64)
    for i in range(min(n, m)):
        w[i, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return w


CASES = {
    # the 1024 x 1024 Bernoulli(1/2) workload, several seeds
    "uniform-1024-s0": lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
    "uniform-1024-s1": lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 1), 1024),
    "uniform-1024-s2": lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 2), 1024),
    # ragged: several column tiles plus a partial word
    "ragged-1000x1300": lambda: (f2gen.uniform(1000, 1300, 3), 1300),
    "ragged-777x2111": lambda: (f2gen.uniform(777, 2111, 4), 2111),
    "tall-3000x500": lambda: (f2gen.uniform(3000, 500, 5), 500),
    "wide-500x3000": lambda: (f2gen.uniform(500, 3000, 6), 3000),
    "tiny-1x1": lambda: (np.ones((1, 1), dtype=np.uint64), 1),
    "tiny-5x7": lambda: (f2gen.uniform(5, 7, 7), 7),
    "exact-64x64": lambda: (f2gen.uniform(64, 64, 8), 64),
    "exact-65x65": lambda: (f2gen.uniform(65, 65, 9), 65),
    "one-row": lambda: (f2gen.uniform(1, 700, 10), 700),
    "one-col": lambda: (f2gen.uniform(700, 1, 11), 1),
    "zero": lambda: (np.zeros((300, 5), dtype=np.uint64), 300),
    "identity": lambda: (eye(300, 300), 300),
    "identity-reversed": lambda: (eye(300, 300)[::-1].copy(), 300),
    "bernoulli0.1-900": lambda: (f2gen.bernoulli(900, 900, 0.1, 12), 900),
    "sparse2-1000": lambda: (f2gen.sparse_rows(1000, 1000, 2, 13), 1000),
    "sparse10-1000": lambda: (f2gen.sparse_rows(1000, 1000, 10, 14), 1000),
    "sparse40-1000": lambda: (f2gen.sparse_rows(1000, 1000, 40, 15), 1000),
}


def fixed_rank(n, m, r, seed):
    X, Y = f2gen.fixed_rank_factors(n, m, r, seed)
    return oracle.mmm(X, Y, r, m, nthreads=oracle.max_threads()), m


CASES.update({
    "rank-half-1024": lambda: fixed_rank(1024, 1024, 512, 20),
    "rank-n-64-1024": lambda: fixed_rank(1024, 1024, 960, 21),
    "rank-1-800": lambda: fixed_rank(800, 900, 1, 22),
    "rank-37-1500x700": lambda: fixed_rank(1500, 700, 37, 23),
    "rank-half-2048x1600": lambda: fixed_rank(2048, 1600, 800, 24),
})


@pytest.mark.parametrize("name", sorted(CASES))
def test_decomposition_matches_oracle(name):
    A, m = CASES[name]()
    got = gpu_decompose(A, m)
    assert_same_decomposition(A, m, got)


@pytest.mark.parametrize("name", ["uniform-1024-s0", "rank-half-1024", "sparse10-1000"])
def test_rank_only_path(name):
    import paper_1209_5198_gb300 as gf2
    A, m = CASES[name]()
    got = gpu_decompose(A, m, factors=False)
    assert_same_decomposition(A, m, got, factors=False)
    assert gf2.gf2_rank(gf2.Mat.from_rowmajor(A, m)) == got["rank"]


def test_repeatable_and_seed_sensitive():
    A = f2gen.uniform(2000, 2000, 31)
    a = gpu_decompose(A, 2000)
    b = gpu_decompose(A, 2000)
    for key in ("perm", "pivcols", "L", "E"):
        assert np.array_equal(a[key], b[key])


def test_padding_is_rejected():
    import paper_1209_5198_gb300 as gf2
    A = f2gen.uniform(100, 70, 32)
    A[5, 1] |= np.uint64(1) << np.uint64(20)  # column 84 >= 70
    with pytest.raises(gf2.Gf2Error) as e:
        gpu_decompose(A, 70)
    assert e.value.status == gf2.GF2_ERR_PADDING


def test_host_entry_point():
    import paper_1209_5198_gb300 as gf2
    n, m = 1500, 1400
    A = f2gen.uniform(n, m, 33)
    k = min(n, m)
    cb = np.ascontiguousarray(f2gen.to_colblocks(A, ld=n + 5))
    perm = np.zeros(n, dtype=np.int32)
    piv = np.zeros(k, dtype=np.int32)
    rank = np.zeros(1, dtype=np.int64)
    L = np.zeros(((k + 63) // 64, n), dtype=np.uint64)
    E = np.zeros(((m + 63) // 64, k), dtype=np.uint64)
    gf2.gf2_decompose_host(n, m, cb, perm, piv, rank, L, E)
    got = dict(perm=perm, pivcols=piv, rank=int(rank[0]), L=f2gen.from_colblocks(L, n),
               E=f2gen.from_colblocks(E, k))
    assert_same_decomposition(A, m, got)
