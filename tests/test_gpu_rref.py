"""Parity of the CUDA reduced row echelon form (gf2_rref on the E factor of
gf2_decompose) with the oracle's textbook Gauss-Jordan, bit for bit: the RREF
is unique, so the two routes must agree exactly.  Shapes span one to many
64-row blocks (several levels of the host recursion), ragged column words,
rank deficiency, sparse rows and degenerate cases; the 32768 x 32768 input
of the benchmark is checked by invariants on sampled rows."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


def eye(n, m):
    w = np.zeros((n, (m + 63) // 64), dtype=np.uint64)
    for i in range(min(n, m)):
        w[i, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return w


def fixed_rank(n, m, r, seed):
    X, Y = f2gen.fixed_rank_factors(n, m, r, seed)
    return oracle.mmm(X, Y, r, m, nthreads=oracle.max_threads()), m


CASES = {
    "uniform-300x333": lambda: (f2gen.uniform(300, 333, f2gen.BASE_SEED, 31), 333),
    "uniform-1024": lambda: (f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
    "ragged-1000x1300": lambda: (f2gen.uniform(1000, 1300, 32), 1300),
    "tall-2000x500": lambda: (f2gen.uniform(2000, 500, 33), 500),
    "wide-200x2000": lambda: (f2gen.uniform(200, 2000, 34), 2000),
    "wide-1300x4000": lambda: (f2gen.uniform(1300, 4000, 35), 4000),
    "rank-600-1024": lambda: fixed_rank(1024, 1024, 600, 36),
    "rank-37-500x700": lambda: fixed_rank(500, 700, 37, 37),
    "rank-1-300": lambda: fixed_rank(300, 300, 1, 38),
    "sparse2-1000": lambda: (f2gen.sparse_rows(1000, 1000, 2, 39), 1000),
    "bernoulli0.1-900": lambda: (f2gen.bernoulli(900, 900, 0.1, 40), 900),
    "zero-100": lambda: (np.zeros((100, 2), dtype=np.uint64), 100),
    "identity-300": lambda: (eye(300, 300), 300),
    "identity-reversed-300": lambda: (eye(300, 300)[::-1].copy(), 300),
    "tiny-1x1": lambda: (np.ones((1, 1), dtype=np.uint64), 1),
    "exact-64x64": lambda: (f2gen.uniform(64, 64, 41), 64),
    "exact-65x65": lambda: (f2gen.uniform(65, 65, 42), 65),
    "one-row": lambda: (f2gen.uniform(1, 700, 43), 700),
    "one-col": lambda: (f2gen.uniform(700, 1, 44), 1),
    "uniform-4096": lambda: (f2gen.uniform(4096, 4096, f2gen.BASE_SEED, 45), 4096),
}


def gpu_rref(A_rm, m):
    n = A_rm.shape[0]
    out = gf2.decompose(gf2.Mat.from_rowmajor(A_rm, m))
    piv_before = out["pivcols"].clone()
    E = gf2.rref(out)
    torch.cuda.synchronize()
    r = int(out["rank"].item())
    assert torch.equal(out["pivcols"], piv_before)  # the pivots are not touched
    return E.to_rowmajor(), out["pivcols"].cpu().numpy(), r, min(n, m)


@pytest.mark.parametrize("name", sorted(CASES))
def test_rref_matches_oracle(name):
    A, m = CASES[name]()
    R, piv, r, k = gpu_rref(A, m)
    ref = oracle.rref(A, m)
    assert r == ref["rank"]
    assert np.array_equal(piv[:r], ref["pivcols"])
    assert np.array_equal(R[:r], ref["R"]), "reduced rows differ"
    assert not R[r:k].any(), "rows past the rank must stay zero"


def test_rref_is_idempotent():
    A, m = CASES["rank-600-1024"]()
    out = gf2.decompose(gf2.Mat.from_rowmajor(A, m))
    once = gf2.rref(out).to_rowmajor()
    twice = gf2.rref(out).to_rowmajor()
    assert np.array_equal(once, twice)


def test_rref_empty_and_errors():
    E = gf2.Mat.empty(0, 10)
    piv = torch.empty(1, dtype=torch.int32, device="cuda")
    gf2.gf2_rref(E, piv)  # nothing to do
    E = gf2.Mat.empty(5, 0)
    gf2.gf2_rref(E, piv)
    lib = gf2.load()
    assert lib.gf2_rref(None, None, None, 0, None) == gf2.GF2_ERR_ARG
    E = gf2.Mat.empty(70, 70)
    e = E.c()
    assert lib.gf2_rref(gf2.ctypes.byref(e), None, None, 0, None) == gf2.GF2_ERR_ARG
    bad = gf2._CMat(E.t.data_ptr(), 70, 70, 60)  # ld < rows
    assert lib.gf2_rref(gf2.ctypes.byref(bad), piv.data_ptr(), None, 0, None) == gf2.GF2_ERR_SHAPE
    assert lib.gf2_rref_workspace_bytes(-1, 5) == 0
    ws = lib.gf2_rref_workspace_bytes(70, 70)
    tiny = torch.empty(8, dtype=torch.uint8, device="cuda")
    piv70 = torch.full((70,), -1, dtype=torch.int32, device="cuda")
    assert ws > 8
    assert lib.gf2_rref(gf2.ctypes.byref(e), piv70.data_ptr(), tiny.data_ptr(), 8, None) == gf2.GF2_ERR_NOMEM


def test_rref_full_size_invariants():
    """32768 x 32768 Bernoulli(1/2): with E saved before the reduction, for
    sampled rows t: R_t is a unit vector on the pivot columns (bit t), and
    E_t = XOR of the R_s over the pivots s whose column E_t has set (E = U R
    with U = E at the pivot columns)."""
    n = m = 32768
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 0)
    out = gf2.decompose(gf2.Mat.from_rowmajor(A, m))
    Ebefore = out["E"].t.clone()
    R = gf2.rref(out)
    torch.cuda.synchronize()
    r = int(out["rank"].item())
    piv = out["pivcols"][:r].cpu().numpy().astype(np.int64)
    Rh = R.to_rowmajor()[:r]
    Eh = gf2.Mat(Ebefore, n, m).to_rowmajor()[:r]
    rng = np.random.default_rng(7)
    rows = np.concatenate([[0, 1, r - 1, r - 2], rng.choice(r, 28, replace=False)])
    for t in rows:
        on_piv = (Rh[t, piv >> 6] >> (piv & 63).astype(np.uint64)) & np.uint64(1)
        assert on_piv.sum() == 1 and on_piv[t] == 1, t
        sel = ((Eh[t, piv >> 6] >> (piv & 63).astype(np.uint64)) & np.uint64(1)).astype(bool)
        assert np.array_equal(np.bitwise_xor.reduce(Rh[sel], axis=0), Eh[t]), t
