"""Parity of the CUDA product over F2 with the oracle, bit for bit."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


BACKENDS = {"auto": 0, "tables": gf2.GF2_MMM_TABLES, "tensor": gf2.GF2_MMM_TENSOR, "strassen": 0}


@pytest.fixture
def cutoff():
    """Runs the test with a given Strassen cutoff, restoring the old one."""
    old = gf2.strassen_cutoff()
    yield gf2.set_strassen_cutoff
    gf2.set_strassen_cutoff(old)


@pytest.mark.parametrize("backend", sorted(BACKENDS))
@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (5, 70, 3), (64, 64, 64), (300, 130, 650), (1024, 1024, 1024),
                                   (1000, 1300, 777), (2048, 64, 4100), (129, 2000, 65), (257, 4099, 191),
                                   (1024, 2048, 1000), (4000, 512, 768), (2048, 2048, 2048)])
def test_product_matches_oracle(n, k, m, backend, cutoff):
    flags = BACKENDS[backend]
    cutoff(128 if backend == "strassen" else gf2.STRASSEN_OFF)
    A = f2gen.uniform(n, k, 41, n, k)
    B = f2gen.uniform(k, m, 42, k, m)
    ref = oracle.mmm(A, B, k, m, nthreads=oracle.max_threads())
    Ad = gf2.Mat.from_rowmajor(A, k, ld=n + 1)
    Bd = gf2.Mat.from_rowmajor(B, m)
    Cd = gf2.Mat.empty(n, m, ld=n + 7)
    gf2.gf2_mmm(Ad, Bd, Cd, flags=flags)
    assert np.array_equal(Cd.to_rowmajor(), ref)
    # accumulate: C ^= A*B twice gives back the original C
    C0 = f2gen.uniform(n, m, 43, n, m)
    Cd = gf2.Mat.from_rowmajor(C0, m)
    gf2.gf2_mmm(Ad, Bd, Cd, accumulate=True, flags=flags)
    assert np.array_equal(Cd.to_rowmajor(), ref ^ C0)
    gf2.gf2_mmm(Ad, Bd, Cd, accumulate=True, flags=flags)
    assert np.array_equal(Cd.to_rowmajor(), C0)


def test_product_dense_ones_exact():
    """All-ones operands: every sum is k, the largest the accumulator holds
    here; entry parity = k mod 2 for both backends."""
    for k in (4095, 4096):
        n = m = 200
        A = np.full((n, (k + 63) // 64), ~np.uint64(0), dtype=np.uint64)
        if k % 64:
            A[:, -1] = (np.uint64(1) << np.uint64(k % 64)) - np.uint64(1)
        B = np.full((k, (m + 63) // 64), ~np.uint64(0), dtype=np.uint64)
        B[:, -1] = (np.uint64(1) << np.uint64(m % 64)) - np.uint64(1)
        ref = oracle.mmm(A, B, k, m)
        for flags in (gf2.GF2_MMM_TABLES, gf2.GF2_MMM_TENSOR):
            Cd = gf2.Mat.empty(n, m)
            gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, k), gf2.Mat.from_rowmajor(B, m), Cd, flags=flags)
            assert np.array_equal(Cd.to_rowmajor(), ref)


@pytest.mark.parametrize("k", [16385, 32769, 65537])
def test_product_long_inner_dimension_ones_exact(k):
    """All-ones operands with sums far above what a low-precision
    accumulation keeps exactly (k > 2^14): every entry is k mod 2 = 1.  The
    tensor-core kernel folds its sums into parity bits every 4096 of the
    inner dimension; both backends must match the oracle."""
    n = m = 128
    A = np.full((n, (k + 63) // 64), ~np.uint64(0), dtype=np.uint64)
    A[:, -1] = (np.uint64(1) << np.uint64(k % 64)) - np.uint64(1)
    B = np.full((k, (m + 63) // 64), ~np.uint64(0), dtype=np.uint64)
    ref = oracle.mmm(A, B, k, m)
    assert (ref == ~np.uint64(0)).all()  # k odd: every entry 1
    for flags in (gf2.GF2_MMM_TABLES, gf2.GF2_MMM_TENSOR):
        Cd = gf2.Mat.empty(n, m)
        gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, k), gf2.Mat.from_rowmajor(B, m), Cd, flags=flags)
        assert np.array_equal(Cd.to_rowmajor(), ref), flags


def test_product_padding_error_both_backends():
    A = f2gen.uniform(100, 300, 45)
    A[7, 4] |= np.uint64(1) << np.uint64(50)  # column 306 >= 300
    B = f2gen.uniform(300, 100, 46)
    for flags in (gf2.GF2_MMM_TABLES, gf2.GF2_MMM_TENSOR):
        with pytest.raises(gf2.Gf2Error) as e:
            gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, 300), gf2.Mat.from_rowmajor(B, 100), gf2.Mat.empty(100, 100),
                        flags=flags)
        assert e.value.status == gf2.GF2_ERR_PADDING


def test_strassen_levels_and_ragged_edges(cutoff):
    """Recursion depths 1..3 (cutoff 256: 2048 -> 1024 -> 512 -> 256), a ragged
    m (padding bits stay zero through the additions), and accumulate."""
    cutoff(256)
    for n, k, m in ((2048, 2048, 2048), (512, 1024, 1000), (1536, 768, 1280)):
        A = f2gen.uniform(n, k, 47, n)
        B = f2gen.uniform(k, m, 48, k)
        C0 = f2gen.uniform(n, m, 49, n)
        ref = oracle.mmm(A, B, k, m, nthreads=oracle.max_threads())
        Cd = gf2.Mat.from_rowmajor(C0, m, ld=n + 3)
        gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, k, ld=n + 1), gf2.Mat.from_rowmajor(B, m, ld=k + 2), Cd,
                    accumulate=True)
        assert np.array_equal(Cd.to_rowmajor(), ref ^ C0)
        Cd = gf2.Mat.empty(n, m)
        gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, k), gf2.Mat.from_rowmajor(B, m), Cd)
        assert np.array_equal(Cd.to_rowmajor(), ref)


def test_product_of_fixed_rank_factors_has_that_rank():
    n, m, r = 2048, 2048, 700
    X, Y = f2gen.fixed_rank_factors(n, m, r, 44)
    A = gf2.mmm(gf2.Mat.from_rowmajor(X, r), gf2.Mat.from_rowmajor(Y, m))
    assert gf2.gf2_rank(A) == r


def test_tensor_peak_probe_runs():
    """The tensor pipe probe (the tensor backend's MMA shape from shared
    memory) returns a positive dense rate and leaves the context usable."""
    tf = gf2.tensor_peak(256)
    assert tf > 0.0
    A = f2gen.uniform(256, 256, 50)
    B = f2gen.uniform(256, 300, 51)
    Cd = gf2.Mat.empty(256, 300)
    gf2.gf2_mmm(gf2.Mat.from_rowmajor(A, 256), gf2.Mat.from_rowmajor(B, 300), Cd, flags=gf2.GF2_MMM_TENSOR)
    assert np.array_equal(Cd.to_rowmajor(), oracle.mmm(A, B, 256, 300))
