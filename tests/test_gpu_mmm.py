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


@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (5, 70, 3), (64, 64, 64), (300, 130, 650), (1024, 1024, 1024),
                                   (1000, 1300, 777), (2048, 64, 4100), (129, 2000, 65)])
def test_product_matches_oracle(n, k, m):
    A = f2gen.uniform(n, k, 41, n, k)
    B = f2gen.uniform(k, m, 42, k, m)
    ref = oracle.mmm(A, B, k, m, nthreads=oracle.max_threads())
    Ad = gf2.Mat.from_rowmajor(A, k, ld=n + 1)
    Bd = gf2.Mat.from_rowmajor(B, m)
    Cd = gf2.Mat.empty(n, m, ld=n + 7)
    gf2.gf2_mmm(Ad, Bd, Cd)
    assert np.array_equal(Cd.to_rowmajor(), ref)
    # accumulate: C ^= A*B twice gives back the original C
    C0 = f2gen.uniform(n, m, 43, n, m)
    Cd = gf2.Mat.from_rowmajor(C0, m)
    gf2.gf2_mmm(Ad, Bd, Cd, accumulate=True)
    assert np.array_equal(Cd.to_rowmajor(), ref ^ C0)
    gf2.gf2_mmm(Ad, Bd, Cd, accumulate=True)
    assert np.array_equal(Cd.to_rowmajor(), C0)


def test_product_of_fixed_rank_factors_has_that_rank():
    n, m, r = 2048, 2048, 700
    X, Y = f2gen.fixed_rank_factors(n, m, r, 44)
    A = gf2.mmm(gf2.Mat.from_rowmajor(X, r), gf2.Mat.from_rowmajor(Y, m))
    assert gf2.gf2_rank(A) == r
