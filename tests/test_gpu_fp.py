"""Parity of the decomposition over F_p (gf2_fp_decompose) with the oracle
(oracle/fp.py), element by element: perm, pivot columns, rank, L and E, on
dense, ragged, tall, wide, fixed-rank, zero and identity matrices and on
primes from 2 to 2^31 - 1; at p = 2 also against the F2 decomposition."""
import numpy as np
import pytest

import f2gen
from oracle import fp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


def run(A: np.ndarray, p: int):
    out = gf2.fp_decompose(torch.from_numpy(np.ascontiguousarray(A, dtype=np.int32)).cuda(), p)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


def compare(A, p):
    ref = fp.ple(A, p)
    got = run(A, p)
    r = ref["rank"]
    assert int(got["rank"][0]) == r
    assert np.array_equal(got["perm"], ref["perm"])
    assert np.array_equal(got["pivcols"][:r], ref["pivcols"])
    assert (got["pivcols"][r:] == -1).all()
    assert np.array_equal(got["L"].astype(np.int64), ref["L"])
    assert np.array_equal(got["E"].astype(np.int64), ref["E"])


def product(X, Y, p):
    return ((X.astype(object) @ Y.astype(object)) % p).astype(np.int64)


PRIMES = [2, 3, 5, 251, 65521, 1000003, 2147483647]


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,m", [(1, 1), (5, 7), (64, 64), (100, 37), (37, 100), (300, 333), (1100, 700)])
def test_uniform_matches_oracle(n, m, p):
    compare(f2gen.fp_uniform(n, m, p, 910, n, m), p)


@pytest.mark.parametrize("p", [3, 65521, 2147483647])
@pytest.mark.parametrize("n,m,r", [(200, 150, 75), (150, 200, 149), (512, 512, 1), (700, 600, 333)])
def test_fixed_rank_matches_oracle(n, m, r, p):
    X, Y = f2gen.fp_fixed_rank_factors(n, m, r, p, 911, n)
    A = product(X, Y, p)
    compare(A, p)


@pytest.mark.parametrize("p", [2, 7, 2147483647])
def test_degenerate(p):
    compare(np.zeros((90, 70), dtype=np.int64), p)
    compare(np.eye(80, dtype=np.int64), p)
    compare(np.eye(80, dtype=np.int64)[::-1].copy(), p)
    A = f2gen.fp_uniform(130, 90, p, 912)
    A[:, 10:40] = 0  # a band of zero columns: no pivots there
    compare(A, p)


def test_larger_matches_oracle():
    p = 65521
    compare(f2gen.fp_uniform(1024, 1024, p, 913), p)


def test_p2_equals_the_f2_decomposition():
    n, m = 700, 900
    words = f2gen.uniform(n, m, 914)
    bits = f2gen.unpack_bits(words, m).astype(np.int64)
    got = run(bits, 2)
    out = gf2.decompose(gf2.Mat.from_rowmajor(words, m))
    torch.cuda.synchronize()
    r = int(out["rank"].item())
    assert int(got["rank"][0]) == r
    assert np.array_equal(got["perm"], out["perm"].cpu().numpy())
    assert np.array_equal(got["E"][:r], f2gen.unpack_bits(out["E"].to_rowmajor(), m)[:r])
    assert np.array_equal(got["L"][:, :r], f2gen.unpack_bits(out["L"].to_rowmajor(), min(n, m))[:, :r])


def test_argument_errors():
    A = torch.zeros((10, 10), dtype=torch.int32, device="cuda")
    for bad_p in (0, 1, 4, 65535, 2 ** 31 + 11):
        with pytest.raises(gf2.Gf2Error) as e:
            gf2.fp_decompose(A, bad_p)
        assert e.value.status == gf2.GF2_ERR_ARG
    A[3, 4] = 7  # an entry >= p
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.fp_decompose(A, 7)
    assert e.value.status == gf2.GF2_ERR_ARG
    assert gf2.fp_is_prime(2147483647) and not gf2.fp_is_prime(2147483647 - 2)


def test_bounded_barrier_gives_up_then_recovers():
    """With one poll per grid-wide wait the multi-CTA panel launch gives up
    (rank -1, nothing traps or hangs); the next call is correct again."""
    p = 251
    A = f2gen.fp_uniform(4096, 96, p, 915)
    At = torch.from_numpy(A.astype(np.int32)).cuda()
    gave_up = False
    try:
        gf2.set_wait_limit(1)
        for _ in range(3):
            out = gf2.fp_decompose(At, p)
            torch.cuda.synchronize()
            if int(out["rank"].item()) == -1:
                gave_up = True
                break
    finally:
        gf2.set_wait_limit(0)
    assert gave_up
    compare(A, p)
