"""Parity of the batched decomposition (one persistent launch over many
matrices) with the oracle, matrix by matrix, bit for bit: perm, pivot
columns, rank, L and E, on batches of mixed sizes, densities and ranks."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402
from tests.gpu_util import assert_same_decomposition  # noqa: E402


def batch_inputs(count, lo, hi, seed):
    """Mixed batch: uniform sizes in [lo, hi], densities 1/2 and 1/10, every
    third matrix a product X Y of random rank r."""
    rng = np.random.default_rng(seed)
    mats = []
    for i in range(count):
        n, m = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        if i % 3 == 2:
            r = int(rng.integers(1, min(n, m) + 1))
            X, Y = f2gen.fixed_rank_factors(n, m, r, seed, i)
            A = oracle.mmm(X, Y, r, m)
        elif i % 3 == 1:
            A = f2gen.bernoulli(n, m, 0.1, seed, i)
        else:
            A = f2gen.uniform(n, m, seed, i)
        mats.append((A, m))
    return mats


def run_batch(mats, factors=True):
    As = [gf2.Mat.from_rowmajor(A, m, ld=A.shape[0] + 1) for A, m in mats]
    outs = gf2.decompose_batched(As, factors=factors)
    torch.cuda.synchronize()
    res = []
    for (A, m), o in zip(mats, outs):
        got = dict(perm=o["perm"].cpu().numpy(), pivcols=o["pivcols"].cpu().numpy(), rank=int(o["rank"].item()))
        if factors:
            got["L"] = o["L"].to_rowmajor()
            got["E"] = o["E"].to_rowmajor()
        res.append(got)
    return res


def test_batched_mixed_sizes_match_oracle():
    mats = batch_inputs(40, 1, 400, 71)
    for (A, m), got in zip(mats, run_batch(mats)):
        assert_same_decomposition(A, m, got)


def test_batched_larger_matrices_match_oracle():
    mats = batch_inputs(12, 300, 1300, 72)
    for (A, m), got in zip(mats, run_batch(mats)):
        assert_same_decomposition(A, m, got)


def test_batched_rank_only():
    mats = batch_inputs(30, 1, 500, 73)
    for (A, m), got in zip(mats, run_batch(mats, factors=False)):
        assert_same_decomposition(A, m, got, factors=False)


def test_batched_degenerate_and_more_matrices_than_ctas():
    mats = [(np.zeros((5, 1), dtype=np.uint64), 64), (np.ones((1, 1), dtype=np.uint64), 1),
            (f2gen.uniform(64, 64, 74), 64), (np.zeros((200, 3), dtype=np.uint64), 150)]
    mats += batch_inputs(900, 1, 96, 75)  # more matrices than resident CTAs
    got = run_batch(mats)
    for (A, m), g in zip(mats, got):
        assert_same_decomposition(A, m, g)


def test_batched_padding_error():
    A = f2gen.uniform(50, 70, 76)
    A[3, 1] |= np.uint64(1) << np.uint64(20)  # column 84 >= 70
    with pytest.raises(gf2.Gf2Error) as e:
        run_batch([(f2gen.uniform(40, 40, 77), 40), (A, 70)])
    assert e.value.status == gf2.GF2_ERR_PADDING


@pytest.mark.parametrize("c8_from", [1, 300, 1 << 62])
def test_batched_table_sizes_match_oracle(c8_from):
    """Every matrix on the 8-bit-table kernel (c8_from = 1), every one on the
    4-bit-table kernel (2^62), and a split batch whose two kernels run side
    by side (300): the same bits as the oracle."""
    old = gf2.batched_c8_from()
    try:
        gf2.set_batched_c8_from(c8_from)
        mats = batch_inputs(24, 1, 700, 78)
        mats.append((f2gen.uniform(1100, 900, 79), 900))
        for (A, m), got in zip(mats, run_batch(mats)):
            assert_same_decomposition(A, m, got)
        # the padding status still comes back from either kernel
        A = f2gen.uniform(500, 70, 80)
        A[3, 1] |= np.uint64(1) << np.uint64(20)
        with pytest.raises(gf2.Gf2Error) as e:
            run_batch([(f2gen.uniform(40, 40, 81), 40), (A, 70), (f2gen.uniform(600, 600, 82), 600)])
        assert e.value.status == gf2.GF2_ERR_PADDING
    finally:
        gf2.set_batched_c8_from(old)


def test_batched_autotune_sets_a_threshold():
    old = gf2.batched_c8_from()
    try:
        t = gf2.batched_autotune(1024)
        assert t == gf2.batched_c8_from()
        assert t in (128, 256, 512, 1024) or t == 1 << 62
        mats = batch_inputs(10, 100, 600, 83)
        for (A, m), got in zip(mats, run_batch(mats)):
            assert_same_decomposition(A, m, got)
    finally:
        gf2.set_batched_c8_from(old)
