"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle element by element."""
import numpy as np
import torch

import f2gen
import oracle
import paper_1209_5198_gb300 as gf2


def gpu_decompose(A_rm: np.ndarray, m: int, factors: bool = True, flags: int = 0):
    """Row-major words -> CUDA decomposition -> host numpy (row-major factors)."""
    n = A_rm.shape[0]
    A = gf2.Mat.from_rowmajor(A_rm, m, ld=n + 3)  # ld > rows exercises the stride
    out = gf2.decompose(A, factors=factors, flags=flags)
    torch.cuda.synchronize()
    res = dict(perm=out["perm"].cpu().numpy(), pivcols=out["pivcols"].cpu().numpy(),
               rank=int(out["rank"].item()))
    if factors:
        res["L"] = out["L"].to_rowmajor()
        res["E"] = out["E"].to_rowmajor()
    # the input must be untouched
    assert np.array_equal(A.to_rowmajor(), A_rm[:, : (m + 63) // 64])
    return res


def assert_same_decomposition(A_rm: np.ndarray, m: int, got: dict, factors: bool = True):
    ref = oracle.ple(A_rm, m, want_L=factors, want_E=factors, nthreads=oracle.max_threads())
    r = ref["rank"]
    assert got["rank"] == r
    assert np.array_equal(got["pivcols"][:r], ref["pivcols"])
    assert (got["pivcols"][r:] == -1).all()
    assert np.array_equal(got["perm"], ref["perm"])
    if factors:
        assert np.array_equal(got["L"], ref["L"]), "L differs"
        assert np.array_equal(got["E"], ref["E"]), "E differs"
    return ref
