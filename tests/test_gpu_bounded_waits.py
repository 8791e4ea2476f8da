"""Bounded device-side waits give up without trapping or hanging: with a
limit of one poll (gf2_debug_set_wait_limit), the grid-wide barriers of
gf2_solve and the progress counters of the persistent decomposition run out,
the calls report GF2_ERR_TIMEOUT, and the GPU context stays usable -- the
same calls with the default limit then match the oracle.  No fault is
provoked: every wait returns by itself."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402


@pytest.fixture
def one_poll():
    gf2.set_wait_limit(1)
    yield
    gf2.set_wait_limit(0)


def test_solve_barrier_gives_up_then_recovers(one_poll):
    n = 8192
    A = f2gen.uniform(n, n, 120)
    B = f2gen.uniform(n, 5, 121).reshape(-1)
    fac = gf2.decompose(gf2.Mat.from_rowmajor(A, n), factors=True)
    Bd = gf2.Mat.from_rowmajor(B.reshape(-1, 1), 5)
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.solve(fac, Bd, n)
    assert e.value.status == gf2.GF2_ERR_TIMEOUT
    gf2.set_wait_limit(0)
    out = gf2.solve(fac, Bd, n)
    ref = oracle.solve(A, n, B, 5)
    assert out["consistent"] == ref["consistent"]
    assert np.array_equal(out["X"].to_rowmajor().reshape(-1), ref["X"])


def test_persistent_waits_give_up_then_recover(one_poll):
    n = 6000
    A = f2gen.uniform(n, n, 122)
    Ad = gf2.Mat.from_rowmajor(A, n)
    o = gf2.Opts(schedule=gf2.SCHEDULE_PERSISTENT)
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.gf2_rank_ex(Ad, o)
    assert e.value.status == gf2.GF2_ERR_TIMEOUT
    gf2.set_wait_limit(0)
    assert gf2.gf2_rank_ex(Ad, o) == oracle.rank(A, n, nthreads=oracle.max_threads())


def test_wait_limit_argument_checks():
    lib = gf2.load()
    assert lib.gf2_debug_set_wait_limit(-1) == gf2.GF2_ERR_ARG
    assert lib.gf2_debug_set_wait_limit(1 << 32) == gf2.GF2_ERR_ARG
    assert lib.gf2_debug_set_wait_limit(0) == gf2.GF2_OK
