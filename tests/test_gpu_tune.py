"""The autotuner on the device: it times the decomposition's speed-only
options, records the fastest for the shape bucket, and a decomposition with
automatic options then uses it and still matches the oracle bit for bit."""
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
def clean_table():
    gf2.tune_clear()
    yield
    gf2.tune_clear()


CANDIDATES = {(64, 8, 0), (64, 4, 0)} | {(128, c, s) for c in (4, 8) for s in (1, 2, 3)}


@pytest.mark.parametrize("n,m", [(1000, 1500), (2048, 2048)])
def test_autotune_records_and_is_used(clean_table, n, m):
    best = gf2.decompose_autotune(n, m)
    key = gf2.tune_device_key()
    assert best.device.decode() == key and best.ms > 0
    assert (best.opts.panel_w, best.opts.table_c, best.opts.schedule) in CANDIDATES
    bn = 1 << max(6, (n - 1).bit_length())
    bm = 1 << max(6, (m - 1).bit_length())
    assert (best.bucket_n, best.bucket_m) == (bn, bm)
    got = gf2.tune_lookup(key, n, m)
    assert got is not None and got.opts.panel_w == best.opts.panel_w and got.opts.schedule == best.opts.schedule
    # a decomposition with automatic options now runs the tuned choice: same bits as the oracle
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 77, n)
    out = gf2.decompose(gf2.Mat.from_rowmajor(A, m))
    torch.cuda.synchronize()
    ref = oracle.ple(A, m)
    r = ref["rank"]
    assert int(out["rank"].item()) == r
    assert np.array_equal(out["perm"].cpu().numpy(), ref["perm"])
    assert np.array_equal(out["L"].to_rowmajor(), ref["L"])
    assert np.array_equal(out["E"].to_rowmajor(), ref["E"])


def test_every_candidate_gives_the_oracle_factors(clean_table):
    """Each option the tuner may pick, forced through a table entry, gives
    the same factors (a tuned choice can never change a result)."""
    n, m = 1500, 1100
    A = f2gen.uniform(n, m, f2gen.BASE_SEED, 78)
    ref = oracle.ple(A, m)
    key = gf2.tune_device_key()
    for pw, tc, sch in sorted(CANDIDATES):
        e = gf2.TuneEntry()
        e.device = key.encode()
        e.kind = gf2.GF2_TUNE_DECOMPOSE
        e.bucket_n, e.bucket_m = 2048, 2048
        e.opts = gf2.Opts(panel_w=pw, table_c=tc, schedule=sch)
        e.ms = 1.0
        gf2.tune_put(e)
        out = gf2.decompose(gf2.Mat.from_rowmajor(A, m))
        torch.cuda.synchronize()
        assert int(out["rank"].item()) == ref["rank"], (pw, tc, sch)
        assert np.array_equal(out["perm"].cpu().numpy(), ref["perm"]), (pw, tc, sch)
        assert np.array_equal(out["E"].to_rowmajor(), ref["E"]), (pw, tc, sch)
        assert np.array_equal(out["L"].to_rowmajor(), ref["L"]), (pw, tc, sch)
