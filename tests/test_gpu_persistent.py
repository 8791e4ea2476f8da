"""The persistent schedule of the decomposition (one cooperative launch:
CTA 0 runs the panel chain, the other CTAs the look-ahead and the pair
updates, ordered by device counters) gives the oracle's factors bit for bit
on every shape, and so does the separate-launch schedule on shapes where
the automatic choice would take the persistent one."""
import numpy as np
import pytest

import f2gen
import oracle
from tests.gpu_util import assert_same_decomposition

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402

NT = oracle.max_threads()


def run(A, m, opts, factors=True):
    n = A.shape[0]
    k = min(n, m)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    piv = torch.empty(max(k, 1), dtype=torch.int32, device="cuda")
    rank = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = gf2.Mat.empty(n, k) if factors else None
    E = gf2.Mat.empty(k, m) if factors else None
    gf2.gf2_decompose_ex(gf2.Mat.from_rowmajor(A, m, ld=n + 1), perm, piv, rank, L, E, opts)
    torch.cuda.synchronize()
    got = dict(perm=perm.cpu().numpy()[:n], pivcols=piv.cpu().numpy()[:k], rank=int(rank.item()))
    if factors:
        got["L"] = L.to_rowmajor()
        got["E"] = E.to_rowmajor()
    return got


def shapes():
    X, Y = f2gen.fixed_rank_factors(3000, 2900, 1234, 90)
    X2, Y2 = f2gen.fixed_rank_factors(2048, 2048, 7, 91)
    return [
        ("1x1", f2gen.uniform(1, 1, 92), 1),
        ("64x64", f2gen.uniform(64, 64, 93), 64),
        ("65x65", f2gen.uniform(65, 65, 94), 65),
        ("one row", f2gen.uniform(1, 700, 95), 700),
        ("one column", f2gen.uniform(900, 1, 96), 1),
        ("128x256", f2gen.uniform(128, 256, 97), 256),
        ("1024 dense", f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
        ("ragged 1500x1333", f2gen.uniform(1500, 1333, 98), 1333),
        ("tall 5000x700", f2gen.uniform(5000, 700, 99), 700),
        ("wide 700x5000", f2gen.uniform(700, 5000, 100), 5000),
        ("odd blocks 4100x4100", f2gen.uniform(4100, 4100, 101), 4100),
        ("rank 1234", oracle.mmm(X, Y, 1234, 2900, nthreads=NT), 2900),
        ("rank 7", oracle.mmm(X2, Y2, 7, 2048, nthreads=NT), 2048),
        ("zero", np.zeros((1000, 16), dtype=np.uint64), 1000),
        ("identity", f2gen.pack_bits(np.eye(777, dtype=np.uint8)), 777),
        ("sparse i=2", f2gen.sparse_rows(3000, 3000, 2, 102), 3000),
        ("sparse i=10", f2gen.sparse_rows(2500, 2500, 10, 103), 2500),
        ("bernoulli 0.1", f2gen.bernoulli(2000, 2100, 0.1, 104), 2100),
    ]


@pytest.mark.parametrize("name", [s[0] for s in shapes()])
@pytest.mark.parametrize("table_c", [0, 4])
def test_persistent_schedule_matches_oracle(name, table_c):
    A, m = next((a, m) for nm, a, m in shapes() if nm == name)
    o = gf2.Opts(schedule=gf2.SCHEDULE_PERSISTENT, table_c=table_c)
    gf2.timing(True)
    try:
        got = run(A, m, o)
        launches = gf2.timing_read()["factor"][1]
    finally:
        gf2.timing(False)
    if min(A.shape[0], m) > 0:
        assert launches == 1, "the persistent kernel did not run"
    assert_same_decomposition(A, m, got)


def test_persistent_rank_only_and_repeat():
    A = f2gen.uniform(6000, 6000, 105)
    o = gf2.Opts(schedule=gf2.SCHEDULE_PERSISTENT)
    ref = oracle.ple(A, 6000, want_L=False, want_E=False, nthreads=NT)
    for _ in range(3):  # the counters are cleared before every run
        got = run(A, 6000, o, factors=False)
        assert got["rank"] == ref["rank"]
        assert np.array_equal(got["perm"], ref["perm"])
        assert np.array_equal(got["pivcols"][:ref["rank"]], ref["pivcols"])


@pytest.mark.parametrize("n,m", [(4160, 4160), (8192, 3000)])
def test_stream_schedule_at_sizes_where_auto_is_persistent(n, m):
    A = f2gen.uniform(n, m, 106, n, m)
    got = run(A, m, gf2.Opts(schedule=gf2.SCHEDULE_STREAMS))
    assert_same_decomposition(A, m, got)


def test_auto_is_the_stream_schedule():
    gf2.timing(True)
    try:
        run(f2gen.uniform(6000, 3000, 107), 3000, None, factors=False)
        t = gf2.timing_read()
    finally:
        gf2.timing(False)
    assert t["factor"][1] == 0 and t["panel"][1] > 0


@pytest.mark.parametrize("name", ["tall", "square", "rank", "sparse", "wide"])
def test_split_schedule_matches_oracle(name):
    """SPLIT: the first three quarters of the panels as separate launches,
    the rest in the persistent launch (from the workspace state they leave)."""
    if name == "tall":
        A, m = f2gen.uniform(9000, 1400, 110), 1400
    elif name == "square":
        A, m = f2gen.uniform(6000, 6000, 111), 6000
    elif name == "rank":
        X, Y = f2gen.fixed_rank_factors(5000, 5000, 2500, 112)
        A, m = oracle.mmm(X, Y, 2500, 5000, nthreads=NT), 5000
    elif name == "sparse":
        A, m = f2gen.sparse_rows(5000, 5000, 3, 113), 5000
    else:
        A, m = f2gen.uniform(4096, 7000, 114), 7000
    gf2.timing(True)
    try:
        got = run(A, m, gf2.Opts(schedule=gf2.SCHEDULE_SPLIT))
        t = gf2.timing_read()
    finally:
        gf2.timing(False)
    assert t["factor"][1] == 1 and t["panel"][1] > 0, "not the split schedule"
    assert_same_decomposition(A, m, got)
