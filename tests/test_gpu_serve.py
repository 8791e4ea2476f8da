"""The serving engine (gf2_server_*): every result equals the oracle's --
rank, consistency mask and the solution with free variables 0 -- and is the
same whether the request runs alone or in the mix (continuous batching,
requests arriving while others are on the GPU, misses decomposed in batched
and plain launches, factors evicted and rebuilt under a small memory
budget), and the same as the one-at-a-time baseline."""
import numpy as np
import pytest

import f2gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA not available", allow_module_level=True)

import paper_1209_5198_gb300 as gf2  # noqa: E402

SIZES = [(64, 64), (100, 300), (333, 200), (256, 256), (512, 512), (448, 500), (700, 650), (1024, 1024),
         (1100, 1500), (2000, 1300)]


class Workload:
    """Seeded matrices (one per key, some of deficient rank) and requests on
    them with keys reused; the host buffers stay alive with the object."""

    def __init__(self, nreq: int, seed: int, sizes=SIZES, keys_per_size: int = 1):
        rng = np.random.default_rng(seed)
        self.mats = {}
        key = 0
        for (n, m) in sizes:
            for _ in range(keys_per_size):
                if key % 3 == 2:  # deficient rank: a product X*Y of rank r
                    r = max(1, min(n, m) // 2)
                    X, Y = f2gen.fixed_rank_factors(n, m, r, seed, key)
                    A = oracle.mmm(X, Y, r, m)
                else:
                    A = f2gen.uniform(n, m, seed, key)
                self.mats[key] = (A, n, m, gf2.host_colblocks(A, m))
                key += 1
        keys = sorted(self.mats)
        self.req = np.zeros(nreq, dtype=gf2.REQUEST_DTYPE)
        self.B, self.X, self.nrhs = [], [], []
        for i in range(nreq):
            k = int(keys[rng.integers(len(keys))]) if i >= len(keys) else keys[i]
            A, n, m, Ah = self.mats[k]
            nrhs = int(rng.choice([0, 1, 7, 33, 64]))
            if nrhs:
                X0 = f2gen.rhs_from_solution(nrhs, m, seed, 1000 + i)
                B = oracle.mmm(A, X0, m, nrhs).reshape(-1)
                if i % 4 == 3:  # some right-hand sides random (mostly inconsistent when deficient)
                    B = f2gen.uniform(n, nrhs, seed, 2000 + i).reshape(-1)
            else:
                B = np.zeros(n, dtype=np.uint64)
            X = np.zeros(m, dtype=np.uint64)
            self.B.append(np.ascontiguousarray(B, dtype=np.uint64))
            self.X.append(X)
            self.nrhs.append(nrhs)
            self.req[i] = (i, k, n, m, Ah.data_ptr(), n, nrhs, self.B[i].ctypes.data, X.ctypes.data, 0.0)
        self._expected = None

    def expected(self):
        if self._expected is None:
            ranks = {k: oracle.rank(A, m) for k, (A, n, m, _) in self.mats.items()}
            exp = []
            for i, r in enumerate(self.req):
                A, n, m, _ = self.mats[int(r["matrix"])]
                if self.nrhs[i]:
                    ref = oracle.solve(A, m, self.B[i], self.nrhs[i])
                    exp.append((ranks[int(r["matrix"])], int(ref["consistent"]), ref["X"].copy()))
                else:
                    exp.append((ranks[int(r["matrix"])], 0, np.zeros(m, dtype=np.uint64)))
            self._expected = exp
        return self._expected

    def results(self, done: np.ndarray):
        out = {}
        for c in done:
            i = int(c["id"])
            assert c["status"] == gf2.GF2_OK, (i, gf2.status_string(int(c["status"])))
            out[i] = (int(c["rank"]), int(c["consistent"]), self.X[i].copy())
        assert sorted(out) == list(range(len(self.req)))
        return out

    def check(self, got: dict):
        for i, (rank, cons, X) in enumerate(self.expected()):
            g = got[i]
            assert g[0] == rank, f"request {i}: rank {g[0]} != {rank}"
            assert g[1] == cons, f"request {i}: consistent {g[1]:#x} != {cons:#x}"
            assert np.array_equal(g[2], X), f"request {i}: X differs"


def run(server: gf2.Server, w: Workload, arrivals=None):
    req = w.req.copy()
    if arrivals is not None:
        req["arrival_us"] = server.clock_us() + 2000.0 + np.asarray(arrivals)
    for X in w.X:
        X[:] = 0
    server.submit(req)
    return w.results(server.wait_all(len(req), timeout_s=300))


def test_mix_matches_oracle_and_stats():
    w = Workload(90, seed=11)
    with gf2.Server(1 << 30, 2048, 2048, max_batch=64) as s:
        got = run(s, w)
        st = s.stats()
    w.check(got)
    assert st["completed"] == len(w.req)
    assert st["misses"] == len(w.mats)
    assert st["hits"] == len(w.req) - len(w.mats)
    assert st["batched_decompositions"] >= 1  # the small misses of the first turn
    assert st["plain_decompositions"] >= 1
    assert st["solve_launches"] >= 1


def test_alone_equals_in_the_mix_equals_serial():
    w = Workload(60, seed=12)
    with gf2.Server(1 << 30, 2048, 2048, max_batch=64) as s:
        mixed = run(s, w)
    alone = {}
    with gf2.Server(1 << 30, 2048, 2048, max_batch=64) as s:
        for i in range(len(w.req)):
            w.X[i][:] = 0
            s.submit(w.req[i:i + 1])
            c = s.wait_all(1, timeout_s=120)
            assert c[0]["status"] == gf2.GF2_OK
            alone[i] = (int(c[0]["rank"]), int(c[0]["consistent"]), w.X[i].copy())
    with gf2.Server(1 << 30, 2048, 2048, serial=True) as s:
        serial = run(s, w)
    for i in range(len(w.req)):
        assert mixed[i][:2] == alone[i][:2] == serial[i][:2], i
        assert np.array_equal(mixed[i][2], alone[i][2]) and np.array_equal(mixed[i][2], serial[i][2]), i
    w.check(mixed)


def test_poisson_arrivals_overlap_and_match_oracle():
    w = Workload(120, seed=13)
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(40.0, size=len(w.req)))  # ~25k requests/s
    with gf2.Server(1 << 30, 2048, 2048, max_batch=32) as s:
        got = run(s, w, arrivals)
        st = s.stats()
    w.check(got)
    assert st["max_batch"] >= 1
    # continuous batching: requests were admitted while earlier launches of
    # the engine were on the GPU, and solve launches were enqueued while
    # others ran -- and every result still equals the oracle's (the same as
    # running the request alone)
    assert st["admitted_in_flight"] > 0, st
    assert st["overlapped_launches"] > 0, st


def test_a_request_the_arena_can_never_hold_fails_alone():
    """Factors larger than the whole factor arena (a 1 MiB budget): those
    requests complete with GF2_ERR_NOMEM, every other request is served and
    equals the oracle."""
    sizes = [(128, 128), (300, 256), (2000, 2000)]
    w = Workload(24, seed=15, sizes=sizes)
    big = 2  # key of the 2000 x 2000 matrix
    with gf2.Server(1 << 20, 2048, 2048, max_batch=16) as s:
        req = w.req.copy()
        for X in w.X:
            X[:] = 0
        s.submit(req)
        done = s.wait_all(len(req), timeout_s=300)
    exp = w.expected()
    seen = 0
    for c in done:
        i = int(c["id"])
        if int(w.req[i]["matrix"]) == big:
            assert c["status"] == gf2.GF2_ERR_NOMEM, (i, int(c["status"]))
            continue
        assert c["status"] == gf2.GF2_OK, (i, gf2.status_string(int(c["status"])))
        rank, cons, X = exp[i]
        assert int(c["rank"]) == rank and int(c["consistent"]) == cons and np.array_equal(w.X[i], X), i
        seen += 1
    assert seen > 0 and len(done) == len(w.req)


def test_eviction_under_a_small_budget():
    # 3 keys per size, factors of 70-260 KiB each; a 1 MiB budget (about
    # 320 KiB of it for the solves) holds two or three, so keys are evicted
    # and, as requests keep arriving (one every 300 us), rebuilt
    sizes = [(512, 512), (1024, 1024), (700, 900)]
    w = Workload(80, seed=14, sizes=sizes, keys_per_size=3)
    with gf2.Server(1 << 20, 1024, 1024, max_batch=16) as s:
        got = run(s, w, np.arange(len(w.req)) * 300.0)
        st = s.stats()
    w.check(got)
    assert st["evictions"] > 0
    assert st["misses"] > len(w.mats)  # rebuilt after eviction


def test_request_errors_complete_with_their_status():
    A = f2gen.uniform(100, 70, 3)
    Ah = gf2.host_colblocks(A, 70)
    B_bad = np.full(100, 0xFF, dtype=np.uint64)  # bits beyond nrhs = 4
    B_ok = np.zeros(100, dtype=np.uint64)
    X = np.zeros(70, dtype=np.uint64)
    big = gf2.host_colblocks(f2gen.uniform(300, 64, 4), 64)
    req = np.zeros(5, dtype=gf2.REQUEST_DTYPE)
    req[0] = (0, 1, 100, 70, Ah.data_ptr(), 100, 4, B_bad.ctypes.data, X.ctypes.data, 0.0)
    req[1] = (1, 1, 100, 70, Ah.data_ptr(), 100, 65, B_ok.ctypes.data, X.ctypes.data, 0.0)
    req[2] = (2, 2, 300, 64, big.data_ptr(), 300, 1, B_ok.ctypes.data, X.ctypes.data, 0.0)  # n > max_n
    req[3] = (3, 1, 100, 70, Ah.data_ptr(), 100, 0, 0, 0, 0.0)
    req[4] = (4, 1, 100, 64, Ah.data_ptr(), 100, 0, 0, 0, 0.0)  # key 1 with another size
    with gf2.Server(64 << 20, 256, 256) as s:
        s.submit(req[:4])
        first = {int(c["id"]): c for c in s.wait_all(4, timeout_s=60)}
        s.submit(req[4:])
        second = {int(c["id"]): c for c in s.wait_all(1, timeout_s=60)}
    assert first[0]["status"] == gf2.GF2_ERR_PADDING
    assert first[1]["status"] == gf2.GF2_ERR_SHAPE
    assert first[2]["status"] == gf2.GF2_ERR_UNSUPPORTED
    assert first[3]["status"] == gf2.GF2_OK and first[3]["rank"] == oracle.rank(A, 70)
    assert second[4]["status"] == gf2.GF2_ERR_SHAPE


def test_large_systems_by_cluster_match_oracle():
    """Systems of 4096 rows or more are solved by a cluster of CTAs (rows
    split across their shared memories): square, wide, tall and
    rank-deficient ones, alone and mixed with small systems in one launch."""
    sizes = [(4096, 4096), (4500, 4200), (6000, 4096), (4096, 4160), (300, 200), (64, 64)]
    w = Workload(16, seed=15, sizes=sizes)
    with gf2.Server(2 << 30, 8192, 8192, max_batch=64) as s:
        got = run(s, w)
    w.check(got)
    alone = {}
    with gf2.Server(2 << 30, 8192, 8192, max_batch=64) as s:
        for i in range(len(w.req)):
            w.X[i][:] = 0
            s.submit(w.req[i:i + 1])
            c = s.wait_all(1, timeout_s=120)
            assert c[0]["status"] == gf2.GF2_OK
            alone[i] = (int(c[0]["rank"]), int(c[0]["consistent"]), w.X[i].copy())
    for i in range(len(w.req)):
        assert got[i][:2] == alone[i][:2] and np.array_equal(got[i][2], alone[i][2]), i
