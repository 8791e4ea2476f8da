"""The factor handle (gf2_factors) and the per-call options (gf2_opts),
through the C ABI, bit for bit against the oracle: every option must give
the same factors (they are unique given the pivot rule, Lemma 4.1), and
calls with different options on different host threads must not disturb one
another."""
import threading

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


def cases():
    X, Y = f2gen.fixed_rank_factors(900, 1300, 333, 71)
    return [("square", f2gen.uniform(1024, 1024, f2gen.BASE_SEED, 0), 1024),
            ("tall", f2gen.uniform(1500, 700, 72), 700),
            ("wide", f2gen.uniform(700, 1500, 73), 1500),
            ("rank333", oracle.mmm(X, Y, 333, 1300), 1300),
            ("sparse", f2gen.sparse_rows(1200, 1200, 3, 74), 1200)]


def handle_factors(F: "gf2.Factors", stream=None) -> dict:
    """The handle's factors on the host.  With a stream, only that stream is
    synchronised: a device-wide synchronisation fails while another thread's
    decomposition captures its CUDA graph."""
    if stream is None:
        torch.cuda.synchronize()
    else:
        stream.synchronize()
    return dict(perm=F.perm.cpu().numpy(), pivcols=F.pivcols.cpu().numpy(), rank=F.rank(),
                L=F.L.to_rowmajor(), E=F.E.to_rowmajor())


@pytest.mark.parametrize("name", [c[0] for c in cases()])
def test_handle_decompose_solve_rref_nullspace(name):
    A, m = next((a, m) for nm, a, m in cases() if nm == name)
    n = A.shape[0]
    with gf2.Factors(n, m) as F:
        F.decompose(gf2.Mat.from_rowmajor(A, m, ld=n + 5))
        got = handle_factors(F)
        assert_same_decomposition(A, m, got)
        # solves with the handle
        B = f2gen.uniform(n, 17, 75).reshape(-1)
        sol = F.solve(gf2.Mat.from_rowmajor(B.reshape(-1, 1), 17))
        ref = oracle.solve(A, m, B, 17)
        assert sol["consistent"] == ref["consistent"]
        assert np.array_equal(sol["X"].to_rowmajor().reshape(-1), ref["X"])
        # the reduced form (E itself unchanged) and the null space
        R = F.rref().to_rowmajor()
        red = oracle.rref(A, m)
        assert np.array_equal(R[:red["rank"]], red["R"]) and not R[red["rank"]:].any()
        assert np.array_equal(F.E.to_rowmajor(), got["E"])
        N = F.nullspace()
        ref_n = oracle.nullspace(A, m)
        assert N.rows == m and N.cols == ref_n["nul"]
        if ref_n["nul"]:
            assert np.array_equal(N.to_rowmajor(), ref_n["N"])
        # a second decomposition into the same handle
        A2 = f2gen.uniform(n, m, 76)
        F.decompose(gf2.Mat.from_rowmajor(A2, m))
        assert_same_decomposition(A2, m, handle_factors(F))


def test_rank_only_handle():
    A = f2gen.uniform(2000, 900, 77)
    with gf2.Factors(2000, 900, rank_only=True) as F:
        F.decompose(gf2.Mat.from_rowmajor(A, 900))
        assert F.L is None and F.E is None
        assert F.rank() == oracle.rank(A, 900, nthreads=NT)
        torch.cuda.synchronize()
        ref = oracle.ple(A, 900, want_L=False, want_E=False)
        assert np.array_equal(F.perm.cpu().numpy(), ref["perm"])
        with pytest.raises(gf2.Gf2Error) as e:
            F.solve(gf2.Mat.from_rowmajor(np.zeros((2000, 1), dtype=np.uint64), 1))
        assert e.value.status == gf2.GF2_ERR_ARG


def test_handle_rejects_another_size():
    with gf2.Factors(100, 100) as F:
        with pytest.raises(gf2.Gf2Error) as e:
            F.decompose(gf2.Mat.from_rowmajor(f2gen.uniform(100, 99, 78), 99))
        assert e.value.status == gf2.GF2_ERR_SHAPE


OPTION_GRID = [gf2.Opts(panel_w=w, table_c=c) for w in (0, 64, 128) for c in (0, 4, 8)]


@pytest.mark.parametrize("o", OPTION_GRID, ids=lambda o: f"w{o.panel_w}-c{o.table_c}")
@pytest.mark.parametrize("n,m", [(2048, 2048), (3000, 1111), (777, 2500), (6000, 640)])
def test_decompose_options_give_the_same_factors(o, n, m):
    A = f2gen.uniform(n, m, 79, n, m)
    k = min(n, m)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    piv = torch.empty(k, dtype=torch.int32, device="cuda")
    rank = torch.zeros(1, dtype=torch.int64, device="cuda")
    L, E = gf2.Mat.empty(n, k), gf2.Mat.empty(k, m)
    gf2.gf2_decompose_ex(gf2.Mat.from_rowmajor(A, m), perm, piv, rank, L, E, o)
    torch.cuda.synchronize()
    got = dict(perm=perm.cpu().numpy(), pivcols=piv.cpu().numpy(), rank=int(rank.item()), L=L.to_rowmajor(),
               E=E.to_rowmajor())
    assert_same_decomposition(A, m, got)
    assert gf2.gf2_rank_ex(gf2.Mat.from_rowmajor(A, m), o) == got["rank"]


def test_two_threads_with_different_options():
    """Two host threads, each on its own stream and handle, decompose and
    multiply with different options at the same time; every result matches
    the oracle."""
    jobs = [(f2gen.uniform(3000, 3000, 80), 3000, gf2.Opts(panel_w=64, table_c=4),
             gf2.Opts(backend=gf2.BACKEND_AUTO, strassen_cutoff=256)),
            (f2gen.uniform(2800, 3100, 81), 3100, gf2.Opts(panel_w=128, table_c=8),
             gf2.Opts(backend=gf2.BACKEND_TABLES))]
    P = f2gen.uniform(1024, 1024, 82)
    Q = f2gen.uniform(1024, 1024, 83)
    PQ = oracle.mmm(P, Q, 1024, 1024, nthreads=NT)
    refs = [oracle.ple(A, m, nthreads=NT) for A, m, _, _ in jobs]
    errors = []

    def work(i):
        try:
            A, m, dopt, mopt = jobs[i]
            n = A.shape[0]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s), gf2.Factors(n, m) as F:
                Ad = gf2.Mat.from_rowmajor(A, m)
                Pd, Qd = gf2.Mat.from_rowmajor(P, 1024), gf2.Mat.from_rowmajor(Q, 1024)
                for _ in range(4):
                    F.decompose(Ad, dopt, stream=s)
                    C = gf2.Mat.empty(1024, 1024)
                    gf2.gf2_mmm_ex(Pd, Qd, C, mopt, stream=s)
                    s.synchronize()
                    got = handle_factors(F, s)
                    ref = refs[i]
                    assert got["rank"] == ref["rank"]
                    assert np.array_equal(got["perm"], ref["perm"])
                    assert np.array_equal(got["L"], ref["L"]) and np.array_equal(got["E"], ref["E"])
                    assert np.array_equal(C.to_rowmajor(), PQ)
        except Exception as e:  # reported by the main thread
            errors.append((i, repr(e)))

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors


@pytest.mark.parametrize("o", [gf2.Opts(backend=b, strassen_cutoff=c)
                               for b, c in ((0, 128), (0, gf2.STRASSEN_OFF), (1, 0), (2, 0))],
                         ids=lambda o: f"b{o.backend}-cut{o.strassen_cutoff}")
def test_product_options(o):
    n, k, m = 1024, 2048, 1000
    A = f2gen.uniform(n, k, 84)
    B = f2gen.uniform(k, m, 85)
    C = gf2.Mat.empty(n, m)
    gf2.gf2_mmm_ex(gf2.Mat.from_rowmajor(A, k), gf2.Mat.from_rowmajor(B, m), C, o)
    assert np.array_equal(C.to_rowmajor(), oracle.mmm(A, B, k, m, nthreads=NT))


@pytest.mark.parametrize("c8_from", [64, 1 << 62])
def test_batched_table_size_option(c8_from):
    """Every matrix on the 8-bit (c8_from = 64) or on the 4-bit kernel by a
    per-call option; the process-wide setting is left alone."""
    import ctypes
    before = gf2.batched_c8_from()
    mats = [(f2gen.uniform(n, m, 86, n, m), m) for n, m in ((100, 200), (700, 650), (64, 64), (1500, 900))]
    As = [gf2.Mat.from_rowmajor(a, m) for a, m in mats]
    lib = gf2.load()
    count = len(As)
    perms = [torch.empty(a.rows, dtype=torch.int32, device="cuda") for a in As]
    pivs = [torch.empty(min(a.rows, a.cols), dtype=torch.int32, device="cuda") for a in As]
    ranks = torch.zeros(count, dtype=torch.int64, device="cuda")
    Ls = [gf2.Mat.empty(a.rows, min(a.rows, a.cols)) for a in As]
    Es = [gf2.Mat.empty(min(a.rows, a.cols), a.cols) for a in As]
    o = gf2.Opts(batched_c8_from=c8_from)
    ns = (ctypes.c_int64 * count)(*[a.rows for a in As])
    ms = (ctypes.c_int64 * count)(*[a.cols for a in As])
    wsb = lib.gf2_decompose_batched_workspace_bytes_ex(count, ns, ms, 1, ctypes.byref(o))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    st = lib.gf2_decompose_batched_ex(count, (gf2._CMat * count)(*[a.c() for a in As]),
                                      (ctypes.c_void_p * count)(*[p.data_ptr() for p in perms]),
                                      (ctypes.c_void_p * count)(*[p.data_ptr() for p in pivs]), ranks.data_ptr(),
                                      (gf2._CMat * count)(*[x.c() for x in Ls]),
                                      (gf2._CMat * count)(*[x.c() for x in Es]), 0, ctypes.byref(o), ws.data_ptr(),
                                      wsb, torch.cuda.current_stream().cuda_stream)
    assert st == gf2.GF2_OK
    torch.cuda.synchronize()
    for i, (a, m) in enumerate(mats):
        got = dict(perm=perms[i].cpu().numpy(), pivcols=pivs[i].cpu().numpy(), rank=int(ranks[i].item()),
                   L=Ls[i].to_rowmajor(), E=Es[i].to_rowmajor())
        assert_same_decomposition(a, m, got)
    assert gf2.batched_c8_from() == before
