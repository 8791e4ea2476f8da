"""The C-ABI library loads and exports every entry point include/gf2.h
declares; host-only entry points answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf2.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gf2_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1209_5198_gb300 import _build
    _build.build()
    import paper_1209_5198_gb300 as g
    return g.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in gf2.h but not exported"


def test_host_only_entry_points(lib):
    assert lib.gf2_version() >= 1
    assert b"padding" in lib.gf2_status_string(3)
    assert lib.gf2_status_string(999) == b"unknown status"
    n = m = 32768
    ws = lib.gf2_decompose_workspace_bytes(n, m, 1)
    assert ws >= 3 * n * (m // 64) * 8  # working copy + L + E, row-major
    assert lib.gf2_decompose_workspace_bytes(n, m, 0) < ws
    assert lib.gf2_rank_workspace_bytes(n, m) >= lib.gf2_decompose_workspace_bytes(n, m, 0)
    # the product: M4RM needs only a status word; the tensor path the byte
    # expansions of A and B; the recursion one level's temporaries per level
    assert 0 < lib.gf2_mmm_workspace_bytes(1000, 2000, 3000, 0) <= 4096
    # tensor backend: both operands expanded to e2m1 entries, two per byte
    assert lib.gf2_mmm_workspace_bytes(1000, 2000, 3000, 4) >= (1024 * 2048 + 3072 * 2048) // 2
    import paper_1209_5198_gb300 as g
    old = g.strassen_cutoff()
    try:
        g.set_strassen_cutoff(2048)
        d = 4096  # one level: S1..S4 (2048 x 32 words), T1..T4 (2048 x 32), X (2048 x 32)
        assert lib.gf2_mmm_workspace_bytes(d, d, d, 0) >= 8 * 9 * 2048 * 32
        assert lib.gf2_mmm_workspace_bytes(d, d, d, 2) <= 4096      # GF2_MMM_TABLES: no recursion
        assert lib.gf2_mmm_workspace_bytes(d, d + 64, d, 0) <= 4096  # odd number of words in k
    finally:
        g.set_strassen_cutoff(old)
    assert lib.gf2_decompose_workspace_bytes(-1, 5, 0) == 0


def test_argument_errors_without_gpu(lib):
    import paper_1209_5198_gb300 as g
    # null matrix descriptor / outputs: rejected before any CUDA call
    assert lib.gf2_decompose(None, None, None, None, None, None, 0, None, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_mmm(None, None, None, 0, 0, None, 0, None) == g.GF2_ERR_ARG
    a = g._CMat(None, 10, 10, 5)  # ld < rows
    assert lib.gf2_mmm(ctypes.byref(a), ctypes.byref(a), ctypes.byref(a), 0, 0, None, 0, None) == g.GF2_ERR_ARG
    b = g._CMat(1, 10, 20, 10)
    c = g._CMat(2, 10, 20, 10)
    d = g._CMat(3, 30, 20, 30)
    # inner dimensions differ (A is 10 x 20, B is 10 x 20)
    assert lib.gf2_mmm(ctypes.byref(b), ctypes.byref(c), ctypes.byref(d), 0, 0, None, 0, None) == g.GF2_ERR_SHAPE
    # unknown flag
    assert lib.gf2_decompose(ctypes.byref(b), ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                             None, None, 0x80, None, 0, None) == g.GF2_ERR_ARG


def test_solve_argument_errors_without_gpu(lib):
    import paper_1209_5198_gb300 as g
    P = ctypes.c_void_p(8)
    L = g._CMat(1, 10, 10, 10)
    E = g._CMat(2, 10, 10, 10)
    B = g._CMat(3, 10, 64, 10)
    X = g._CMat(4, 10, 64, 10)
    args = lambda b, x: (ctypes.byref(L), ctypes.byref(E), P, P, P, ctypes.byref(b), ctypes.byref(x), P, 0, None, 0, None)
    assert lib.gf2_solve(None, None, None, None, None, None, None, None, 0, None, 0, None) == g.GF2_ERR_ARG
    B65 = g._CMat(3, 10, 65, 10)
    X65 = g._CMat(4, 10, 65, 10)
    assert lib.gf2_solve(*args(B65, X65)) == g.GF2_ERR_SHAPE       # more than 64 right-hand sides
    X3 = g._CMat(4, 10, 3, 10)
    assert lib.gf2_solve(*args(B, X3)) == g.GF2_ERR_SHAPE          # X has other columns than B
    X12 = g._CMat(4, 12, 64, 12)
    assert lib.gf2_solve(*args(B, X12)) == g.GF2_ERR_SHAPE         # E is not min(n,m) x m
    assert lib.gf2_solve_workspace_bytes(-1, 5) == 0
    assert lib.gf2_solve_workspace_bytes(32768, 32768) >= 8 * (32768 + 32768 + 2 * 512 * 64)


def test_serving_records_match_the_c_layout(tmp_path):
    """The numpy record types of the binding have the C structs' sizes and
    field offsets (a C program built against include/gf2.h prints them)."""
    import shutil
    import subprocess

    import paper_1209_5198_gb300 as g
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    fields_req = [f for f in g.REQUEST_DTYPE.names]
    fields_done = [f for f in g.COMPLETION_DTYPE.names]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gf2.h"', "int main(void) {",
             '  printf("req %zu\\n", sizeof(gf2_request));',
             '  printf("done %zu\\n", sizeof(gf2_completion));',
             '  printf("stats %zu\\n", sizeof(gf2_server_stats));']
    lines += [f'  printf("req.{f} %zu\\n", offsetof(gf2_request, {f}));' for f in fields_req]
    lines += [f'  printf("done.{f} %zu\\n", offsetof(gf2_completion, {f}));' for f in fields_done]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(got["req"]) == g.REQUEST_DTYPE.itemsize
    assert int(got["done"]) == g.COMPLETION_DTYPE.itemsize
    assert int(got["stats"]) == 8 * len(g.STATS_FIELDS)
    for f in fields_req:
        assert int(got[f"req.{f}"]) == g.REQUEST_DTYPE.fields[f][1], f
    for f in fields_done:
        assert int(got[f"done.{f}"]) == g.COMPLETION_DTYPE.fields[f][1], f


def test_server_argument_errors_without_gpu(lib):
    import paper_1209_5198_gb300 as g
    h = ctypes.c_void_p()
    assert lib.gf2_server_create(0, 16, 16, 8, 0, ctypes.byref(h)) == g.GF2_ERR_ARG
    assert lib.gf2_server_create(1 << 20, 0, 16, 8, 0, ctypes.byref(h)) == g.GF2_ERR_ARG
    assert lib.gf2_server_create(1 << 20, 16, 16, 0, 0, ctypes.byref(h)) == g.GF2_ERR_ARG
    assert lib.gf2_server_create(1 << 20, 16, 16, 8, 0x10, ctypes.byref(h)) == g.GF2_ERR_ARG
    assert lib.gf2_server_create(1 << 20, 16, 16, 8, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_server_submit(None, None, 0) == g.GF2_ERR_ARG
    cnt = ctypes.c_int(0)
    assert lib.gf2_server_poll(None, None, 0, 0, ctypes.byref(cnt)) == g.GF2_ERR_ARG
    assert lib.gf2_server_destroy(None) == g.GF2_ERR_ARG


def test_host_entry_point_checks_padding_on_the_host(lib):
    """gf2_decompose_host reads the padding bits of its host input before any
    device work: a bit beyond the last column is reported without a GPU."""
    import numpy as np
    import paper_1209_5198_gb300 as g
    n, m = 10, 70  # two column blocks, 6 columns used in the second
    A = np.zeros((2, n), dtype=np.uint64)
    A[1, 3] = np.uint64(1) << np.uint64(40)  # column 104 >= 70
    perm = np.zeros(n, dtype=np.int32)
    rank = np.zeros(1, dtype=np.int64)
    lib.gf2_decompose_host.restype = ctypes.c_int
    st = lib.gf2_decompose_host(ctypes.c_int64(n), ctypes.c_int64(m), A.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(n),
                                perm.ctypes.data_as(ctypes.c_void_p), None, rank.ctypes.data_as(ctypes.c_void_p),
                                None, None, ctypes.c_uint(0), None, ctypes.c_size_t(0), None)
    assert st == g.GF2_ERR_PADDING


def test_reduced_form_null_space_and_rank_workspaces_without_gpu(lib):
    """Workspace queries and argument checks of gf2_rref, gf2_nullspace,
    gf2_rank's transposed route and gf2_op_counts answer on the host."""
    S = ctypes.c_size_t
    lib.gf2_rref_workspace_bytes.restype = S
    lib.gf2_nullspace_workspace_bytes.restype = S
    lib.gf2_rank_workspace_bytes.restype = S
    lib.gf2_decompose_workspace_bytes.restype = S
    I64 = ctypes.c_int64
    lib.gf2_rref_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_nullspace_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_rank_workspace_bytes.argtypes = [I64, I64]
    lib.gf2_decompose_workspace_bytes.argtypes = [I64, I64, ctypes.c_int]
    # RREF: 64 words per 64-row block plus the top level's gathered operand
    k = m = 32768
    assert lib.gf2_rref_workspace_bytes(k, m) >= k * 8 + (k // 2) * (k // 2 // 64) * 8
    assert lib.gf2_rref_workspace_bytes(-1, 3) == 0
    assert lib.gf2_rref_workspace_bytes(64, 100) > 0  # one block: no product
    # null space: one int32 per free column
    assert lib.gf2_nullspace_workspace_bytes(1000, 300) >= 700 * 4
    assert lib.gf2_nullspace_workspace_bytes(10, 11) == 0  # rank > m
    # rank: a wide matrix holds its transpose on top of the decomposition's workspace
    wide = lib.gf2_rank_workspace_bytes(1000, 5000)
    assert wide >= ((1000 + 63) // 64) * 5000 * 8 + lib.gf2_decompose_workspace_bytes(5000, 1000, 0)
    assert lib.gf2_rank_workspace_bytes(5000, 1000) >= lib.gf2_decompose_workspace_bytes(5000, 1000, 0)
    # argument errors before any device work
    assert lib.gf2_rref(None, None, None, S(0), None) == 1  # GF2_ERR_ARG
    assert lib.gf2_nullspace(None, None, I64(0), None, None, S(0), None) == 1
    out = (ctypes.c_uint64 * 9)()
    assert lib.gf2_op_counts(None, 9, 0) == 1
    assert lib.gf2_op_counts(out, -1, 0) == 1
    assert lib.gf2_op_counts(out, 9, 0) == 7  # GF2_ERR_UNSUPPORTED: the release build counts nothing


def test_options_and_factor_structs_match_the_c_layout(tmp_path):
    """gf2_opts and gf2_factors of the binding have the C structs' sizes and
    field offsets."""
    import shutil
    import subprocess

    import paper_1209_5198_gb300 as g
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"gf2_opts": g.Opts, "gf2_factors": g._CFactors}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gf2.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        lines += [f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));' for f, _ in py._fields_]
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout2.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout2"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_options_are_validated_without_gpu(lib):
    """gf2_opts_check and every _ex entry point reject bad options before any
    device work (so these run without a GPU)."""
    import paper_1209_5198_gb300 as g
    ok = g.Opts()
    assert g.opts_check(None) == g.GF2_OK
    assert g.opts_check(ok) == g.GF2_OK
    good = [dict(panel_w=64), dict(panel_w=128), dict(table_c=4), dict(table_c=8), dict(tile_words=4),
            dict(backend=g.BACKEND_TABLES), dict(backend=g.BACKEND_TENSOR), dict(strassen_cutoff=128),
            dict(strassen_cutoff=g.STRASSEN_OFF), dict(batched_c8_from=512),
            dict(schedule=g.SCHEDULE_STREAMS), dict(schedule=g.SCHEDULE_PERSISTENT), dict(schedule=g.SCHEDULE_SPLIT),
            dict(panel_w=64, table_c=4, tile_words=4, backend=1, strassen_cutoff=4096, batched_c8_from=1)]
    bad_arg = [dict(panel_w=-64), dict(panel_w=96), dict(table_c=-1), dict(table_c=17), dict(tile_words=-4),
               dict(backend=3), dict(backend=-1), dict(strassen_cutoff=-1), dict(strassen_cutoff=127),
               dict(batched_c8_from=-5), dict(schedule=4), dict(schedule=-1), dict(reserved=1)]
    unsupported = [dict(panel_w=192), dict(panel_w=256), dict(table_c=6), dict(table_c=16), dict(tile_words=2),
                   dict(tile_words=8)]
    for kw in good:
        assert g.opts_check(g.Opts(**kw)) == g.GF2_OK, kw
    for kw in bad_arg:
        assert g.opts_check(g.Opts(**kw)) == g.GF2_ERR_ARG, kw
    for kw in unsupported:
        assert g.opts_check(g.Opts(**kw)) == g.GF2_ERR_UNSUPPORTED, kw
    # the _ex entry points return the same status before touching the device
    bad = ctypes.byref(g.Opts(panel_w=96))
    a = g._CMat(1, 64, 64, 64)  # (never dereferenced)
    assert lib.gf2_decompose_ex(ctypes.byref(a), None, None, None, None, None, 0, bad, None, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_rank_ex(ctypes.byref(a), ctypes.byref(ctypes.c_int64()), 0, bad, None, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_mmm_ex(ctypes.byref(a), ctypes.byref(a), ctypes.byref(a), 0, 0, bad, None, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_decompose_batched_ex(1, ctypes.byref(a), None, None, None, None, None, 0,
                                        ctypes.byref(g.Opts(tile_words=8)), None, 0, None) == g.GF2_ERR_UNSUPPORTED
    assert lib.gf2_mmm_workspace_bytes_ex(64, 64, 64, 0, bad) == 0
    # a backend flag and a backend option together
    both = ctypes.byref(g.Opts(backend=g.BACKEND_TENSOR))
    assert lib.gf2_mmm_ex(ctypes.byref(a), ctypes.byref(a), ctypes.byref(a), 0, g.GF2_MMM_TABLES, both, None, 0,
                          None) == g.GF2_ERR_ARG


def test_factor_handle_argument_errors_without_gpu(lib):
    """gf2_factors_* reject bad arguments before any allocation, and a zeroed
    handle frees as a no-op."""
    import paper_1209_5198_gb300 as g
    F = g._CFactors()
    assert lib.gf2_factors_alloc(None, 4, 4, 0) == g.GF2_ERR_ARG
    assert lib.gf2_factors_alloc(ctypes.byref(F), -1, 4, 0) == g.GF2_ERR_ARG
    assert lib.gf2_factors_alloc(ctypes.byref(F), 4, -1, 0) == g.GF2_ERR_ARG
    assert lib.gf2_factors_alloc(ctypes.byref(F), 4, 4, 8) == g.GF2_ERR_ARG
    assert lib.gf2_factors_alloc(ctypes.byref(F), 1 << 31, 4, 0) == g.GF2_ERR_UNSUPPORTED
    assert lib.gf2_factors_free(None) == g.GF2_ERR_ARG
    assert lib.gf2_factors_free(ctypes.byref(F)) == g.GF2_OK  # zeroed: nothing to free
    a = g._CMat(None, 4, 4, 4)
    r = ctypes.c_int64()
    assert lib.gf2_factors_decompose(ctypes.byref(F), ctypes.byref(a), 0, None, None) == g.GF2_ERR_ARG
    assert lib.gf2_factors_rank(ctypes.byref(F), ctypes.byref(r), None) == g.GF2_ERR_ARG
    assert lib.gf2_factors_solve(ctypes.byref(F), ctypes.byref(a), ctypes.byref(a), None, 0, None) == g.GF2_ERR_ARG
    assert lib.gf2_factors_rref(ctypes.byref(F), ctypes.byref(a), None) == g.GF2_ERR_ARG
    assert lib.gf2_factors_nullspace(ctypes.byref(F), ctypes.byref(a), None) == g.GF2_ERR_ARG
