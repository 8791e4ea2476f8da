"""Pins of the plain CPU oracle against facts fixed outside of it.

Every oracle function is checked here against something other than itself:
the paper's worked examples (tests/golden), brute-force enumeration on all
tiny matrices, exact reconstruction by numpy integer products, the
invariants of the factors, ranks known by construction, a textbook closed
form (rank distribution of random square matrices), and agreement of two
independent routes through the decomposition (bit-level elimination vs the
block algorithm with Procedure buildZ).
"""
import itertools
import os

import numpy as np
import pytest

import f2gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits_of(words, cols):
    return f2gen.unpack_bits(words, cols).astype(np.int64)


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([int(v) for v in vals])
    return out


# ------------------------------------------------------------ brute force

def span_size(rows_int):
    """Number of distinct XOR combinations of the given row integers."""
    span = {0}
    for r in rows_int:
        span |= {s ^ r for s in span}
    return len(span)


def brute_rank(bits):
    rows = [int("".join(str(int(b)) for b in row[::-1]) or "0", 2) for row in bits]
    return int(np.log2(span_size(rows)))


def brute_profile(bits):
    n, m = bits.shape
    prof, prev = [], 0
    for j in range(m):
        r = brute_rank(bits[:, : j + 1])
        if r > prev:
            prof.append(j)
        prev = r
    return prof


def check_ple_invariants(Abits, out):
    n, m = Abits.shape
    r = out["rank"]
    perm = np.asarray(out["perm"])
    assert sorted(perm.tolist()) == list(range(n)), "perm is not a permutation"
    piv = np.asarray(out["pivcols"])
    assert len(piv) == r
    assert np.all(np.diff(piv) > 0), "pivot columns not increasing"
    kmax = min(n, m)
    L = bits_of(out["L"], kmax)[:, :r] if kmax else np.zeros((n, 0), dtype=np.int64)
    E = bits_of(out["E"], m)[:r] if kmax else np.zeros((0, m), dtype=np.int64)
    # L: unit lower trapezoidal
    for t in range(r):
        assert L[t, t] == 1
        assert not L[:t, t].any(), "L not lower triangular"
    # E: echelon with leading ones at the pivot columns
    for t in range(r):
        nz = np.nonzero(E[t])[0]
        assert nz.size and nz[0] == piv[t], "E row does not lead at its pivot column"
    # unused columns / rows of the outputs are zero
    assert not bits_of(out["L"], kmax)[:, r:].any() if kmax else True
    assert not bits_of(out["E"], m)[r:].any() if kmax else True
    # reconstruction, exactly, by an integer product mod 2
    assert np.array_equal((L @ E) % 2, Abits[perm]), "P*A != L*E"


# ------------------------------------------------------------ golden data

def test_packing_example():
    g = read_golden("packing_example.txt")
    b = g["b"][0][0]
    bits = np.array(g["row"], dtype=np.uint8)
    words = f2gen.pack_bits(bits, b)
    assert words.tolist() == g["words"]
    assert f2gen.colmajor_flat(words) == g["colmajor"][0]
    assert np.array_equal(f2gen.unpack_bits(words, bits.shape[1], b), bits)


def test_jr_example_and_pseudo_inverse():
    g = read_golden("jr_example.txt")
    J = np.array(g["J"])
    R = np.array(g["R"])
    assert np.array_equal(J.T @ J % 2, np.eye(2, dtype=int))
    assert not (J.T @ R % 2).any()
    # A 3-row panel whose first two rows have pivot bits {0, 2} (column 1 is
    # column 0 repeated) and whose third row is their sum: the block route
    # must find the same pivots and store Y = D Z = (1, 1) below them.
    B = np.array([[1, 1, 0], [0, 0, 1]])
    D = (B[0] + B[1]) % 2
    A = np.vstack([B, D])
    out = oracle.blockdecomp(f2gen.pack_bits(A), 3, 3)
    assert out["pivcols"].tolist() == g["pivots"][0]
    assert out["rank"] == g["r"][0][0]
    assert int(out["Wb"][0, 2]) == 0b11
    # the completed square block J B + R is non-singular and Z = (JB+R)^-1 J
    # satisfies B Z = I (eq. pre:W)
    JBR = (J @ B + R) % 2
    det = round(np.linalg.det(JBR)) % 2
    assert det == 1


# ------------------------------------------------------------ exhaustive

@pytest.mark.parametrize("n,m", [(1, 1), (2, 3), (3, 2), (3, 3), (3, 4), (4, 3), (4, 4)])
def test_exhaustive_tiny(n, m):
    """Every n x m matrix: rank, column rank profile, null-space size, P*A=L*E."""
    for code in range(1 << (n * m)):
        bits = np.array([(code >> k) & 1 for k in range(n * m)], dtype=np.int64).reshape(n, m)
        out = oracle.ple(f2gen.pack_bits(bits), m)
        r = out["rank"]
        assert r == brute_rank(bits)
        assert out["pivcols"].tolist() == brute_profile(bits)
        check_ple_invariants(bits, out)
        if code % 7 == 0:  # null-space count 2^(m-r), by enumerating all x
            zero = sum(1 for x in itertools.product((0, 1), repeat=m) if not ((bits @ np.array(x)) % 2).any())
            assert zero == 1 << (m - r)


def test_all_5x5_sampled_rank():
    rng = np.random.default_rng(5)
    for code in rng.integers(0, 1 << 25, size=3000):
        bits = np.array([(int(code) >> k) & 1 for k in range(25)], dtype=np.int64).reshape(5, 5)
        out = oracle.ple(f2gen.pack_bits(bits), 5)
        assert out["rank"] == brute_rank(bits)
        assert out["pivcols"].tolist() == brute_profile(bits)


@pytest.mark.parametrize("seed", range(40))
def test_random_small_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 9)), int(rng.integers(1, 13))
    p = [0.5, 0.2, 0.8][seed % 3]
    bits = (rng.random((n, m)) < p).astype(np.int64)
    out = oracle.ple(f2gen.pack_bits(bits), m)
    assert out["rank"] == brute_rank(bits)
    assert out["pivcols"].tolist() == brute_profile(bits)
    check_ple_invariants(bits, out)


# ------------------------------------------------------------ larger shapes

def matrices():
    """(name, row-major words, cols) covering dense, deficient, sparse, edge cases."""
    yield "uniform-130x200", f2gen.uniform(130, 200, 1), 200
    yield "uniform-200x130", f2gen.uniform(200, 130, 2), 130
    yield "uniform-64x64", f2gen.uniform(64, 64, 3), 64
    yield "bernoulli0.1-150x150", f2gen.bernoulli(150, 150, 0.1, 4), 150
    yield "sparse3-120x150", f2gen.sparse_rows(120, 150, 3, 5), 150
    X, Y = f2gen.fixed_rank_factors(150, 170, 37, 6)
    yield "rank37-150x170", oracle.mmm(X, Y, 37, 170), 170
    yield "zero-70x90", np.zeros((70, 2), dtype=np.uint64), 90
    eye = np.zeros((90, 2), dtype=np.uint64)
    for i in range(90):
        eye[i, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    yield "identity-90", eye, 90
    r1 = np.zeros((77, 2), dtype=np.uint64)
    r1[::3] = f2gen.uniform(1, 100, 7)
    yield "rank1-77x100", r1, 100
    dup = f2gen.uniform(40, 100, 8)
    yield "dup-rows-80x100", np.vstack([dup, dup]), 100
    yield "one-row", f2gen.uniform(1, 150, 9), 150
    yield "one-col", f2gen.uniform(150, 1, 10), 1


@pytest.mark.parametrize("name,A,m", list(matrices()), ids=[x[0] for x in matrices()])
def test_ple_invariants_and_two_routes(name, A, m):
    bits = bits_of(A, m)
    out = oracle.ple(A, m)
    check_ple_invariants(bits, out)
    rr = oracle.rref(A, m)
    assert rr["rank"] == out["rank"]
    assert np.array_equal(rr["pivcols"], out["pivcols"])
    # the row space of E is the row space of A: same reduced form
    rE = oracle.rref(out["E"][: out["rank"]], m) if out["rank"] else {"R": rr["R"][:0]}
    assert np.array_equal(rE["R"], rr["R"])
    # the paper's block algorithm (Procedure buildZ) at several word sizes
    # picks exactly the same rows in the same order
    for b in (1, 3, 8, 32, 64):
        blk = oracle.blockdecomp(A, m, b)
        assert blk["rank"] == out["rank"], b
        assert np.array_equal(blk["perm"], out["perm"]), b
        assert np.array_equal(blk["pivcols"], out["pivcols"]), b
        assert sum(blk["rblock"]) == out["rank"]
        check_figure1_storage(bits, blk, b)


def check_figure1_storage(Abits, blk, b):
    """P*A = L_b * U_b for the in-place storage of Figure 1 (block form)."""
    n, m = Abits.shape
    mub = (m + b - 1) // b
    Wb = blk["Wb"]
    r = blk["rank"]
    Lb = np.zeros((n, r), dtype=np.int64)
    Ub = np.zeros((r, m), dtype=np.int64)
    R = 0
    for j in range(mub):
        rj = int(blk["rblock"][j])
        for s in range(rj):
            Lb[R + s, R + s] = 1
            for q in range(j, mub):
                w = int(Wb[q, R + s])
                for t in range(b):
                    c = q * b + t
                    if c < m and (w >> t) & 1:
                        Ub[R + s, c] = 1
        for i in range(R + rj, n):
            y = int(Wb[j, i])
            for s in range(rj):
                if (y >> s) & 1:
                    Lb[i, R + s] = 1
        R += rj
    assert np.array_equal((Lb @ Ub) % 2, Abits[blk["perm"]])


# ------------------------------------------------------------ known ranks

@pytest.mark.parametrize("n,m,r", [(100, 120, 50), (120, 100, 100), (256, 256, 192), (200, 300, 1), (64, 64, 0)])
def test_fixed_rank_products(n, m, r):
    X, Y = f2gen.fixed_rank_factors(n, m, r, 11)
    A = oracle.mmm(X, Y, r, m)
    ref = (bits_of(X, r) @ bits_of(Y, m)) % 2 if r else np.zeros((n, m), dtype=np.int64)
    assert np.array_equal(bits_of(A, m), ref)
    assert oracle.rank(X, r) == r
    assert oracle.rank(Y, m) == r
    out = oracle.ple(A, m)
    assert out["rank"] == r
    check_ple_invariants(ref, out)
    # the pivot columns of X*Y are those of Y (X has full column rank)
    assert np.array_equal(out["pivcols"], oracle.ple(Y, m)["pivcols"])


def test_rank_distribution_of_random_square():
    """Corank of a uniform n x n matrix over F2 tends to
    2^(-d^2) prod_{i>d}(1-2^-i) / prod_{i<=d}(1-2^-i): 0.2888, 0.5776, 0.1284."""
    N, n = 6000, 64
    ranks = np.array([oracle.rank(f2gen.uniform(n, n, 1000, s), n) for s in range(N)])
    inf = np.prod([1 - 2.0 ** -i for i in range(1, 200)])
    for d in range(3):
        head = np.prod([1 - 2.0 ** -i for i in range(1, d + 1)])
        p = 2.0 ** (-d * d) * inf / head ** 2
        frac = np.mean(ranks == n - d)
        sigma = np.sqrt(p * (1 - p) / N)
        assert abs(frac - p) < 5 * sigma, (d, frac, p)
    assert np.all(ranks >= n - 5)


# ------------------------------------------------------------ product

@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (5, 70, 3), (64, 64, 64), (100, 130, 65), (33, 1, 200)])
def test_mmm_against_integer_product(n, k, m):
    A = f2gen.uniform(n, k, 21)
    B = f2gen.uniform(k, m, 22)
    C = oracle.mmm(A, B, k, m)
    ref = (bits_of(A, k) @ bits_of(B, m)) % 2
    assert np.array_equal(bits_of(C, m), ref)
    C0 = f2gen.uniform(n, m, 23)
    Cacc = oracle.mmm(A, B, k, m, C=C0)
    assert np.array_equal(bits_of(Cacc, m), (ref + bits_of(C0, m)) % 2)


def test_mmm_identities():
    n = 300
    A, B, C = (f2gen.uniform(n, n, s) for s in (31, 32, 33))
    ab_c = oracle.mmm(oracle.mmm(A, B, n, n), C, n, n)
    a_bc = oracle.mmm(A, oracle.mmm(B, C, n, n), n, n)
    assert np.array_equal(ab_c, a_bc)
    eye = f2gen.pack_bits(np.eye(n, dtype=np.uint8))
    assert np.array_equal(oracle.mmm(A, eye, n, n), A)
    assert np.array_equal(oracle.mmm(eye, A, n, n), A)


# ------------------------------------------------------------ solve / rref

@pytest.mark.parametrize("seed", range(12))
def test_solve_against_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    n, m, k = int(rng.integers(1, 7)), int(rng.integers(1, 9)), int(rng.integers(1, 6))
    bits = (rng.random((n, m)) < 0.5).astype(np.int64)
    if seed % 3 == 0 and n > 1:
        bits[-1] = bits[0]  # force a dependent row
    B = rng.integers(0, 2, size=(n, k))
    Bw = f2gen.pack_bits(B).reshape(-1)
    out = oracle.solve(f2gen.pack_bits(bits), m, Bw, k)
    piv = brute_profile(bits)
    X = f2gen.unpack_bits(out["X"].reshape(-1, 1), k)
    for c in range(k):
        sols = [np.array(x) for x in itertools.product((0, 1), repeat=m)
                if np.array_equal((bits @ np.array(x)) % 2, B[:, c])]
        consistent = (out["consistent"] >> c) & 1
        assert consistent == (1 if sols else 0)
        if sols:
            # the unique solution that is zero on every non-pivot column
            cand = [x for x in sols if not any(x[j] for j in range(m) if j not in piv)]
            assert len(cand) == 1
            assert np.array_equal(X[:, c], cand[0])
        else:
            assert not X[:, c].any()


def test_solve_consistent_rhs_larger():
    n, m, k = 150, 170, 64
    X, Y = f2gen.fixed_rank_factors(n, m, 90, 41)
    A = oracle.mmm(X, Y, 90, m)
    X0 = f2gen.rhs_from_solution(k, m, 42)
    B = oracle.mmm(A, X0, m, k)
    out = oracle.solve(A, m, B.reshape(-1), k)
    assert out["consistent"] == (1 << 64) - 1
    Xs = f2gen.unpack_bits(out["X"].reshape(-1, 1), k).astype(np.int64)
    assert np.array_equal((bits_of(A, m) @ Xs) % 2, bits_of(B, k))


@pytest.mark.parametrize("n,m", [(3, 3), (3, 4), (4, 3)])
def test_rref_against_enumeration(n, m):
    for code in range(0, 1 << (n * m), 3):
        bits = np.array([(code >> k) & 1 for k in range(n * m)], dtype=np.int64).reshape(n, m)
        rr = oracle.rref(f2gen.pack_bits(bits), m)
        piv = brute_profile(bits)
        assert rr["pivcols"].tolist() == piv
        R = bits_of(rr["R"], m) if rr["rank"] else np.zeros((0, m), dtype=np.int64)
        # each RREF row is the unique span element with a 1 at its pivot
        # and 0 at every other pivot column
        span = set()
        for sel in itertools.product((0, 1), repeat=n):
            span.add(tuple((np.array(sel) @ bits) % 2))
        for t, p in enumerate(piv):
            want = [v for v in span if v[p] == 1 and all(v[q] == 0 for q in piv if q != p)
                    and all(v[c] == 0 for c in range(p))]
            assert len(want) == 1
            assert tuple(R[t]) == want[0]


def test_prefix_run_matches_full_run():
    """col_limit stops the same run early: the pivots, perm prefix and the
    first multipliers do not depend on later columns."""
    n, m, k = 300, 400, 150
    A = f2gen.uniform(n, m, 51)
    full = oracle.ple(A, m)
    part = oracle.ple(A, m, col_limit=k)
    r = part["rank"]
    assert np.array_equal(part["pivcols"], full["pivcols"][:r])
    assert np.array_equal(part["perm"][:r], full["perm"][:r])
    assert np.array_equal(part["E"][:r], full["E"][:r])
