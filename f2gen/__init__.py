"""Seeded synthetic F2 matrices and the bit-packed storage format.

This module is the one piece shared by the plain CPU oracle and the CUDA
library's tests and benchmark.  It holds no arithmetic of the decomposition
method: it only draws random bits, packs and unpacks them, and lays words out
in the two layouts used in this project.

Storage (Section 3 of the paper): an n x m matrix over F2 is held as an
n x mu array of unsigned words, mu = ceil(m/64); bit t of word q of row i is
entry a[i, 64q+t] (least significant bit = leftmost column), and bits at
columns >= m are zero.  ``rowmajor`` arrays here have shape (n, mu) with row
i's words contiguous; the library boundary uses *column blocks* (the paper's
column-major order of the word matrix): word (i, q) at offset q*ld + i, which
is just the transpose ``colblocks = rowmajor.T``.

Random bits come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the k-th output of a stream keyed by ``key`` is
``mix64(key + (k + 1) * GAMMA)``.  Every draw is therefore a pure function of
(seed, tags, counter) and the same matrix is produced on any machine.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

# Base seed of every workload in this project (the arXiv number of the paper).
BASE_SEED = 0x12095198


def mix64(z):
    """SplitMix64 output function on a uint64 numpy array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def mix64_int(x: int) -> int:
    """Scalar SplitMix64 output function on a Python int (mod 2**64)."""
    z = x & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *tags: int) -> int:
    """Key of an independent stream: the seed folded with each tag through mix64."""
    k = mix64_int((seed + 0x9E3779B97F4A7C15) & MASK64)
    for t in tags:
        k = mix64_int(k ^ ((t * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & MASK64))
    return k


def draws(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream keyed by ``key``."""
    k = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(key) + k * GAMMA
    return mix64(x)


def words_per_row(m: int) -> int:
    return (m + 63) // 64


def pad_mask(m: int) -> np.uint64:
    """Mask of the valid bits of the last word of a row with m columns."""
    r = m % 64
    return np.uint64(MASK64 if r == 0 else (1 << r) - 1)


def mask_padding(words: np.ndarray, m: int) -> np.ndarray:
    mu = words_per_row(m)
    if mu and m % 64:
        words[:, mu - 1] &= pad_mask(m)
    return words


# ---------------------------------------------------------------- matrices

def uniform(n: int, m: int, seed: int = BASE_SEED, *tags: int) -> np.ndarray:
    """n x m matrix with i.i.d. Bernoulli(1/2) entries, row-major words (n, mu)."""
    mu = words_per_row(m)
    w = draws(stream_key(seed, 1, n, m, *tags), 0, n * mu).reshape(n, mu)
    return mask_padding(w, m)


def bernoulli(n: int, m: int, p: float, seed: int = BASE_SEED, *tags: int) -> np.ndarray:
    """n x m matrix with i.i.d. Bernoulli(p) entries.

    p == 1/2 uses whole random words (same as ``uniform``); otherwise entry
    (i, j) is one iff the high 32 bits of draw number i*m + j are below
    floor(p * 2**32).
    """
    if p == 0.5:
        return uniform(n, m, seed, *tags)
    mu = words_per_row(m)
    thr = np.uint64(int(p * 2 ** 32))
    key = stream_key(seed, 2, n, m, int(p * 2 ** 32), *tags)
    out = np.zeros((n, mu), dtype=np.uint64)
    chunk = max(1, (1 << 22) // max(m, 1))
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        bits = (draws(key, a * m, (b - a) * m) >> np.uint64(32)) < thr
        out[a:b] = pack_bits(bits.reshape(b - a, m))
    return out


def sparse_rows(n: int, m: int, nnz: int, seed: int = BASE_SEED, *tags: int) -> np.ndarray:
    """n x m matrix whose every row has exactly ``nnz`` ones at distinct uniform
    positions (the sparse low-rank family of Section 7 of the paper)."""
    assert 0 <= nnz <= m
    key = stream_key(seed, 3, n, m, nnz, *tags)
    out = np.zeros((n, words_per_row(m)), dtype=np.uint64)
    if nnz == 0:
        return out
    cand = 4 * nnz + 8
    pos = (draws(key, 0, n * cand).reshape(n, cand) >> np.uint64(32)) * np.uint64(m) >> np.uint64(32)
    pos = pos.astype(np.int64)
    for i in range(n):
        _, first = np.unique(pos[i], return_index=True)
        take = pos[i][np.sort(first)][:nnz]
        j = 0
        while take.size < nnz:  # practically never: top up deterministically
            extra = int((mix64_int(key ^ (i * 7919 + j)) >> 32) * m >> 32)
            if extra not in take:
                take = np.append(take, extra)
            j += 1
        np.bitwise_or.at(out[i], take // 64, np.left_shift(np.uint64(1), (take % 64).astype(np.uint64)))
    return out


def permutation(count: int, key: int) -> np.ndarray:
    """A seeded permutation of range(count): argsort of ``count`` random keys."""
    return np.argsort(draws(key, 0, count), kind="stable").astype(np.int64)


def fixed_rank_factors(n: int, m: int, r: int, seed: int = BASE_SEED, *tags: int):
    """Factors X (n x r) and Y (r x m) of full rank r, row-major words.

    X = P1 [T; G] with T unit lower triangular (r x r), G uniform, P1 a
    random row permutation; Y = [U H] P2 with U unit upper triangular, H
    uniform, P2 a random column permutation.  The product X*Y has rank
    exactly r; computing it is left to the caller (each side uses its own
    product).
    """
    assert 0 <= r <= min(n, m)
    key = stream_key(seed, 4, n, m, r, *tags)
    rw = words_per_row(r)
    # T: row i keeps random bits below the diagonal and a one on it.
    tg = uniform(n, r, key, 10)
    if r:
        tri = _lower_mask(r)
        tg[:r] &= tri
        _set_diagonal(tg[:r])
    p1 = permutation(n, stream_key(key, 11))
    X = np.ascontiguousarray(tg[p1])
    # Y = [U H] P2, built in row chunks through unpacked bits.
    Y = np.zeros((r, words_per_row(m)), dtype=np.uint64)
    p2 = permutation(m, stream_key(key, 12))
    chunk = max(1, (1 << 23) // max(m, 1))
    for a in range(0, r, chunk):
        b = min(r, a + chunk)
        rows = np.arange(a, b)
        raw = draws(stream_key(key, 13), a * words_per_row(m), (b - a) * words_per_row(m))
        bits = unpack_bits(raw.reshape(b - a, words_per_row(m)), m)
        cols = np.arange(m)
        # U part: columns < r, keep strictly-upper bits, force the diagonal.
        upper = cols[None, :r] > rows[:, None]
        bits[:, :r] &= upper
        bits[np.arange(b - a), rows] = 1
        Y[a:b] = pack_bits(bits[:, p2])
    return X, Y


def _lower_mask(r: int) -> np.ndarray:
    """Row-major word mask of the strictly lower triangle of an r x r matrix."""
    rw = words_per_row(r)
    i = np.arange(r)[:, None]
    q = np.arange(rw)[None, :]
    full = q < (i // 64)
    part = q == (i // 64)
    shift = (i % 64).astype(np.uint64)
    with np.errstate(over="ignore"):
        pm = (np.uint64(1) << shift) - np.uint64(1)
    return np.where(full, np.uint64(MASK64), np.where(part, pm, np.uint64(0))).astype(np.uint64)


def _set_diagonal(w: np.ndarray) -> None:
    i = np.arange(w.shape[0])
    w[i, i // 64] |= np.left_shift(np.uint64(1), (i % 64).astype(np.uint64))


def rhs_from_solution(n_rhs: int, m: int, seed: int = BASE_SEED, *tags: int) -> np.ndarray:
    """m x n_rhs matrix X0 (one word per row, n_rhs <= 64) used to make B = A*X0."""
    assert 1 <= n_rhs <= 64
    return uniform(m, n_rhs, seed, 5, *tags)


# ---------------------------------------------------------------- F_p

def fp_uniform(n: int, m: int, p: int, seed: int = BASE_SEED, *tags: int) -> np.ndarray:
    """n x m matrix of residues mod p (int64), entry (i, j) = the high 32 bits
    of draw i*m + j, times p, over 2^32 (uniform up to a bias below p/2^32)."""
    assert 2 <= p < 2 ** 31
    key = stream_key(seed, 20, n, m, p, *tags)
    hi = (draws(key, 0, n * m) >> np.uint64(32)).astype(np.uint64)
    return ((hi * np.uint64(p)) >> np.uint64(32)).astype(np.int64).reshape(n, m)


def fp_fixed_rank_factors(n: int, m: int, r: int, p: int, seed: int = BASE_SEED, *tags: int):
    """Factors X (n x r) and Y (r x m) of full rank r over F_p (int64 residues):
    X = P1 [T; G] with T unit lower triangular, Y = [U H] P2 with U unit upper
    triangular, G, H and the off-diagonal entries uniform, P1 / P2 random row /
    column permutations.  X Y mod p has rank exactly r; the product is left to
    the caller."""
    assert 0 <= r <= min(n, m)
    key = stream_key(seed, 21, n, m, r, p, *tags)
    tg = fp_uniform(n, r, p, key, 1)
    i = np.arange(r)
    if r:
        tg[:r] = np.where(i[None, :] < i[:, None], tg[:r], 0)
        tg[i, i] = 1
    X = np.ascontiguousarray(tg[permutation(n, stream_key(key, 2))])
    uh = fp_uniform(r, m, p, key, 3)
    if r:
        cols = np.arange(m)
        uh[:, :r] = np.where(cols[None, :r] > i[:, None], uh[:, :r], 0)
        uh[i, i] = 1
    Y = np.ascontiguousarray(uh[:, permutation(m, stream_key(key, 4))])
    return X, Y


# ---------------------------------------------------------------- packing

def pack_bits(bits: np.ndarray, b: int = 64) -> np.ndarray:
    """Pack a 0/1 array (rows, cols) into words of b bits, LSB = leftmost column.

    Returns an array (rows, ceil(cols/b)) of uint64 whose values are < 2**b.
    """
    bits = np.asarray(bits).astype(np.uint8) & 1
    rows, cols = bits.shape
    nw = (cols + b - 1) // b
    if b == 64:
        padded = np.zeros((rows, nw * 64), dtype=np.uint8)
        padded[:, :cols] = bits
        by = np.packbits(padded.reshape(rows, nw * 8, 8), axis=2, bitorder="little")
        return np.ascontiguousarray(by.reshape(rows, nw * 8)).view("<u8").astype(np.uint64).reshape(rows, nw)
    out = np.zeros((rows, nw), dtype=np.uint64)
    for t in range(b):
        col = np.arange(nw) * b + t
        ok = col < cols
        out[:, ok] |= bits[:, col[ok]].astype(np.uint64) << np.uint64(t)
    return out


def unpack_bits(words: np.ndarray, cols: int, b: int = 64) -> np.ndarray:
    """Inverse of ``pack_bits``: (rows, nw) words -> (rows, cols) uint8 0/1."""
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    rows, nw = words.shape
    if b == 64:
        by = words.astype("<u8").view(np.uint8).reshape(rows, nw * 8)
        bits = np.unpackbits(by, axis=1, bitorder="little")
        return bits[:, :cols].copy()
    out = np.zeros((rows, cols), dtype=np.uint8)
    for t in range(b):
        col = np.arange(nw) * b + t
        ok = col < cols
        out[:, col[ok]] = ((words[:, ok] >> np.uint64(t)) & np.uint64(1)).astype(np.uint8)
    return out


def to_colblocks(rowmajor: np.ndarray, ld: int | None = None) -> np.ndarray:
    """Row-major words (n, mu) -> column-block words (mu, ld), word (i,q) at [q, i]."""
    n, mu = rowmajor.shape
    ld = n if ld is None else ld
    assert ld >= n
    out = np.zeros((mu, ld), dtype=np.uint64)
    out[:, :n] = rowmajor.T
    return out


def from_colblocks(colblocks: np.ndarray, n: int) -> np.ndarray:
    """Column-block words (mu, ld) -> row-major words (n, mu)."""
    return np.ascontiguousarray(np.asarray(colblocks, dtype=np.uint64)[:, :n].T)


def colmajor_flat(words: np.ndarray) -> list[int]:
    """The paper's column-major listing of a word matrix (Section 3 example)."""
    return [int(x) for x in np.asarray(words).T.reshape(-1)]
