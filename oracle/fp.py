"""Plain CPU oracle of the decomposition over a prime field F_p.

TEST INFRASTRUCTURE ONLY: imported by tests/ (never by the CUDA library or
its binding).  Matrices are numpy int64 arrays of residues 0 <= a < p, p a
prime below 2^31 (products of two residues stay below 2^62).

The paper states the method over F2 and, in the remark after eq.
(cond:nonsing:Bk) (Section 4.2), its change over F_q: a row qualifies as the
pivot of a column when its reduced entry beta is nonzero (instead of one),
and beta then stays on the diagonal of the echelon factor.  With the pivot
rule of Procedure buildZ -- the first qualifying row in the current order,
exchanged into the pivot slot, no column exchanges -- the factors are the
PLE form, unique given that rule (Lemma 4.1 at b = 1, with beta != 1
allowed): this function is that elimination written out, one column at a
time.
"""
from __future__ import annotations

import numpy as np


def inverse(beta: int, p: int) -> int:
    """beta^-1 mod p by the extended Euclidean algorithm."""
    r0, r1, s0, s1 = p, beta % p, 0, 1
    while r1:
        q = r0 // r1
        r0, r1 = r1, r0 - q * r1
        s0, s1 = s1, s0 - q * s1
    if r0 != 1:
        raise ZeroDivisionError(f"{beta} has no inverse mod {p}")
    return s0 % p


def ple(A: np.ndarray, p: int) -> dict:
    """P A = L E over F_p.  Returns perm ((P A)[i] = A[perm[i]]), pivcols (the
    r pivot columns), rank r, L (n x k, unit lower trapezoidal; columns past r
    zero) and E (k x m, row echelon with E[t][pivcols[t]] = beta_t; rows past r
    zero), k = min(n, m)."""
    W = np.array(A, dtype=np.int64) % p
    n, m = W.shape
    k = min(n, m)
    perm = np.arange(n, dtype=np.int64)
    L = np.zeros((n, k), dtype=np.int64)
    pivcols = []
    t = 0
    for j in range(m):
        if t == n:
            break
        rows = np.nonzero(W[t:, j])[0]
        if rows.size == 0:
            continue  # no qualifying row: no pivot in this column
        i = t + int(rows[0])  # the first qualifying row in the current order
        if i != t:  # exchange whole rows, the multipliers stored so far included
            W[[t, i]] = W[[i, t]]
            perm[[t, i]] = perm[[i, t]]
            L[[t, i], :t] = L[[i, t], :t]
        beta = int(W[t, j])
        inv = inverse(beta, p)
        below = np.nonzero(W[t + 1:, j])[0] + t + 1
        if below.size:
            mult = (W[below, j] * inv) % p
            W[below, :] = (W[below, :] - (mult[:, None] * W[t, :][None, :]) % p) % p
            L[below, t] = mult
        L[t, t] = 1
        pivcols.append(j)
        t += 1
    E = np.zeros((k, m), dtype=np.int64)
    E[:t] = W[:t]
    return {"perm": perm, "pivcols": np.array(pivcols, dtype=np.int64), "rank": t, "L": L, "E": E}


def rank(A: np.ndarray, p: int) -> int:
    return ple(A, p)["rank"]
