/*
 * f2_oracle.c -- plain, slow, obviously-correct CPU reference for the F2
 * matrix decomposition of Bertolazzi & Rimoldi, "Fast matrix decomposition
 * in F2" (arXiv 1209.5198).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or table with the
 * CUDA path.
 *
 * Storage: every matrix here is ROW-MAJOR bit-packed (the paper's Section 3
 * packing, rows contiguous): row i of an r x c matrix occupies the words
 * M[i*ld .. i*ld + ceil(c/64)), bit t of word q is column 64q+t
 * (least significant bit = leftmost column), bits at columns >= c are zero.
 *
 * Functions and the passage each one follows:
 *   f2o_ple         Lemma 4.1 with the block size b = 1 (remark after Lemma
 *                   4.1: the b = 1 decomposition is PLE), pivot rule of
 *                   Procedure buildZ (first qualifying row in current order,
 *                   transposition with the current pivot slot), Section 4.3.
 *   f2o_blockdecomp The iterative block decomposition of Section 4 (eq. (Aj),
 *                   Lemma 4.1) for a general word size b <= 64, with the
 *                   pivot rows and pseudo-inverse of each block grown by the
 *                   incremental inverse of Section 4.2 (eqs. Bk:FACT,
 *                   cond:nonsing:Bk, fact:pre:Z), the row exchanges of
 *                   Section 4.3 and the inserted rows of Section 4.4, and
 *                   in-place storage as in Figure 1.  Second, independent
 *                   route to the same P.
 *   f2o_mmm         The definition of the matrix product over F2 (Section 1):
 *                   C[i] = XOR over k with A[i][k] = 1 of B[k].
 *   f2o_rref        Reduced row echelon form by textbook Gauss-Jordan
 *                   elimination (unique; uses of the decomposition, Section 1).
 *   f2o_solve       A x = b for up to 64 right-hand sides by Gauss-Jordan on
 *                   [A | B]; free variables are set to 0.
 *
 * Parity pins: see tests/test_oracle_pins.py (brute force on all tiny
 * matrices, reconstruction, invariants, known ranks, the paper's worked
 * examples, agreement of the two decomposition routes).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define F2O_OK 0
#define F2O_ERR_ARG 1
#define F2O_ERR_NOMEM 4

static int64_t nwords(int64_t cols) { return (cols + 63) / 64; }

static int getbit(const uint64_t *row, int64_t j) { return (int)((row[j >> 6] >> (j & 63)) & 1u); }

static void setbit(uint64_t *row, int64_t j) { row[j >> 6] |= (uint64_t)1 << (j & 63); }

static void swap_words(uint64_t *a, uint64_t *b, int64_t cnt) {
    for (int64_t q = 0; q < cnt; ++q) {
        uint64_t t = a[q];
        a[q] = b[q];
        b[q] = t;
    }
}

static int popcount_odd(uint64_t x) { return __builtin_popcountll(x) & 1; }

/* ------------------------------------------------------------------ PLE --
 * Bit-level elimination, column by column (block size b = 1):
 *   for each column j: the pivot is the first row i >= t (current order)
 *   whose entry in column j is 1; rows i and t are exchanged (full rows,
 *   including the multipliers of L already stored, and the permutation);
 *   every later row with a 1 in column j gets the pivot row added and its
 *   multiplier L[i][t] = 1.
 * Output: perm (P*A)[i] = A[perm[i]]; pivcols[0..rank); L (n x min(n,m),
 * unit lower trapezoidal, first `rank` columns meaningful); E (min(n,m) x m,
 * row echelon, first `rank` rows) with P*A = L*E.
 * col_limit >= 0 stops after the columns j < col_limit (a prefix of the same
 * run: the pivots of those columns depend on those columns only).
 */
int f2o_ple(int64_t n, int64_t m, const uint64_t *A, int64_t lda,
            int32_t *perm, int32_t *pivcols, int64_t *rank_out,
            uint64_t *L, int64_t ldl, uint64_t *E, int64_t lde,
            int64_t col_limit, int nthreads)
{
    if (n < 0 || m < 0 || (n > 0 && m > 0 && (!A || lda < nwords(m))) || !rank_out) return F2O_ERR_ARG;
    const int64_t mu = nwords(m);
    const int64_t kmax = n < m ? n : m;
    const int64_t lw = nwords(kmax) > 0 ? nwords(kmax) : 1;
    if (L && ldl < nwords(kmax)) return F2O_ERR_ARG;
    if (E && lde < mu) return F2O_ERR_ARG;
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n * mu + 1));
    uint64_t *Lw = (uint64_t *)calloc((size_t)(n * lw + 1), sizeof(uint64_t));
    int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!W || !Lw || !pr) { free(W); free(Lw); free(pr); return F2O_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        memcpy(W + i * mu, A + i * lda, sizeof(uint64_t) * (size_t)mu);
        pr[i] = (int32_t)i;
    }
    if (nthreads < 1) nthreads = 1;
    int64_t t = 0;
    const int64_t jend = (col_limit >= 0 && col_limit < m) ? col_limit : m;
    for (int64_t j = 0; j < jend && t < n; ++j) {
        const int64_t q = j >> 6;
        int64_t piv = -1;
        for (int64_t i = t; i < n; ++i) {
            if (getbit(W + i * mu, j)) { piv = i; break; }
        }
        if (piv < 0) continue;
        if (piv != t) {
            swap_words(W + piv * mu, W + t * mu, mu);
            swap_words(Lw + piv * lw, Lw + t * lw, lw);
            int32_t tmp = pr[piv]; pr[piv] = pr[t]; pr[t] = tmp;
        }
        pivcols[t] = (int32_t)j;
        setbit(Lw + t * lw, t);
        const uint64_t *prow = W + t * mu;
        #pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1 && (n - t) * (mu - q) > 65536)
        for (int64_t i = t + 1; i < n; ++i) {
            uint64_t *row = W + i * mu;
            if (getbit(row, j)) {
                for (int64_t w = q; w < mu; ++w) row[w] ^= prow[w];
                setbit(Lw + i * lw, t);
            }
        }
        ++t;
    }
    *rank_out = t;
    if (perm) memcpy(perm, pr, sizeof(int32_t) * (size_t)n);
    if (L) {
        for (int64_t i = 0; i < n; ++i) {
            memset(L + i * ldl, 0, sizeof(uint64_t) * (size_t)ldl);
            memcpy(L + i * ldl, Lw + i * lw, sizeof(uint64_t) * (size_t)nwords(kmax));
        }
    }
    if (E) {
        for (int64_t i = 0; i < kmax; ++i) {
            memset(E + i * lde, 0, sizeof(uint64_t) * (size_t)lde);
            if (i < t) memcpy(E + i * lde, W + i * mu, sizeof(uint64_t) * (size_t)mu);
        }
    }
    free(W); free(Lw); free(pr);
    return F2O_OK;
}

/* ------------------------------------------------- block pivot search --
 * Row selection and pseudo-inverse of one column block of b-bit words
 * a[0..rows), written from the equations of Sections 4.2-4.4 (not from the
 * printed procedure):
 *
 *   The square matrix S = J B + R of Section 4.1 is grown one row at a time.
 *   After k rows its leading k x k minor S_k is nonsingular; its inverse Z_k
 *   is held as k explicit COLUMN vectors zc[0..k) (bit i of zc[t] = entry
 *   (i, t) of Z_k) and the rows of S as b-bit words srow[0..k).
 *   For bit k let c = column k of S_k (bit i = bit k of srow[i]) and
 *   ct = Z_k c.  A candidate row (r^T, alpha, beta^T) -- r its first k bits,
 *   alpha its bit k -- extends S_k to a nonsingular S_{k+1} iff
 *   alpha xor r^T Z_k c = alpha xor parity(r & ct) = 1 (eq. cond:nonsing:Bk).
 *   The first candidate at or after the current pivot slot, in the current
 *   row order, is exchanged with that slot (Section 4.3).  If no row
 *   qualifies, the virtual row (0^T, 1, 0^T) of Section 4.4 is inserted:
 *   r = 0 and alpha = 1 satisfy the condition trivially.
 *   Z_{k+1} follows eq. (fact:pre:Z): with rho^T = r^T Z_k,
 *     column t < k becomes zc[t] xor rho_t ct, with rho_t as its entry k
 *     (the rank-one update Z_k xor ct rho^T and the new bottom row rho^T),
 *     and the new column k is ct with entry k equal to 1.
 * At the end Z = S^{-1} J (eq. pre:W): the columns of S^{-1} at the real
 * rows, so that B Z = I and D Z = Y.  It is returned by rows (Zr[i] bit s =
 * entry (i, s), s < r).  P[k] = index in a[] (before the exchange) of the
 * row chosen for bit k, or -1 for an inserted row.  Returns r.
 */
static int select_block_pivots(uint64_t *a, int64_t rows, int b, uint64_t *Zr, int64_t *P)
{
    uint64_t zc[64], srow[64];
    int real[64];
    int64_t slot = 0;
    int r = 0;
    for (int k = 0; k < b; ++k) {
        const uint64_t kbit = (uint64_t)1 << k;
        const uint64_t low = kbit - 1; /* the first k columns */
        uint64_t ct = 0;               /* Z_k c */
        for (int t = 0; t < k; ++t)
            if (srow[t] & kbit) ct ^= zc[t];
        uint64_t row = kbit; /* the virtual row unless a real one qualifies */
        P[k] = -1;
        for (int64_t i = slot; i < rows; ++i) {
            const int alpha = (int)((a[i] >> k) & 1);
            if (alpha ^ popcount_odd(a[i] & low & ct)) {
                P[k] = i;
                row = a[i];
                a[i] = a[slot];
                a[slot] = row;
                ++slot;
                break;
            }
        }
        const uint64_t rk = row & low;
        for (int t = 0; t < k; ++t)
            if (popcount_odd(rk & zc[t])) zc[t] ^= ct | kbit;
        zc[k] = ct | kbit;
        srow[k] = row;
        if (P[k] >= 0) real[r++] = k;
    }
    for (int i = 0; i < b; ++i) {
        uint64_t w = 0;
        for (int s = 0; s < r; ++s)
            if ((zc[real[s]] >> i) & 1) w |= (uint64_t)1 << s;
        Zr[i] = w;
    }
    return r;
}

/* -------------------------------------------------------- block driver --
 * Iterative block decomposition of Section 4 with word size b (1..64).
 * The matrix is held as the paper does: column blocks of b-bit words,
 * word (i, q) at Wb[q*n + i].  For each block j:
 *   the pivot search on rows R..n of block j (selects B^(j), gives Z and
 *   r_j); the same transpositions are applied to the whole rows (every other
 *   block, including the L multipliers stored to the left, and perm);
 *   Y = D * Z for the rows below the pivots (eq. pre:W);
 *   A^(j+1) = E xor Y * C on the blocks to the right (eq. Aj);
 *   Y is stored in place of D (Figure 1) and R += r_j.
 * Outputs: perm, pivcols (b*j + k for the bits k with P[k] != -1, in
 * order), rank, r_j per block, and the final in-place storage Wb (Figure 1:
 * U block rows on and right of the diagonal blocks, Y multipliers below).
 */
int f2o_blockdecomp(int64_t n, int64_t m, int b, const uint64_t *A, int64_t lda,
                    int32_t *perm, int32_t *pivcols, int64_t *rank_out,
                    int32_t *rblock, uint64_t *Wb_out)
{
    if (n < 0 || m < 0 || b < 1 || b > 64 || !rank_out) return F2O_ERR_ARG;
    const int64_t mub = (m + b - 1) / b;
    const uint64_t bmask = b == 64 ? ~(uint64_t)0 : (((uint64_t)1 << b) - 1);
    uint64_t *Wb = (uint64_t *)calloc((size_t)(n * mub + 1), sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!Wb || !y || !pr) { free(Wb); free(y); free(pr); return F2O_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        pr[i] = (int32_t)i;
        for (int64_t c = 0; c < m; ++c)
            if (getbit(A + i * lda, c)) Wb[(c / b) * n + i] |= (uint64_t)1 << (c % b);
    }
    int64_t R = 0;
    for (int64_t j = 0; j < mub && R < n; ++j) {
        uint64_t Z[64];
        int64_t P[64];
        uint64_t *panel = Wb + j * n + R;
        const int bj = (int)((m - j * b) < b ? (m - j * b) : b);
        const int r = select_block_pivots(panel, n - R, bj, Z, P);
        if (rblock) rblock[j] = r;
        /* the transpositions, in the order the search made them */
        int s = 0;
        for (int k = 0; k < bj; ++k) {
            if (P[k] < 0) continue;
            const int64_t r1 = R + s, r2 = R + P[k];
            pivcols[R + s] = (int32_t)(j * b + k);
            if (r1 != r2) {
                for (int64_t q = 0; q < mub; ++q) {
                    if (q == j) continue; /* block j was exchanged by the search */
                    uint64_t tmp = Wb[q * n + r1]; Wb[q * n + r1] = Wb[q * n + r2]; Wb[q * n + r2] = tmp;
                }
                int32_t tp = pr[r1]; pr[r1] = pr[r2]; pr[r2] = tp;
            }
            ++s;
        }
        /* Y = D * Z (r bits per row) */
        for (int64_t i = R + r; i < n; ++i) {
            uint64_t d = Wb[j * n + i] & bmask, acc = 0;
            for (int t = 0; t < bj; ++t)
                if (d & ((uint64_t)1 << t)) acc ^= Z[t];
            y[i] = acc;
        }
        /* Schur complement update E <- E xor Y*C on the blocks to the right */
        for (int64_t q = j + 1; q < mub; ++q) {
            for (int64_t i = R + r; i < n; ++i) {
                uint64_t acc = 0;
                for (int t = 0; t < r; ++t)
                    if (y[i] & ((uint64_t)1 << t)) acc ^= Wb[q * n + R + t];
                Wb[q * n + i] ^= acc;
            }
        }
        for (int64_t i = R + r; i < n; ++i) Wb[j * n + i] = y[i];
        R += r;
    }
    *rank_out = R;
    if (perm) memcpy(perm, pr, sizeof(int32_t) * (size_t)n);
    if (Wb_out) memcpy(Wb_out, Wb, sizeof(uint64_t) * (size_t)(n * mub));
    free(Wb); free(y); free(pr);
    return F2O_OK;
}

/* ------------------------------------------------------------- product --
 * C = A*B (accumulate = 0) or C ^= A*B (accumulate = 1), A n x k, B k x m:
 * row i of the product is the XOR of the rows k of B with A[i][k] = 1.
 */
int f2o_mmm(int64_t n, int64_t k, int64_t m, const uint64_t *A, int64_t lda,
            const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, int accumulate, int nthreads)
{
    if (n < 0 || k < 0 || m < 0) return F2O_ERR_ARG;
    const int64_t mu = nwords(m);
    if (nthreads < 1) nthreads = 1;
    #pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1 && n * k > 65536)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t *c = C + i * ldc;
        if (!accumulate) memset(c, 0, sizeof(uint64_t) * (size_t)mu);
        for (int64_t t = 0; t < k; ++t) {
            if (!getbit(A + i * lda, t)) continue;
            const uint64_t *brow = B + t * ldb;
            for (int64_t w = 0; w < mu; ++w) c[w] ^= brow[w];
        }
    }
    return F2O_OK;
}

/* ---------------------------------------------------------------- RREF --
 * Textbook Gauss-Jordan: for each column, take any row at or below the
 * current one with a 1 there, move it up, clear the column in every other
 * row.  The reduced form is unique, so the choice of row does not matter.
 * R receives n rows: the first `rank` form the RREF, the rest are zero.
 */
int f2o_rref(int64_t n, int64_t m, const uint64_t *A, int64_t lda,
             uint64_t *R, int64_t ldr, int32_t *pivcols, int64_t *rank_out)
{
    if (n < 0 || m < 0 || !R || ldr < nwords(m) || !rank_out) return F2O_ERR_ARG;
    const int64_t mu = nwords(m);
    for (int64_t i = 0; i < n; ++i) {
        memset(R + i * ldr, 0, sizeof(uint64_t) * (size_t)ldr);
        memcpy(R + i * ldr, A + i * lda, sizeof(uint64_t) * (size_t)mu);
    }
    int64_t t = 0;
    for (int64_t j = 0; j < m && t < n; ++j) {
        int64_t piv = -1;
        for (int64_t i = t; i < n; ++i)
            if (getbit(R + i * ldr, j)) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != t) swap_words(R + piv * ldr, R + t * ldr, mu);
        for (int64_t i = 0; i < n; ++i) {
            if (i != t && getbit(R + i * ldr, j))
                for (int64_t w = 0; w < mu; ++w) R[i * ldr + w] ^= R[t * ldr + w];
        }
        if (pivcols) pivcols[t] = (int32_t)j;
        ++t;
    }
    *rank_out = t;
    return F2O_OK;
}

/* --------------------------------------------------------------- solve --
 * A x = b for nrhs <= 64 right-hand sides: B holds one word per row of A
 * (bit c = right-hand side c), X receives one word per column of A.
 * Gauss-Jordan on the augmented matrix [A | B]; the solution with every
 * free variable 0 is x[pivcol_t] = (reduced B)[t].  Right-hand side c is
 * consistent iff its bit is 0 in every reduced row at or beyond the rank;
 * the columns of inconsistent right-hand sides are returned as 0.
 */
int f2o_solve(int64_t n, int64_t m, const uint64_t *A, int64_t lda, int nrhs,
              const uint64_t *B, uint64_t *X, uint64_t *consistent_out)
{
    if (n < 0 || m < 0 || nrhs < 1 || nrhs > 64 || !B || !X || !consistent_out) return F2O_ERR_ARG;
    const int64_t mu = nwords(m);
    const int64_t ld = mu + 1; /* augmented row: mu words of A, then the RHS word */
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n * ld + 1));
    int32_t *pc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!W || !pc) { free(W); free(pc); return F2O_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        memcpy(W + i * ld, A + i * lda, sizeof(uint64_t) * (size_t)mu);
        W[i * ld + mu] = B[i];
    }
    int64_t t = 0;
    for (int64_t j = 0; j < m && t < n; ++j) {
        int64_t piv = -1;
        for (int64_t i = t; i < n; ++i)
            if (getbit(W + i * ld, j)) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != t) swap_words(W + piv * ld, W + t * ld, ld);
        for (int64_t i = 0; i < n; ++i)
            if (i != t && getbit(W + i * ld, j))
                for (int64_t w = 0; w < ld; ++w) W[i * ld + w] ^= W[t * ld + w];
        pc[t] = (int32_t)j;
        ++t;
    }
    const uint64_t all = nrhs == 64 ? ~(uint64_t)0 : (((uint64_t)1 << nrhs) - 1);
    uint64_t bad = 0;
    for (int64_t i = t; i < n; ++i) bad |= W[i * ld + mu];
    bad &= all;
    const uint64_t ok = all & ~bad;
    memset(X, 0, sizeof(uint64_t) * (size_t)m);
    for (int64_t s = 0; s < t; ++s) X[pc[s]] = W[s * ld + mu] & ok;
    *consistent_out = ok;
    free(W); free(pc);
    return F2O_OK;
}

/* Number of threads an OpenMP region would use (1 without OpenMP). */
int f2o_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
