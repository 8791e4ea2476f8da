/*
 * gf2.h -- C ABI of a GB300 (sm_103a) library for dense linear algebra over
 * F2: the block decomposition P*A = L*E of Bertolazzi & Rimoldi, "Fast
 * matrix decomposition in F2" (arXiv 1209.5198), with row permutations only
 * (no column swaps), its rank, its echelon form, linear solves, and the
 * matrix product over F2.
 *
 * Matrix layout (Section 3 of the paper).  An r x c matrix over F2 is held
 * as ceil(c/64) "column blocks" of 64-bit words in DEVICE memory: the word
 * for row i and column block q is w[q*ld + i] (ld >= r), and bit t of that
 * word is entry (i, 64q + t) -- the least significant bit is the leftmost
 * column (the paper's bit order).  Bits at columns >= c must be zero
 * ("padding"); the library checks this unless GF2_NOCHECK is given.
 *
 * Streams.  Every call is asynchronous on the CUDA stream passed as `stream`
 * (a cudaStream_t; NULL = the legacy default stream) unless its name ends in
 * _host, or a padding check is requested (the check reads one flag back).
 *
 * Workspace.  Calls that need scratch memory take (workspace, ws_bytes).
 * Pass a device buffer of at least the size the matching *_workspace_bytes
 * function returns; pass NULL to let the library use its own buffer, which
 * it allocates on first use, grows when needed and keeps per device until
 * gf2_release_workspace().  The library's own buffer is shared by every call
 * on that device: calls that use it must not overlap in time.
 *
 * Errors.  Every entry point returns a status: GF2_OK or one of the codes
 * below.  No exception crosses the ABI.  On an error nothing is launched,
 * except GF2_ERR_CUDA, which reports a failed CUDA call.
 */
#ifndef GF2_H
#define GF2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF2_OK 0
#define GF2_ERR_ARG 1         /* NULL pointer, negative size, bad flag      */
#define GF2_ERR_SHAPE 2       /* inner dimensions differ, ld < rows, k > 64 */
#define GF2_ERR_PADDING 3     /* a bit at a column >= cols is set           */
#define GF2_ERR_NOMEM 4       /* workspace too small / allocation failed    */
#define GF2_ERR_CUDA 5        /* a CUDA runtime call failed                 */
#define GF2_ERR_TIMEOUT 6     /* a bounded device-side wait gave up         */
#define GF2_ERR_UNSUPPORTED 7 /* size beyond what this build handles        */

/* flags */
#define GF2_NOCHECK 1u    /* skip the padding check of the inputs */
#define GF2_MMM_TABLES 2u /* gf2_mmm: Four Russians passes (M4RM) */
#define GF2_MMM_TENSOR 4u /* gf2_mmm: tensor cores (e4m3 products, exact mod 2; k < 2^24) */

typedef struct gf2_mat {
    uint64_t *w;          /* device pointer, column blocks (see above) */
    int64_t rows, cols;   /* matrix size in entries                     */
    int64_t ld;           /* words between column blocks, >= rows       */
} gf2_mat;

/* Human-readable text for a status code (static storage, never NULL). */
const char *gf2_status_string(int status);

/* Library ABI version (increments on incompatible changes). */
int gf2_version(void);

/* Frees the library-owned workspace of the current device (safe to call
 * when none exists).  Synchronises the device. */
int gf2_release_workspace(void);

/* ------------------------------------------------------------------------
 * Per-call options.  Every field 0 means "automatic": the library's default,
 * or the process-wide setting of the matching setter below
 * (gf2_mmm_set_strassen_cutoff, gf2_batched_set_c8_from), which are only
 * defaults.  The entry points ending in _ex take a gf2_opts (NULL = all 0),
 * so that callers on different threads can use different settings without
 * touching shared state.  No field changes a result: every option gives the
 * same bits (the factors are unique given the pivot rule, the product is
 * exact); they change only speed and memory.
 *   panel_w          decomposition: columns per trailing update (Section 5,
 *                    the wide-panel form): 64 = one update per 64-column
 *                    block, 128 = one update per pair of blocks (default).
 *                    Other multiples of 64: GF2_ERR_UNSUPPORTED.
 *   table_c          decomposition: bits per Four Russians table of the
 *                    trailing update (Section 6): 4 or 8; 0 = 8, and 4 for a
 *                    single-block update with fewer than 4096 rows below it.
 *                    Other values up to 16: GF2_ERR_UNSUPPORTED.
 *   tile_words       words per column tile of the working copy: 4 (the only
 *                    one built; others GF2_ERR_UNSUPPORTED).
 *   backend          product: GF2_BACKEND_AUTO (M4RM under Strassen-Winograd),
 *                    GF2_BACKEND_TABLES (M4RM alone), GF2_BACKEND_TENSOR.
 *   schedule         decomposition by pairs of panels: GF2_SCHEDULE_STREAMS
 *                    runs it as separate launches on three streams (one CTA
 *                    per panel; the trailing updates beside the look-ahead
 *                    kernels on the same SMs); GF2_SCHEDULE_PERSISTENT as one
 *                    cooperative persistent launch (one CTA per SM: CTA 0
 *                    runs the panel chain, the others the look-ahead and the
 *                    trailing updates, ordered by device counters);
 *                    GF2_SCHEDULE_SPLIT the first three quarters of the
 *                    panels as separate launches and the rest persistent;
 *                    AUTO is STREAMS (the fastest measured at 32768; also
 *                    with panel_w 64 and on a device that cannot hold one CTA
 *                    per SM, whatever is asked).  A persistent run whose
 *                    bounded device waits give up writes rank -1 (the other
 *                    outputs are then undefined); the calls that read the
 *                    rank back return GF2_ERR_TIMEOUT.
 *   strassen_cutoff  product: the Strassen-Winograd cutoff, >= 128
 *                    (GF2_STRASSEN_OFF: no recursion); 0 = the process one.
 *   batched_c8_from  batched decomposition: the size from which a matrix
 *                    uses 8-bit tables (gf2_batched_set_c8_from); 0 = the
 *                    process one.
 * Negative values and values the field does not know: GF2_ERR_ARG. */
#define GF2_BACKEND_AUTO 0
#define GF2_BACKEND_TABLES 1
#define GF2_BACKEND_TENSOR 2
#define GF2_STRASSEN_OFF ((int64_t)1 << 62)

#define GF2_SCHEDULE_AUTO 0
#define GF2_SCHEDULE_STREAMS 1
#define GF2_SCHEDULE_PERSISTENT 2
#define GF2_SCHEDULE_SPLIT 3

typedef struct gf2_opts {
    int32_t panel_w;
    int32_t table_c;
    int32_t tile_words;
    int32_t backend;
    int32_t schedule;
    int32_t reserved;         /* must be 0 */
    int64_t strassen_cutoff;
    int64_t batched_c8_from;
} gf2_opts;

/* Checks a gf2_opts without using the GPU: GF2_OK, GF2_ERR_ARG or
 * GF2_ERR_UNSUPPORTED, as an _ex call with it would return first.  NULL is
 * valid (all automatic). */
int gf2_opts_check(const gf2_opts *o);

/* ------------------------------------------------------------------------
 * Product over F2 (Section 1 and Section 6 of the paper).
 *   C = A*B        (accumulate == 0)
 *   C = C xor A*B  (accumulate != 0)
 * A is n x k, B is k x m, C is n x m (all column blocks, device memory,
 * owned by the caller).  C must not alias A or B.  Exact: every result bit
 * is the parity of the AND of a row of A and a column of B, whatever the
 * backend:
 *   default / no backend flag: the Four Russians method (M4RM, Section 6),
 *       one kernel on the column blocks (tables of 8 rows of B in shared
 *       memory, C kept in registers over the inner dimension), under
 *       Strassen-Winograd recursion (7 products, 15 additions per level;
 *       the recursion of Section 5) while n, k and m are all at least the
 *       Strassen cutoff, n is even, k a whole even number of words and m an
 *       even number of words.  The cutoff is off until gf2_mmm_autotune or
 *       gf2_mmm_set_strassen_cutoff sets it.
 *   GF2_MMM_TABLES: M4RM alone (no recursion).
 *   GF2_MMM_TENSOR: the fifth-generation tensor cores (tcgen05.mma of
 *       kind::f8f6f4 with operands loaded by TMA, accumulators in tensor
 *       memory): every entry an e2m1 0 or 1, the integer sums in fp32
 *       folded into parity bits every 4096 of the inner dimension, entry =
 *       lowest bit; k < 2^24, else M4RM.  This backend synchronises the
 *       stream once before it returns, to read its error word: a device
 *       wait that gave up returns GF2_ERR_TIMEOUT.
 * The workspace depends on the backend and the recursion depth: size it
 * with the same flags (and after the same cutoff setting).
 * Errors: GF2_ERR_ARG (NULL, both backend flags), GF2_ERR_SHAPE (A.cols !=
 * B.rows, C not n x m, ld < rows), GF2_ERR_PADDING, GF2_ERR_NOMEM,
 * GF2_ERR_UNSUPPORTED (a dimension >= 2^31), GF2_ERR_CUDA.
 */
size_t gf2_mmm_workspace_bytes(int64_t n, int64_t k, int64_t m, unsigned flags);
int gf2_mmm(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags,
            void *workspace, size_t ws_bytes, void *stream);

/* gf2_mmm with per-call options: opts->backend and opts->strassen_cutoff
 * take the place of the backend flags and of the process-wide cutoff (flags
 * may still hold GF2_NOCHECK; a backend flag together with a backend option
 * is GF2_ERR_ARG).  Size the workspace with gf2_mmm_workspace_bytes_ex and
 * the same options. */
size_t gf2_mmm_workspace_bytes_ex(int64_t n, int64_t k, int64_t m, unsigned flags, const gf2_opts *opts);
int gf2_mmm_ex(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags,
               const gf2_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* The Strassen cutoff of the default product (a process-wide setting).
 * gf2_mmm_autotune times, on the current device, square products of size d
 * = 2048, 4096, ... up to max_dim (at most 32768) with M4RM alone and with
 * one Strassen-Winograd level, and sets the cutoff to the smallest d from
 * which one level is faster at d and at every larger size tried (off when
 * it never is); *cutoff receives it.  It allocates about 3 d^2/8 bytes plus
 * one level's temporaries, synchronises the stream and leaves the device
 * memory as it found it.  gf2_mmm_set_strassen_cutoff sets it directly
 * (>= 128; 2^62 turns the recursion off).  Errors: GF2_ERR_ARG,
 * GF2_ERR_NOMEM, GF2_ERR_CUDA. */
int gf2_mmm_autotune(int64_t max_dim, int64_t *cutoff, void *stream);

/* ------------------------------------------------------------------------
 * Decomposition over a prime field F_p (the remark after eq.
 * (cond:nonsing:Bk), Section 4.2: over F_q the pivot condition becomes "the
 * reduced entry beta is nonzero" and beta stays on the diagonal).  A is n x
 * m, row-major 32-bit residues (entry (i, j) at A[i*lda + j], device, read
 * only, every entry < p), p a prime with 2 <= p < 2^31.  Column by column,
 * the first row in the current order whose reduced entry is nonzero is
 * exchanged into the pivot slot and the rows after it are eliminated; no
 * column is exchanged.  Outputs (device, owned by the caller):
 *   perm[n]      (P A)[i] = A[perm[i]]
 *   pivcols[k]   the r pivot columns, increasing, then -1 (k = min(n, m))
 *   *rank        r (int64; -1 if a bounded device wait gave up)
 *   L (optional) n x k row-major (ldl >= k): unit lower trapezoidal, columns
 *                >= r zero
 *   E (optional) k x m row-major (lde >= m): row echelon, E[t][pivcols[t]] =
 *                beta_t != 0, zero before it; rows >= r zero
 * with P A = L E (mod p); for p = 2 the factors equal gf2_decompose's.
 * Asynchronous on `stream`, except the entry check (skipped with
 * GF2_NOCHECK), which synchronises it once.  Workspace:
 * gf2_fp_decompose_workspace_bytes(n, m) (about 4 n m bytes), or NULL for the
 * library's own.  Errors: GF2_ERR_ARG (p not a prime in [2, 2^31), NULL
 * pointers, an entry >= p), GF2_ERR_SHAPE (lda < m, ldl < k, lde < m),
 * GF2_ERR_NOMEM, GF2_ERR_UNSUPPORTED (n or m >= 2^31, n above 1024 rows per
 * SM of the device, or no cooperative launch), GF2_ERR_CUDA. */
size_t gf2_fp_decompose_workspace_bytes(int64_t n, int64_t m);
int gf2_fp_is_prime(uint32_t p);
int gf2_fp_decompose(const uint32_t *A, int64_t lda, int64_t n, int64_t m, uint32_t p, int32_t *perm,
                     int32_t *pivcols, int64_t *rank, uint32_t *L, int64_t ldl, uint32_t *E, int64_t lde,
                     unsigned flags, void *workspace, size_t ws_bytes, void *stream);

/* A measurement aid with no counterpart in the paper: the rate of the
 * tensor pipe for the MMA shape the tensor backend issues (tcgen05.mma
 * kind::f8f6f4, 128 x 256 x 32, 8-bit operands in, fp32 out) from shared memory, with
 * no loads: one CTA per SM issues iters x 4 MMAs into one accumulator.
 * *tflops receives dense TFLOP/s (2 flops per multiply-add) on the current
 * device, timed by CUDA events on the stream, which it synchronises.
 * Errors: GF2_ERR_ARG (iters < 1, tflops NULL), GF2_ERR_TIMEOUT,
 * GF2_ERR_CUDA. */
int gf2_tensor_peak(int64_t iters, double *tflops, void *stream);
int gf2_mmm_set_strassen_cutoff(int64_t cutoff);
int64_t gf2_mmm_strassen_cutoff(void);

/* ------------------------------------------------------------------------
 * Decomposition P*A = L*E (Section 4, Lemma 4.1 of the paper: block
 * elimination with pseudo-inverse Z, Procedure buildZ for the row
 * permutation, Schur-complement update A(j+1) = E xor Y C by M4RM, eq. (Aj)).
 * A is n x m and is not modified.  With r = rank(A) and k = min(n, m):
 *   perm    int32[n], device: row i of P*A is row perm[i] of A.  The pivot
 *           rule is the paper's: within each column block, bit by bit, the
 *           first row (in the current order) that satisfies the
 *           non-singularity condition (eq. cond:nonsing:Bk) is exchanged with
 *           the current pivot slot.
 *   pivcols int32[k], device: pivcols[t] (t < r) is the column of the t-th
 *           pivot, increasing (the column rank profile of A); entries t >= r
 *           are set to -1.
 *   rank    int64*, device: receives r.
 *   L       n x k (may be NULL): unit lower trapezoidal, L[t][t] = 1, zero
 *           above the diagonal and in columns >= r.
 *   E       k x m (may be NULL): row echelon, row t (t < r) has its leading
 *           one at pivcols[t]; rows >= r are zero.
 * The factors are the bit-level PLE form (remark after Lemma 4.1: the block
 * decomposition with b = 1 is PLE); P, pivcols and r are the same for every
 * block size.  Exact over F2: P*A = L*E bit for bit.
 * Asynchronous on `stream` (after the padding check, which synchronises it
 * once unless GF2_NOCHECK).  The second call with the same shape and buffers
 * captures the launch sequence into a CUDA graph on the library's streams
 * (thread-local capture mode) and later calls replay it; while a call
 * captures, a device-wide synchronisation from another host thread
 * (cudaDeviceSynchronize, torch.cuda.synchronize) fails with
 * cudaErrorStreamCaptureUnsupported, so multi-threaded callers synchronise
 * their own streams instead.
 * Errors: GF2_ERR_ARG, GF2_ERR_SHAPE (ld < rows, L or E of the wrong size),
 * GF2_ERR_PADDING, GF2_ERR_NOMEM, GF2_ERR_UNSUPPORTED (n >= 2^31), GF2_ERR_CUDA.
 */
size_t gf2_decompose_workspace_bytes(int64_t n, int64_t m, int want_factors);
int gf2_decompose(const gf2_mat *A, int32_t *perm, int32_t *pivcols, int64_t *rank,
                  gf2_mat *L, gf2_mat *E, unsigned flags,
                  void *workspace, size_t ws_bytes, void *stream);

/* gf2_decompose with per-call options (panel_w, table_c, tile_words; the
 * product fields are ignored).  Same outputs, bit for bit, for every
 * option. */
int gf2_decompose_ex(const gf2_mat *A, int32_t *perm, int32_t *pivcols, int64_t *rank,
                     gf2_mat *L, gf2_mat *E, unsigned flags, const gf2_opts *opts,
                     void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Autotuner of the decomposition (the paper tunes its block size b and
 * table size c by hand for one CPU, Sections 6.1 and 7).  Options that
 * change only speed -- panel_w 64 or 128 (Section 5's wide panel), table_c
 * 4 or 8 (Section 6), and for panel_w 128 the three schedules -- are timed
 * on the current device and the fastest is kept per (device, shape bucket).
 * The shape bucket of an n x m matrix is the pair of powers of two at or
 * above n and m (at least 64 each).  Every later gf2_decompose,
 * gf2_decompose_ex, gf2_rank, gf2_decompose_host or gf2_factors_decompose
 * call whose options leave panel_w, table_c and schedule at 0 (or NULL)
 * uses the entry of its bucket on its device, when there is one; options
 * never change a result.  The entries are process-wide, guarded by a lock;
 * gf2_tune_save / gf2_tune_load write and merge them as a JSON file:
 *   {"gf2_tune": 1, "entries": [{"device": "...", "kind": "decompose",
 *    "bucket_n": N, "bucket_m": M, "panel_w": .., "table_c": ..,
 *    "tile_words": .., "backend": .., "schedule": .., "strassen_cutoff": ..,
 *    "batched_c8_from": .., "ms": ..}, ...]}
 * (any key order and whitespace; a file of another shape is GF2_ERR_ARG and
 * loads nothing). */
#define GF2_TUNE_DECOMPOSE 0

typedef struct gf2_tune_entry {
    char device[64];   /* device key, as gf2_tune_device_key writes it (no quotes or backslashes) */
    int32_t kind;      /* GF2_TUNE_DECOMPOSE */
    int32_t reserved;  /* must be 0 */
    int64_t bucket_n;  /* shape bucket: powers of two >= 64 */
    int64_t bucket_m;
    gf2_opts opts;     /* the fastest options measured for the bucket */
    double ms;         /* their time, milliseconds per decomposition */
} gf2_tune_entry;

/* The key of the current device: its name, SM count and compute capability.
 * Errors: GF2_ERR_ARG (out NULL or len too small), GF2_ERR_CUDA. */
int gf2_tune_device_key(char *out, int64_t len);
/* Inserts an entry, replacing the one of the same device, kind and bucket.
 * Host only.  Errors: GF2_ERR_ARG (NULL, empty or unterminated device key,
 * a key with '"', '\\' or control characters, a bucket that is not a power of
 * two >= 64, reserved != 0, ms < 0, options gf2_opts_check rejects). */
int gf2_tune_put(const gf2_tune_entry *e);
/* The entry of (device, kind) for the bucket of n x m: *found = 1 and *out
 * filled, or *found = 0.  Host only.  Errors: GF2_ERR_ARG. */
int gf2_tune_lookup(const char *device, int32_t kind, int64_t n, int64_t m, gf2_tune_entry *out, int *found);
int64_t gf2_tune_count(void);
int gf2_tune_clear(void);
/* JSON file of every entry / merge of a file's entries (GF2_ERR_ARG when the
 * file cannot be opened or does not have the shape above). */
int gf2_tune_save(const char *path);
int gf2_tune_load(const char *path);
/* Times every candidate (3 untimed calls, then the best of 3, CUDA events on
 * `stream`) on a seeded uniform random n x m matrix made on the device, with
 * L and E when want_factors, and stores the fastest as the entry of the
 * bucket of n x m on the current device; *best receives it.  It allocates
 * the matrix, the outputs and a workspace, synchronises the stream and frees
 * them before it returns.  Errors: GF2_ERR_ARG (best NULL, n or m < 1 or
 * >= 2^31), GF2_ERR_NOMEM, GF2_ERR_TIMEOUT, GF2_ERR_CUDA. */
int gf2_decompose_autotune(int64_t n, int64_t m, int want_factors, gf2_tune_entry *best, void *stream);

/* Reduced row echelon form, in place (Gauss-Jordan: the paper names it
 * among the uses of the decomposition, Section 1, and leaves it to the
 * textbook).  E (k x m, column blocks, device) is an echelon factor as
 * gf2_decompose leaves it: row t has its leading one at pivcols[t] (device
 * int32[k], increasing) when pivcols[t] >= 0, and rows with pivcols[t] = -1
 * are zero.  E becomes R = U^-1 E, U = E restricted to the pivot columns
 * (unit upper triangular): every pivot column is then a unit column.  R is
 * the unique reduced form of the row space, whatever the pivot order.  An E
 * not in that form gives an unspecified result (it is not checked).
 * Asynchronous on `stream`; scratch from the workspace
 * (gf2_rref_workspace_bytes(k, m)) or, with workspace = NULL, from the
 * library's own.  Errors: GF2_ERR_ARG (E or pivcols null with k, m > 0),
 * GF2_ERR_SHAPE (ld < rows), GF2_ERR_NOMEM, GF2_ERR_UNSUPPORTED (k or
 * m >= 2^31), GF2_ERR_CUDA. */
size_t gf2_rref_workspace_bytes(int64_t k, int64_t m);
int gf2_rref(gf2_mat *E, const int32_t *pivcols, void *workspace, size_t ws_bytes, void *stream);

/* Null-space basis (Section 1 names it among the uses of the
 * decomposition): from the reduced row echelon form R (k x m, as gf2_rref
 * leaves E; device), its pivot columns (device int32, the first `rank`
 * entries increasing) and the rank (host value), the m x (m - rank) matrix
 * N (column blocks, device) whose columns are a basis of {x : A x = 0}:
 * column j belongs to the j-th free (non-pivot) column f_j, increasing --
 * N[f_j][j] = 1, N[pivcols[t]][j] = R[t][f_j], every other entry 0.  Given
 * R this basis is unique.  Asynchronous on `stream`; scratch: m - rank
 * int32 (gf2_nullspace_workspace_bytes; workspace = NULL: the library's).
 * Errors: GF2_ERR_ARG (null pointers, rank < 0 or > min(k, m)),
 * GF2_ERR_SHAPE (N not m x (m - rank), ld < rows), GF2_ERR_NOMEM,
 * GF2_ERR_UNSUPPORTED (m >= 2^31), GF2_ERR_CUDA. */
size_t gf2_nullspace_workspace_bytes(int64_t m, int64_t rank);
int gf2_nullspace(const gf2_mat *R, const int32_t *pivcols, int64_t rank, gf2_mat *N, void *workspace,
                  size_t ws_bytes, void *stream);

/* Rank of A (n x m) only: the decomposition without storing L and E
 * (Lemma 4.1: rank(A) = sum of the r_j).  A wide matrix (n < m) is ranked
 * through its transpose, formed in the workspace (rank(A) = rank(A^T); with
 * more rows than columns the decomposition takes fewer panels, Section 7).
 * rank_host receives the value; the call synchronises the stream.  Errors as
 * gf2_decompose. */
size_t gf2_rank_workspace_bytes(int64_t n, int64_t m);
int gf2_rank(const gf2_mat *A, int64_t *rank_host, unsigned flags,
             void *workspace, size_t ws_bytes, void *stream);
/* gf2_rank with per-call options (those of gf2_decompose_ex). */
int gf2_rank_ex(const gf2_mat *A, int64_t *rank_host, unsigned flags, const gf2_opts *opts,
                void *workspace, size_t ws_bytes, void *stream);

/* Rank of A (n x m, n <= 4096 and m <= 4096) without allocating anything.
 * No counterpart in the paper: this exists for callers that may not
 * allocate device memory when they call in -- for instance a program that
 * reserves a fixed device-memory budget at start-up and forbids allocations
 * afterwards, or a framework that owns every device buffer.  The scratch is
 * a static array of about 2.7 MiB inside the library (held by every GPU that
 * loads the library, until the process exits).  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress), so make the
 * first call before any stream capture.  Calls on one device share the
 * array: calls that overlap on the GPU race.  rank_dev: device int64 that
 * receives the rank (written asynchronously on `stream`, which the call
 * synchronises once to check the padding bits).  Runs the same kernels as
 * gf2_rank on the one stream given.  Errors: GF2_ERR_ARG, GF2_ERR_SHAPE,
 * GF2_ERR_UNSUPPORTED (n or m > 4096), GF2_ERR_PADDING, GF2_ERR_CUDA. */
int gf2_rank_noalloc(const gf2_mat *A, int64_t *rank_dev, void *stream);

/* Same as gf2_decompose, end to end from HOST memory: A_host holds the
 * column blocks (word (i,q) at A_host[q*lda + i]); the factors are copied
 * back to the host buffers given (L_host/E_host may be NULL; their column
 * blocks use ld = n and ld = min(n,m)).  Host buffers should be pinned for
 * full copy bandwidth.  Device memory comes from the workspace (see
 * gf2_decompose_host_workspace_bytes).  The padding bits are checked on the
 * host copy (GF2_ERR_PADDING before any device work).  Synchronises the
 * stream once, at the end. */
size_t gf2_decompose_host_workspace_bytes(int64_t n, int64_t m, int want_factors);
int gf2_decompose_host(int64_t n, int64_t m, const uint64_t *A_host, int64_t lda,
                       int32_t *perm_host, int32_t *pivcols_host, int64_t *rank_host,
                       uint64_t *L_host, uint64_t *E_host, unsigned flags,
                       void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Batched decomposition: `count` independent matrices, each decomposed as
 * gf2_decompose would (same pivot rule, same outputs, bit for bit), in one
 * persistent launch: one CTA factors one matrix at a time (Lemma 4.1 block by
 * block) and takes the next from a shared queue, largest work first.  Meant
 * for many small and medium systems (each n, m <= 4096).
 *   A[i]        n_i x m_i (column blocks, device; not modified)
 *   perm[i]     device int32[n_i]; pivcols[i] device int32[min(n_i, m_i)]
 *   rank        device int64[count]
 *   L, E        arrays of count descriptors as gf2_decompose (both or neither;
 *               NULL: rank, perm and pivcols only)
 * The descriptor arrays are read on the host during the call.  The call
 * synchronises the stream once (it reads the padding status back).  The
 * workspace depends on the table-size split (gf2_batched_set_c8_from):
 * size it after setting that.
 * Errors: GF2_ERR_ARG, GF2_ERR_SHAPE, GF2_ERR_PADDING, GF2_ERR_NOMEM,
 * GF2_ERR_UNSUPPORTED (a matrix with more than 4096 rows or columns),
 * GF2_ERR_CUDA.
 */
size_t gf2_decompose_batched_workspace_bytes(int count, const int64_t *n, const int64_t *m, int want_factors);
int gf2_decompose_batched(int count, const gf2_mat *A, int32_t *const *perm, int32_t *const *pivcols,
                          int64_t *rank, const gf2_mat *L, const gf2_mat *E, unsigned flags,
                          void *workspace, size_t ws_bytes, void *stream);
/* The same with per-call options (batched_c8_from); size the workspace with
 * gf2_decompose_batched_workspace_bytes_ex and the same options. */
size_t gf2_decompose_batched_workspace_bytes_ex(int count, const int64_t *n, const int64_t *m, int want_factors,
                                                const gf2_opts *opts);
int gf2_decompose_batched_ex(int count, const gf2_mat *A, int32_t *const *perm, int32_t *const *pivcols,
                             int64_t *rank, const gf2_mat *L, const gf2_mat *E, unsigned flags,
                             const gf2_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* The batched kernel's table size: matrices whose larger dimension is at
 * least c8_from use Four Russians tables of 8 bits (64 KB per CTA, three CTAs
 * per SM), the others tables of 4 bits (8 KB, four CTAs per SM); a batch with
 * both runs the two kernels side by side.  gf2_batched_autotune times both
 * on batches of square d x d matrices, d = 128, 256, ... up to max_dim (at
 * most 4096), and sets c8_from to the smallest d from which 8-bit tables are
 * faster there and at every larger d tried (2^62: never); *c8_from receives
 * it, and times_ms (may be NULL; 2 floats per d tried, smallest d first)
 * the measured batch times with 4- and 8-bit tables.  It allocates up to a
 * few GB, synchronises the stream and frees it all.  gf2_batched_set_c8_from sets it directly (default 1024).  A
 * process-wide setting.  Errors: GF2_ERR_ARG, GF2_ERR_NOMEM, GF2_ERR_CUDA. */
int gf2_batched_autotune(int64_t max_dim, int64_t *c8_from, float *times_ms, void *stream);
int gf2_batched_set_c8_from(int64_t dim);
int64_t gf2_batched_c8_from(void);

/* ------------------------------------------------------------------------
 * Linear systems A X = B over F2 from the factors of P*A = L*E (the use of
 * the decomposition in Section 1 of the paper; forward and back
 * substitution with the factors of Lemma 4.1).
 *   L, E, perm, pivcols, rank   exactly as gf2_decompose wrote them for an
 *           n x m matrix A (L is n x min(n,m), E is min(n,m) x m; device).
 *   B       n x nrhs, 1 <= nrhs <= 64: one column block, so row i of B is the
 *           word B->w[i] (bit c = right-hand side c).  Not modified.
 *   X       m x nrhs (one column block), receives the solutions: for every
 *           consistent right-hand side c, column c of X is the solution with
 *           every free variable (non-pivot column) 0; the column of an
 *           inconsistent right-hand side is 0.
 *   consistent  device uint64: bit c set iff A x = column c of B has a
 *           solution (bits >= nrhs are 0).
 * Steps: v = P B; forward substitution with the unit lower triangle of L
 * (rows < r); right-hand side c is consistent iff bit c of every residual
 * row r..n-1 is 0; back substitution with E at the pivot columns.
 * The call synchronises the stream once, to read the status of its bounded
 * device-side waits and of the padding check.
 * Errors: GF2_ERR_ARG (NULL, bad flag), GF2_ERR_SHAPE (nrhs outside 1..64,
 * X not m x nrhs, L or E not the sizes above), GF2_ERR_PADDING (a bit of B
 * at a column >= nrhs; checked unless GF2_NOCHECK), GF2_ERR_NOMEM,
 * GF2_ERR_UNSUPPORTED (n or m >= 2^31), GF2_ERR_TIMEOUT (a grid-wide wait
 * gave up; the outputs are then undefined), GF2_ERR_CUDA.
 */
size_t gf2_solve_workspace_bytes(int64_t n, int64_t m);
int gf2_solve(const gf2_mat *L, const gf2_mat *E, const int32_t *perm, const int32_t *pivcols,
              const int64_t *rank, const gf2_mat *B, gf2_mat *X, uint64_t *consistent,
              unsigned flags, void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Factor handle: the factors of one decomposition in device memory that the
 * handle owns (Lemma 4.1 and Figure 1: P, the pivot columns, L, E, and the
 * block form's per-block data -- Z, the within-block maps T_j and T_j^-1 --
 * which the handle keeps opaquely), with the scratch its calls need, so
 * that solves, reduced forms and null spaces take the handle instead of
 * loose arrays and use no shared workspace.
 *   n, m      the matrix size the handle was allocated for
 *   rank      host copy of the rank: -1 until gf2_factors_rank reads it
 *   perm      device int32[n]; pivcols device int32[min(n, m)]
 *   rank_dev  device int64, written by gf2_factors_decompose
 *   L, E      n x min(n, m) and min(n, m) x m column blocks in device
 *             memory (w = NULL with GF2_FACTORS_RANK_ONLY)
 *   flags     as given to gf2_factors_alloc
 *   impl      library-owned; do not touch
 * Calls on one handle must not overlap in time (issue them on one stream,
 * or wait between streams); calls on different handles may.
 * gf2_factors_alloc(F, n, m, flags): fills *F and allocates its device
 * memory (cudaMalloc; about the size of A for the scratch, plus L and E).
 *   GF2_ERR_ARG (F NULL, n or m < 0, unknown flag), GF2_ERR_UNSUPPORTED
 *   (n or m >= 2^31), GF2_ERR_NOMEM.
 * gf2_factors_free(F): releases it (waits for the device first) and zeroes
 *   *F; a zeroed handle frees as a no-op.  GF2_ERR_ARG for F NULL.
 * gf2_factors_decompose(F, A, flags, opts, stream): P*A = L*E of an n x m
 *   A into the handle, as gf2_decompose_ex (flags: GF2_NOCHECK).
 * gf2_factors_rank(F, rank_host, stream): synchronises the stream and reads
 *   the rank (also into F->rank).
 * gf2_factors_solve(F, B, X, consistent, flags, stream): as gf2_solve with
 *   the handle's factors (needs L and E).
 * gf2_factors_rref(F, R, stream): R (min(n, m) x m, the caller's) receives
 *   the reduced row echelon form of E; the handle is unchanged.
 * gf2_factors_nullspace(F, N, stream): N (m x (m - rank), the caller's)
 *   receives the null-space basis of gf2_nullspace; synchronises the stream
 *   once to read the rank, and the first call allocates the handle's copy
 *   of the reduced form (kept until gf2_factors_free).
 * Errors as the matching loose-array entry points, plus GF2_ERR_ARG for a
 * handle without L and E where they are needed, and GF2_ERR_SHAPE for a
 * matrix of another size than the handle's. */
#define GF2_FACTORS_RANK_ONLY 1u

typedef struct gf2_factors {
    int64_t n, m;
    int64_t rank;
    int32_t *perm;
    int32_t *pivcols;
    int64_t *rank_dev;
    gf2_mat L, E;
    uint32_t flags;
    void *impl;
} gf2_factors;

int gf2_factors_alloc(gf2_factors *F, int64_t n, int64_t m, unsigned flags);
int gf2_factors_free(gf2_factors *F);
int gf2_factors_decompose(gf2_factors *F, const gf2_mat *A, unsigned flags, const gf2_opts *opts, void *stream);
int gf2_factors_rank(gf2_factors *F, int64_t *rank_host, void *stream);
int gf2_factors_solve(const gf2_factors *F, const gf2_mat *B, gf2_mat *X, uint64_t *consistent, unsigned flags,
                      void *stream);
int gf2_factors_rref(const gf2_factors *F, gf2_mat *R, void *stream);
int gf2_factors_nullspace(gf2_factors *F, gf2_mat *N, void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request engine for rank and solve requests on many matrices
 * (the paper's use of the decomposition, Section 1: many systems over F2,
 * each factored once and then solved as right-hand sides arrive).  No
 * counterpart in the paper's code; the arithmetic is gf2_decompose's and
 * gf2_solve's, bit for bit.
 *
 * The engine runs on its own host thread.  Requests carry a matrix key; the
 * factors of a key stay resident in device memory (an arena of
 * `device_bytes`, least recently used factors evicted first when room is
 * needed) so that later requests on the same key only solve.  Continuous
 * batching: a request is admitted once it has arrived and its memory fits;
 * misses are decomposed (several small matrices, up to 512 x 512, together
 * in one batched launch, the others by the plain decomposition, up to four
 * side by side); every solve whose factors
 * are ready joins the next solve launch, one CTA per request, while up to
 * four earlier launches are still on the GPU.  Each CTA writes its results
 * to mapped host memory and raises a per-request flag, so a request is
 * complete as soon as its own CTA is done.
 * GF2_SERVE_SERIAL: one request at a time through gf2_decompose and
 * gf2_solve, waiting for each (the one-at-a-time baseline), same residency.
 */
#define GF2_SERVE_SERIAL 1u

typedef struct gf2_server gf2_server;

typedef struct gf2_request {
    uint64_t id;          /* caller's tag, returned in the completion                     */
    uint64_t matrix;      /* key: requests with the same key share resident factors and
                             must give the same n, m (and the same A)                     */
    int64_t n, m;         /* size of A, 1 <= n, m <= the server's limits                  */
    const uint64_t *A;    /* HOST column blocks of A (word (i,q) at A[q*lda + i], padding
                             bits 0); read only when the key's factors are not resident   */
    int64_t lda;          /* >= n                                                         */
    int32_t nrhs;         /* 0: rank only; 1..64: solve A X = B                            */
    const uint64_t *B;    /* HOST, n words, bit c = right-hand side c (bits >= nrhs 0)     */
    uint64_t *X;          /* HOST, m words out: the solutions as gf2_solve gives them      */
    double arrival_us;    /* earliest admission on the server clock (0: on submission)     */
} gf2_request;

typedef struct gf2_completion {
    uint64_t id;
    int32_t status;       /* GF2_OK or the error of this request                          */
    int32_t hit;          /* 1: the factors were resident (or being built) on admission   */
    int64_t rank;
    uint64_t consistent;  /* bit c: right-hand side c has a solution                      */
    double arrival_us;    /* max(arrival_us, submission time)                              */
    double admit_us, done_us;
} gf2_completion;

typedef struct gf2_server_stats {
    int64_t completed, hits, misses, evictions;
    int64_t solve_launches, batched_decompositions, plain_decompositions;
    int64_t max_batch, resident_bytes, arena_bytes;
    int64_t admitted_in_flight;   /* requests admitted while a launch of the engine was on the GPU */
    int64_t overlapped_launches;  /* solve launches enqueued while another launch was on the GPU   */
} gf2_server_stats;

/* Creates an engine on the current device.  device_bytes: the device memory
 * for factors, staging and solve scratch (one eighth of it, at most 1 GiB,
 * is kept for the solve launches); max_n, max_m: the largest matrix
 * accepted (a plain-decomposition workspace of that size is kept outside the
 * arena); max_batch: solves per launch (<= 4096).
 * Errors: GF2_ERR_ARG, GF2_ERR_NOMEM, GF2_ERR_CUDA. */
int gf2_server_create(int64_t device_bytes, int64_t max_n, int64_t max_m, int max_batch, unsigned flags,
                      gf2_server **out);
/* Queues `count` requests (descriptors copied; the host buffers A, B, X must
 * stay valid until the request completes).  A request that is malformed
 * (sizes, nrhs, padding bits of A or B, a key reused with another size)
 * completes at once with its error.  Thread-safe.  Errors: GF2_ERR_ARG. */
int gf2_server_submit(gf2_server *server, const gf2_request *requests, int count);
/* Moves up to `max` completions to `out` (*count of them), waiting up to
 * wait_us microseconds for the first one (0: no wait).  Thread-safe. */
int gf2_server_poll(gf2_server *server, gf2_completion *out, int max, int64_t wait_us, int *count);
/* The server clock: microseconds since gf2_server_create. */
double gf2_server_clock_us(const gf2_server *server);
int gf2_server_stats_read(const gf2_server *server, gf2_server_stats *stats);
/* Finishes every request already submitted, then frees the engine. */
int gf2_server_destroy(gf2_server *server);

/* ------------------------------------------------------------------------
 * Diagnostics (no counterpart in the paper; used by the benchmark).
 * gf2_launch_count: kernels this library has launched since it was loaded.
 * gf2_timing_enable(1): from now on every launch is bracketed by CUDA events
 *   recorded on the launch's own stream, grouped by kernel class
 *   (GF2_KCLASS_*).  gf2_timing_read synchronises on the last event and
 *   returns the summed device time in ms and the number of launches of one
 *   class since the last gf2_timing_reset.  Host-side state is guarded by a
 *   mutex; the events are created on the current device.
 */
#define GF2_KCLASS_PANEL 0   /* pivot selection + pseudo-inverse (buildZ)     */
#define GF2_KCLASS_NEXT 1    /* Y = D Z, L multipliers, next column tile     */
#define GF2_KCLASS_UPDATE 2  /* wide trailing update / product pass (M4RM)   */
#define GF2_KCLASS_LAYOUT 3  /* layout conversions and final outputs         */
#define GF2_KCLASS_SOLVE 4   /* forward / back substitution (gf2_solve)      */
#define GF2_KCLASS_FACTOR 5  /* the whole decomposition in one persistent launch */
#define GF2_NUM_KCLASSES 6
int64_t gf2_launch_count(void);
int gf2_timing_enable(int on);
int gf2_timing_reset(void);
int gf2_timing_read(int kernel_class, double *total_ms, int64_t *launches);

/* ------------------------------------------------------------------------
 * Operation counts (the cost model of Section 6 and of the complexity
 * estimate of Section 7).  Only the op-counting build of the library
 * (compiled with -DGF2_COUNT_OPS, a separate libgf2_count.so) counts; the
 * release build returns GF2_ERR_UNSUPPORTED and has no counting code in its
 * kernels.
 *
 * Every count is in operations on 64-bit words (the paper's Xor_b, b = 64):
 *   GF2_OP_UPDATES     (panel, row, word) triples of the trailing update
 *                      A(j+1) = E + Y C: a word of a row below panel j's
 *                      pivots that receives panel j's update (rows whose
 *                      multiplier y is zero take none)
 *   GF2_OP_YROWS       rows whose multiplier y = d Z is formed (Y = D Z)
 *   GF2_OP_LOOKUPS8    table lookups XORed into a word, c = 8 tables (the
 *                      wide update)
 *   GF2_OP_LOOKUPS4    the same, c = 4 tables (the look-ahead update, and
 *                      the one-panel wide update of fewer than 4096 rows)
 *   GF2_OP_TABLE8      table entries x != 0 formed, per word, c = 8 tables
 *   GF2_OP_TABLE4      the same, c = 4 tables
 *   GF2_OP_MMM_LOOKUPS the product's table lookups (c = 8) XORed into a word
 *   GF2_OP_MMM_TABLE   the product's table entries x != 0 formed, per word
 *   GF2_OP_MMM_ADDS    words of the explicit matrix additions of the
 *                      Strassen-Winograd recursion
 * Words past the last column block (tile padding) are not counted.  The
 * update and lookup counts take each (panel, row, word) once, also where
 * several CTAs that share a column tile each redo the update of the second
 * panel's pivot rows of a pair; the table counts take every copy that a CTA
 * builds for itself.
 *
 * gf2_op_counts(out, count, reset): synchronises the current device, writes
 * min(count, GF2_NUM_OPS) counters to out (host memory) and, when reset is
 * nonzero, sets them to zero.  Returns GF2_OK, GF2_ERR_ARG (out null or
 * count < 0), GF2_ERR_UNSUPPORTED (release build) or GF2_ERR_CUDA.
 */
#define GF2_OP_UPDATES 0
#define GF2_OP_YROWS 1
#define GF2_OP_LOOKUPS8 2
#define GF2_OP_LOOKUPS4 3
#define GF2_OP_TABLE8 4
#define GF2_OP_TABLE4 5
#define GF2_OP_MMM_LOOKUPS 6
#define GF2_OP_MMM_TABLE 7
#define GF2_OP_MMM_ADDS 8
#define GF2_NUM_OPS 9
int gf2_op_counts(uint64_t *out, int count, int reset);

/* Device timeline of the decomposition's kernels, in the trace build only
 * (libgf2_trace.so, compiled with -DGF2_TRACE; the kernels read the GPU's
 * global timer).  No counterpart in the paper: it measures where the time
 * of the serial panel chain goes.  Per panel j < 4096 it keeps thirteen
 * nanosecond stamps, slot-major (out[slot * 4096 + j]):
 *   0 panel kernel released, 1 its rows loaded and the previous panel's
 *   update applied, 2 pivot loop done, 3 coordinate maps written (end),
 *   4 / 5 first start / last end of the look-ahead kernel of panel j,
 *   6 / 7 first start / last end of the trailing update(s) of panel j (a
 *   pair's update is filed under its second panel), and the panel's end
 *   phase step by step: 8 U^-1 and Comp done, 9 T done, 10 T^-1 done,
 *   11 Zp done (before the stores), and 12 panel kernel entered (before
 *   it waits for the previous panel; separate launches only).
 * 0 = not recorded.  The panel stamps are overwritten by every run; the
 * launch spans accumulate (earliest start, latest end) until a read with
 * reset = 1 clears every stamp, so clear them right before the
 * decomposition to trace.  gf2_trace_read(out, count,
 * reset) synchronises the current device and writes min(count, 13 * 4096)
 * values.  Returns GF2_OK, GF2_ERR_ARG (out null or count < 0),
 * GF2_ERR_UNSUPPORTED (every other build) or GF2_ERR_CUDA. */
/* The number of polls after which a bounded device-side wait gives up
 * (the grid-wide barriers of gf2_solve, the progress counters of the
 * persistent decomposition), for every later call in the process; 0
 * restores each wait's default (about a second).  No counterpart in the
 * paper: it exists so that a test can make a wait run out (GF2_ERR_TIMEOUT
 * from gf2_solve; rank -1 and GF2_ERR_TIMEOUT from the calls that read the
 * rank of a persistent decomposition) and check that the GPU context stays
 * usable.  Errors: GF2_ERR_ARG (polls < 0 or >= 2^32). */
int gf2_debug_set_wait_limit(int64_t polls);

#define GF2_TRACE_PANELS 4096
#define GF2_TRACE_SLOTS 12
int gf2_trace_read(uint64_t *out, int64_t count, int reset);

#ifdef __cplusplus
}
#endif

#endif /* GF2_H */
