// Internal declarations shared by the CUDA translation units of the F2
// library.  Nothing here is part of the C ABI (include/gf2.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gf2 {

// Words of one column tile of the working copy (32 bytes of a row); a lane
// of the trailing update owns one 128-bit word pair of a row's tile, so a
// warp covers 16 rows of a tile.
constexpr int kTileWords = 4;
// Y buffers and active lists kept per panel, cyclically: an update may still
// read those of panel j while the look-ahead kernels of panels up to j + 5
// write theirs
constexpr int kRing = 8;
constexpr int kLanesPerRow = kTileWords / 2;
constexpr int kRowsPerWarp = 32 / kLanesPerRow;
// Four Russians table width c (Section 6 of the paper): a 64-bit multiplier
// is split into 8 chunks of 8 bits, each looked up in a 256-entry table.
constexpr int kTableBits = 8;
constexpr int kNumTables = 64 / kTableBits;
constexpr int kPanelThreads = 128;

// Everything one column block ("panel" j, 64 columns) of the decomposition
// leaves for the kernels that follow it.  Coordinates: the r pivot rows of
// the panel are B_0..B_{r-1} (raw panel words, in pivot order) and their
// echelon forms E_0..E_{r-1} (E_s = B_s reduced by E_0..E_{s-1}).
//   For any panel word d in the row space of the panel:
//     y(d)      = XOR_{bits p of d} Zp[p]   -> d = sum_s y_s B_s   (Y = D Z)
//     lambda(d) = XOR_{bits p of d} Comp[p] -> d = sum_s lambda_s E_s
//   Tinv[s] = coordinates of E_s in the B_s   (row s of T^-1)
//   T[s]    = coordinates of B_s in the E_s   (row s of T, unit lower)
struct PanelInfo {
    int32_t R;          // first pivot position of the panel (R_j)
    int32_t r;          // pivots found in the panel (r_j)
    int32_t pivbit[64]; // bit (column within the panel) of pivot s
    uint64_t Zp[64];
    uint64_t Comp[64];
    uint64_t Tinv[64];
    uint64_t T[64];
    uint64_t Erow[64];  // E_s restricted to the panel's 64 columns
    int32_t prow[64];   // storage row of pivot s
};

// Device state of one decomposition.  W is a working copy of A: storage
// row i is row i of A and never moves; perm maps positions to storage rows
// (row i of P*A is storage row perm[i]), so a row exchange is an exchange of
// two perm entries and no data moves.  W is TILED by column tiles of
// kTileWords words: tile T holds words 4T..4T+3 of every storage row, row
// after row (32 contiguous bytes per row), so word q of row i is at
//   W[(q / 4) * tstride + 4 * i + q % 4],   tstride = 4 * n.
// A warp that updates 16 consecutive rows of a tile touches 512 contiguous
// bytes.
struct DecompCtx {
    uint64_t *W;
    int64_t tstride;    // words from one column tile of W to the next (kTileWords * n)
    int64_t lde;        // words per row of Eint, a multiple of kTileWords
    int32_t *perm;      // [n] position -> storage row (the output perm)
    int32_t *pivcols;   // [k]
    PanelInfo *info;    // [mu]
    uint64_t *Y;        // [kRing][n] per storage row: y of panel j in Y[j % kRing]; 0 for pivot rows
    uint64_t *F;        // [2][n] per storage row: its word j with every panel < j applied, in F[j % 2]
                        // (j >= 1; written by the look-ahead kernel of panel j-1; word j of W
                        // itself never receives panel j-1's update)
    int32_t *pivpanel;  // [n] per storage row: panel where it became a pivot (INT32_MAX: not yet)
    int32_t *act;       // [kRing][n] act[j % kRing]: the storage rows that are not pivots of panels <= j
                        // (ascending within each 256-entry piece), written by the look-ahead of panel j
    int32_t *nact;      // [mu] number of entries of act after panel j (zero before the run)
    int32_t *orw;       // [mu] set by the look-ahead of panel j-2 after a rank-deficient panel: bit 1 =
                        // looked, bit 0 = some row not a pivot of panels <= j-2 has a nonzero word j
                        // after the updates of panels <= j-2 (zero before the run); or null.  With
                        // r_{j-1} = 0, orw[j] == 2 means panel j has no pivot
    uint64_t *Lint;     // [n x ldl] per storage row, or null (rank only)
    int64_t ldl;
    uint64_t *Eint;     // [k x lde] per pivot index (row-major), or null
    int32_t n, m, mu, kmax;
    int32_t *zpos;      // [n] the panel's list of nonzero rows behind its window (positions), or null
    uint64_t *zraw;     // [n] their raw panel words (both null: the panel scans without a list)
    int32_t pair;       // wide updates by pairs of panels (j even, j+1)
    int32_t info_ring;  // info holds only panels j-1 and j (info[j % 2]): the batched form
    int32_t tab_c;      // table bits of the wide updates: 4, 8, or 0 (8; 4 for one panel with < 4096 rows)
    const int32_t *fail;  // nonzero after the run: a bounded device wait gave up (the rank reads -1); or null
};

// The PanelInfo of panel j.
__device__ __forceinline__ PanelInfo *panel_info(const DecompCtx &c, int j)
{
    return c.info + (c.info_ring ? (j & 1) : j);
}

// Index of word q of storage row i in the tiled W.
__device__ __forceinline__ int64_t widx(const DecompCtx &c, int64_t i, int q)
{
    return (int64_t)(q / kTileWords) * c.tstride + i * kTileWords + (q % kTileWords);
}

// Row-major operands of a product C ^= A * B over F2 for one 64-row slice
// of B (k-block kb): the multiplier of row i is word kb of A's row i.
// Operands of a product C (+)= A B over F2, all in column blocks (word (i, q)
// at X[q*ld + i]): A is n x k, B is k x (64 mw), C is n x (64 mw).
struct MmmCtx {
    const uint64_t *A; int64_t lda;
    const uint64_t *B; int64_t ldb;
    uint64_t *C; int64_t ldc;
    int32_t n, k, mw;
    int32_t mode;                     // kMmmStore, kMmmXor or kMmmAtomicXor
};
constexpr int kMmmStore = 0;      // C = A B
constexpr int kMmmXor = 1;        // C ^= A B
constexpr int kMmmAtomicXor = 2;  // C ^= A B by atomics (the inner dimension split over CTAs)

// One matrix of a batched decomposition (the caller's buffers; column blocks).
struct BatchItem {
    const uint64_t *A; int64_t lda;
    int32_t n, m;
    int32_t *perm, *pivcols;
    int64_t *rank;
    uint64_t *L; int64_t ldl;   // null: rank only
    uint64_t *E; int64_t lde;
};

// A batched decomposition: the items, the order in which CTAs take them, and
// one scratch slice per CTA (offsets in words within a slice).
struct BatchCtx {
    const BatchItem *items;
    const int32_t *order;       // items by decreasing work
    int32_t *next_item;         // shared counter (zero before the launch)
    uint32_t *err;              // padding flag
    uint64_t *scratch;
    int64_t scratch_words;      // per CTA
    int64_t off_y, off_info, off_pivpanel, off_lint, off_eint;
    int32_t count, factors, check;
};

// Operands of a solve A X = B from the factors P*A = L*E (column blocks).
struct SolveCtx {
    const int32_t *perm, *pivcols;
    const int64_t *rank;
    const uint64_t *L; int64_t ldl;   // n x min(n,m)
    const uint64_t *E; int64_t lde;   // min(n,m) x m
    const uint64_t *B;                // [n] right-hand sides, bit c = column c
    uint64_t *X;                      // [m] solutions
    uint64_t *consistent;             // one word: bit c = right-hand side c is consistent
    uint64_t rhs_mask;                // the nrhs low bits
    uint64_t *v;                      // [n] P*B, then the residual rows
    uint64_t *y;                      // [min(n,m)] forward result, then back-substitution state
    uint64_t *linv;                   // [ceil(min(n,m)/64)][64] inverse diagonal blocks of L (rows)
    uint64_t *uinv;                   // [ceil(m/64)][64] inverse diagonal blocks of E at its pivots
    int32_t *qstart;                  // [ceil(m/64)+1] first pivot whose column is >= 64q
    uint32_t *sync;                   // [2] barrier count, error bits (1 wait gave up, 2 padding)
    uint64_t *bad;                    // one word: OR of the residual rows
    int32_t n, m;
    int32_t check;                    // report right-hand-side bits beyond nrhs
    uint32_t wait_limit;              // polls after which a grid-wide wait gives up
};

// One solve of a serving batch: the operands, where its rank goes and the
// word that is set once its outputs are written (both may be mapped host
// memory).  nrhs == 0: the rank alone.
struct ServeItem {
    SolveCtx c;
    int64_t *rank_out;
    uint32_t *done;
    int32_t nrhs;
};

// ---- launchers (each returns the cudaError_t of its launch)
cudaError_t launch_ingest(const uint64_t *A, int64_t lda, int32_t n, int32_t mu, uint64_t last_mask,
                          uint64_t *W, int64_t ldw, int32_t *perm_identity, int32_t *pivpanel_init,
                          uint32_t *err, cudaStream_t s);  // row-major W (ldw words per row)
cudaError_t launch_ingest_tiled(const uint64_t *A, int64_t lda, int32_t n, int32_t mu, uint64_t last_mask,
                                uint64_t *W, int32_t *perm_identity, int32_t *pivpanel_init, uint32_t *err,
                                cudaStream_t s);  // tiled W (see DecompCtx), words up to a multiple of 8
cudaError_t launch_colblocks_from_rowmajor(const uint64_t *R, int64_t ldr, const int32_t *row_of,
                                           int32_t rows, int32_t words, uint64_t *out, int64_t ldo,
                                           cudaStream_t s);
cudaError_t launch_finish_E(const DecompCtx &c, uint64_t *E, int64_t lde, cudaStream_t s);
cudaError_t launch_finish_scalars(const DecompCtx &c, int64_t *rank, cudaStream_t s);
cudaError_t launch_panel(const DecompCtx &c, int j, cudaStream_t s);
// The factorization (pairs of panels) from panel j_start (even) on in one
// cooperative persistent launch (csrc/k_factor.cu): the panels before it,
// their look-aheads and pair updates done; `progress` is
// factor_progress_ints(mu) int32 of device memory, set up by
// launch_factor_init on the same stream; it receives the run's failure word
// (c.fail points into it).  Returns cudaErrorNotSupported when the kernel
// cannot have one CTA resident on every SM.
int64_t factor_progress_ints(int mu);
cudaError_t launch_factor_init(int32_t *progress, int mu, int j_start, cudaStream_t s);
cudaError_t launch_factor(const DecompCtx &c, int32_t *progress, int j_start, cudaStream_t s);
cudaError_t factor_available();  // cudaErrorNotSupported: the device cannot hold one CTA per SM
// The polls after which a bounded device wait gives up: the value set by
// gf2_debug_set_wait_limit, else `dflt` (csrc/gf2_api.cu).
int64_t device_wait_limit(int64_t dflt);
const int32_t *factor_fail_word(const int32_t *progress);
cudaError_t launch_next(const DecompCtx &c, int j, cudaStream_t s);
// the wide update of panel j (np = 1) or of the pair j, j+1 (np = 2)
// the wide update of panel j (np = 1) or of panels j, j+1 (np = 2) on its
// tiles from the skip-th on, at most limit of them
cudaError_t launch_rest(const DecompCtx &c, int j, int np, int est_active_rows, cudaStream_t s, int skip = 0,
                        int limit = 1 << 30);
int rest_tiles(const DecompCtx &c, int j, int np, int *tile_first);
cudaError_t prepare_update_kernels();  // one-time kernel attributes (before any capture)
cudaError_t prepare_panel_kernel();
// the Four Russians product (csrc/k_mmm.cu); with mode kMmmStore or kMmmXor
// the launch may split the inner dimension (then C is zeroed first for
// kMmmStore and updated by atomics)
cudaError_t launch_mmm(MmmCtx c, cudaStream_t s);
// D = X ^ Y over rows x words (column blocks; D may be X)
cudaError_t launch_xor(uint64_t *D, int64_t ldd, const uint64_t *X, int64_t ldx, const uint64_t *Y, int64_t ldy,
                       int64_t rows, int64_t words, cudaStream_t s);
cudaError_t launch_solve(const SolveCtx &c, cudaStream_t s);  // one cooperative launch
// one CTA per item, items[0] first; max_n: the largest n among the items
cudaError_t launch_serve_solve(const ServeItem *items, int count, int32_t *next, int64_t max_n, cudaStream_t s);
// large systems: one cluster of kServeClusterCTAs CTAs per item (items[0 ..
// count)); max_n the largest n
constexpr int kServeClusterCTAs = 8;
bool serve_by_cluster(int64_t n);
cudaError_t launch_serve_cluster(const ServeItem *items, int count, int64_t max_n, cudaStream_t s);
int batch_ctas_per_sm(int c);  // c = 4 or 8: the batched kernel's table size
// the product on the tensor cores (k < 2^24, csrc/k_umma.cu): A8 = A and
// B8 = B^T as e2m1 entries 0 / 1.0, K contiguous, n_pad and m_pad rows of
// mma_row_bytes(k_pad) bytes (dimensions rounded up to mma_pad)
int64_t mma_pad(int64_t x);
int64_t mma_row_bytes(int64_t k_pad);  // bytes of one expanded operand row of k_pad entries
cudaError_t launch_expand_operands(const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb, int n, int k, int m,
                                   uint8_t *A8, uint8_t *B8, cudaStream_t s);
// the tcgen05 product from the expanded operands; err: ORed with 1 when a
// device wait gave up
cudaError_t launch_umma_product(const uint8_t *A8, const uint8_t *B8, int n_pad, int m_pad, int k_pad, uint64_t *C,
                                int64_t ldc, int n, int m, int accumulate, uint32_t *err, cudaStream_t s);
// the tensor pipe's kind::f8f6f4 rate: ctas CTAs issue iters x 4 MMAs of
// 128 x 256 x 32 each (umma_peak_flops_per_iter() flops per iteration)
cudaError_t launch_umma_peak(int ctas, int iters, uint32_t *err, cudaStream_t s);
double umma_peak_flops_per_iter();
// rows words of the last column block with a bit outside mask -> *err |= 1
cudaError_t launch_check_last_block(const uint64_t *last, int rows, uint64_t mask, uint32_t *err, cudaStream_t s);
cudaError_t launch_batch(const BatchCtx &b, int grid, int c, cudaStream_t s);
// T = A^T for A n x m in column blocks (T: m x n, ld ldt >= m; csrc/k_transpose.cu)
cudaError_t launch_transpose_bits(const uint64_t *A, int64_t lda, int64_t n, int64_t m, uint64_t *T, int64_t ldt,
                                  cudaStream_t s);
// the reduced row echelon form (csrc/k_rref.cu): every 64-row block of E
// (k x m) reduced by its own pivot columns (V: 64 ceil(k/64) words of
// scratch), and the bits of rows [a, a+rows) at the columns
// pivcols[c0 .. c0+ncols) as column blocks
cudaError_t launch_rref_diag(uint64_t *E, int64_t ld, const int32_t *pivcols, int64_t k, int64_t m, uint64_t *V,
                             cudaStream_t s);
cudaError_t launch_gather_cols(const uint64_t *E, int64_t ld, int64_t m, const int32_t *pivcols, int64_t a, int64_t rows,
                               int64_t c0, int64_t ncols, uint64_t *out, int64_t ldo, cudaStream_t s);
// the null-space basis N (m x (m - r), ld ldn) from R and its r pivot
// columns (free: m - r int32 of scratch)
cudaError_t launch_nullspace(const uint64_t *R, int64_t ldr, const int32_t *pivcols, int64_t r, int64_t m, int32_t *free,
                             uint64_t *N, int64_t ldn, cudaStream_t s);

// ---- host helpers shared by the entry points (gf2_api.cu)
// the batched decomposition of checked items (each n, m <= 4096); with
// GF2_NOCHECK it does not synchronise the stream
size_t decompose_batched_items_bytes(int count, const BatchItem *items, bool factors);
int decompose_batched_items(int count, const BatchItem *items, bool factors, unsigned flags, void *workspace,
                            size_t ws_bytes, void *stream);
void add_launches(int64_t k);  // kernels launched outside the entry points' own counting

// ---- operation counters of the op-counting build (-DGF2_COUNT_OPS; the
// counter kinds are GF2_OP_* of include/gf2.h).  Each translation unit with
// counted kernels keeps its own device array (no relocatable device code)
// and adds it into acc (GF2_NUM_OPS entries) from the host.
enum OpKind {
    kOpUpdates = 0,
    kOpYRows = 1,
    kOpLookups8 = 2,
    kOpLookups4 = 3,
    kOpTable8 = 4,
    kOpTable4 = 5,
    kOpMmmLookups = 6,
    kOpMmmTable = 7,
    kOpMmmAdds = 8,
    kNumOps = 9
};
// ---- device timeline of the trace build (-DGF2_TRACE; gf2_trace_read of
// include/gf2.h): globaltimer stamps (ns) per panel j, slot-major
// ([slot][j], kTraceMaxPanels entries per slot).  Panel phases come from the
// CTA's thread 0; a multi-CTA launch keeps the earliest start (atomicMin)
// and the latest end (atomicMax) over its CTAs' threads 0.  Each translation
// unit with traced kernels keeps its own array and the host merges them
// (panels: csrc/k_panel.cu, look-ahead and updates: csrc/k_update.cu).
constexpr int kTraceMaxPanels = 4096;
enum TraceSlot {
    kTrPanelStart = 0,  // panel kernel released (after griddepcontrol.wait)
    kTrPanelLoaded = 1, // its rows loaded and the previous panel's update applied (fast path ready)
    kTrPanelLoop = 2,   // pivot loop and exchanges done
    kTrPanelEnd = 3,    // coordinate maps written (end of the kernel)
    kTrNextStart = 4,
    kTrNextEnd = 5,
    kTrRestStart = 6,   // every update launch of panel j (pair: j = the second panel)
    kTrRestEnd = 7,
    // the panel's end phase, step by step (between kTrPanelLoop and kTrPanelEnd)
    kTrPanelUinv = 8,   // U^-1 (backward sweep) and Comp
    kTrPanelT = 9,      // T = lambda(B)
    kTrPanelTinv = 10,  // T^-1 (backward sweep)
    kTrPanelZp = 11,    // Zp = Comp T^-1 (before the stores)
    kTrPanelEntry = 12, // panel kernel entered (before griddepcontrol.wait)
    kTrSlots = 13
};
__host__ __device__ constexpr bool trace_panel_slot(int slot) { return slot <= kTrPanelEnd || slot >= kTrPanelUinv; }
#ifdef GF2_TRACE
#define GF2_TR(...) __VA_ARGS__
__device__ __forceinline__ unsigned long long trace_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Start and end of one launch: thread 0 of every CTA keeps the earliest
// start (stored complemented, so that both slots take atomicMax from zero)
// and, when it leaves the kernel by any return, the latest end.
struct TraceSpan {
    unsigned long long *end_slot;
    __device__ TraceSpan(unsigned long long *start_slot, unsigned long long *end) : end_slot(end)
    {
        if (threadIdx.x == 0) atomicMax(start_slot, ~trace_clock());
    }
    __device__ ~TraceSpan()
    {
        if (threadIdx.x == 0) atomicMax(end_slot, trace_clock());
    }
};
cudaError_t read_panel_trace(unsigned long long *out, bool reset);   // csrc/k_panel.cu
cudaError_t read_update_trace(unsigned long long *out, bool reset);  // csrc/k_update.cu
cudaError_t read_factor_trace(unsigned long long *out, bool reset);  // csrc/k_factor.cu
#else
#define GF2_TR(...)
#endif

#ifdef GF2_COUNT_OPS
#define GF2_OPS(...) __VA_ARGS__
cudaError_t read_update_ops(unsigned long long *acc, bool reset);  // csrc/k_update.cu
cudaError_t read_factor_ops(unsigned long long *acc, bool reset);  // csrc/k_factor.cu
cudaError_t read_mmm_ops(unsigned long long *acc, bool reset);     // csrc/k_mmm.cu
#else
#define GF2_OPS(...)
#endif

}  // namespace gf2
