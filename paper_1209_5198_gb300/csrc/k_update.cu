// Trailing update A(j+1) = E xor Y C (eq. (Aj) of the paper) by the Method
// of Four Russians (M4RM, Section 6): the r <= 64 pivot rows C of panel j
// are combined, per 4-word column tile, into 64/c tables of 2^c entries (one
// XOR per entry), and every other row then takes 64/c table lookups and
// XORs per word, indexed by the c-bit chunks of its multiplier y.
//
// Two kernels per panel:
//   k_next  y = d Z and lambda = d Comp for every row (d = the row's word in
//           column j; Y is kept per storage row for k_rest), the L
//           multipliers, word j+1 of every row with panel j applied (into a
//           side buffer F, not into W) and the tile holding word j+2;
//           it runs next to the panel kernel of block j+1.
//   k_rest  every column tile after that one; persistent (one CTA per SM),
//           each CTA takes a contiguous range of (tile, row chunk) items and
//           rebuilds its tables only when the tile changes.
// Rows are visited in STORAGE order (tiled W, storage row = row of A), from
// a list of the rows that are not pivots yet, which the look-ahead kernel
// compacts panel by panel; the multiplier array is indexed by storage row,
// so no position->row indirection sits in the hot loop.
//
// GB300 layout choices: W is stored by 4-word column tiles, each tile
// contiguous over the rows, so one row's tile is 32 contiguous bytes and 16
// consecutive rows of a tile are 512; a warp covers 16 rows x 4 words with
// 128-bit accesses (lane = row slot (lane/2) x word pair (lane%2)); the
// tables sit in shared memory as [table quad][x][quarter][4 words], and the
// four rows of a quarter-warp (one 128-bit shared-memory phase) read tables
// g, g^1, g^2, g^3, which live in the four 32-byte quarters of the bank
// space, so lookups are conflict-free for any y.
#include <mutex>

#include "update_core.cuh"

namespace gf2 {
namespace {

#ifdef GF2_TRACE
__device__ unsigned long long g_update_trace[kTrSlots * kTraceMaxPanels];  // the trace build's launch spans
#endif

// -------------------------------------------------------------------- k_next
// The look-ahead of panel j (next_body, csrc/update_core.cuh), one chunk of
// 256 rows per CTA.
constexpr int kNextThreads = 256;
constexpr int kNextRows = 256;  // storage rows per CTA (one wave next to the k_rest CTAs)

// <= 64 registers: a 256-thread CTA fits next to a persistent 512 x 96 k_rest CTA
__global__ void __launch_bounds__(kNextThreads, 4) k_next(DecompCtx c, int j)
{
    __shared__ __align__(16) uint64_t smem[kNextSmemWords];
    __shared__ int keep_row[kNextRows];  // the rows that stay active, by list entry
    __shared__ int keep_warp[kNextThreads / 32 + 1];
    GF2_TR(const int jt = j < kTraceMaxPanels ? j : kTraceMaxPanels - 1;
           TraceSpan span(g_update_trace + kTrNextStart * kTraceMaxPanels + jt,
                          g_update_trace + kTrNextEnd * kTraceMaxPanels + jt);)
    next_body<kNextThreads, kNextRows>(c, j, blockIdx.x, smem, keep_row, keep_warp);
}

// -------------------------------------------------------------------- k_rest
// The wide update of panel j (NP = 1) or of the pair j, j+1 (NP = 2) on the
// tiles [tile_first, tile_first + ntiles): persistent (one CTA per SM but
// one); each CTA takes a contiguous range of (tile, 256-entry chunk of the
// active list) items and builds its tables once per tile.
constexpr int kRestThreads = 512;
constexpr int kRestU = 6;   // row groups of 16 rows per warp and iteration (one panel)
constexpr int kRest2U = 4;  // the same for a pair
constexpr int kRestHeadU = 1;  // the same for a pair's one-tile head launch (256-row items: every warp busy)
constexpr int kRestHeadMinRows = 16384;  // rows below the pair from which a head runs with kRestHeadU

template <int C, int U, int NP>
// at most 96 registers: 512 x 96 leaves room on the SM for a k_next CTA
// (256 x 64) next to this persistent CTA
__global__ void __maxnreg__(96) k_rest(DecompCtx c, int j, int tile_first, int ntiles)
{
    static_assert(NP == 1 || NP == 2, "one panel or a pair");
    static_assert(C == 4 || C == 8, "4- or 8-bit tables");
    // a programmatic dependent of the previous update on this stream: wait
    // for it to complete (and its writes to be visible), then let the next
    // one be scheduled
    // The panels' results and the active list come from kernels of the
    // other streams, which this launch waits for in full: they are read
    // before the wait.
    const PanelInfo *pi0 = c.info + j;
    const PanelInfo *pi1 = c.info + j + NP - 1;
    const int r0 = pi0->r, r1 = NP == 2 ? pi1->r : 0;
    // the rows to update: the list of the rows that are not pivots of
    // panels <= j + NP - 1 (the rows that are have y = 0)
    const int jl = j + NP - 1;
    const int nact = c.nact[jl];
    // (with no row left the tiles are still visited when E is wanted: the
    // pivot rows' echelon words come from the same tables)
    const int nchunks = max((nact + kRestChunk - 1) / kRestChunk, c.Eint ? 1 : 0);
    const int64_t items = (int64_t)ntiles * nchunks;
    const int64_t i0 = items * blockIdx.x / gridDim.x, i1 = items * (blockIdx.x + 1) / gridDim.x;
    const bool work = (r0 != 0 || r1 != 0) && i0 < i1;
    // The one-row-group variant (the head launches: one tile, one chunk per
    // CTA, a serial latency chain) also loads its pivot rows' storage rows,
    // their multipliers and its first rows before the wait.
    constexpr bool PRE = U == 1;
    RestPre<NP, kRestThreads> pre{};
    RestIter<U> first{};
    if (PRE && work) {
        rest_preload<NP, kRestThreads>(c, j, r0, r1, pre);
        const int chunk = (int)(i0 % nchunks);
        const int chunk_end = (int)((min(i1, (i0 / nchunks + 1) * nchunks) - 1) % nchunks) + 1;
        rest_iter_load<U, NP>(c, j, chunk * kRestChunk + (int)(threadIdx.x >> 5) * kRowsPerWarp * U,
                              min(nact, chunk_end * kRestChunk), first);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    GF2_TR(const int jt = j + NP - 1 < kTraceMaxPanels ? j + NP - 1 : kTraceMaxPanels - 1;
           TraceSpan span(g_update_trace + kTrRestStart * kTraceMaxPanels + jt,
                          g_update_trace + kTrRestEnd * kTraceMaxPanels + jt);)
    extern __shared__ __align__(16) uint64_t smem[];
    if (!work) return;
    UpdOps ops;
    // The item range is split into segments of one tile each: one table
    // build per segment, then one pipelined pass over its rows.
    for (int64_t it = i0; it < i1;) {
        const bool seg0 = it == i0;
        const int tile = tile_first + (int)(it / nchunks);
        const int chunk = (int)(it % nchunks);
        const int64_t seg_end = min(i1, (int64_t)(tile - tile_first + 1) * nchunks);
        const int chunk_end = (int)((seg_end - 1) % nchunks) + 1;
        it = seg_end;
        const int rb = chunk * kRestChunk, re = min(nact, chunk_end * kRestChunk);
        if (PRE) {
            rest_prepare<C, NP, kRestThreads, PRE>(c, j, tile, chunk == 0, smem, ops, pre);
            if (seg0) rest_pass<C, U, NP, kRestThreads, PRE>(c, j, tile, rb, re, smem, ops, first);
            else rest_pass<C, U, NP, kRestThreads>(c, j, tile, rb, re, smem, ops);
        } else {
            rest_prepare<C, NP, kRestThreads>(c, j, tile, chunk == 0, smem, ops);
            rest_pass<C, U, NP, kRestThreads>(c, j, tile, rb, re, smem, ops);
        }
    }
    GF2_OPS(add_ops(g_update_ops, kOpUpdates, ops.upd); add_ops(g_update_ops, C == 8 ? kOpLookups8 : kOpLookups4, ops.lk);
            add_ops(g_update_ops, C == 8 ? kOpTable8 : kOpTable4, ops.tab);)
}

int g_num_sms = 0;

int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <class K>
cudaError_t allow_smem(K kernel, int bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

// Shared-memory limits of the kernels that need more than 48 KB, once per
// device (must run before a stream capture records their launches).
cudaError_t prepare_update_kernels()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = allow_smem(k_rest<8, kRestU, 1>, rest_smem_bytes<8, 1>());
    if (e == cudaSuccess) e = allow_smem(k_rest<8, kRest2U, 2>, rest_smem_bytes<8, 2>());
    if (e == cudaSuccess) e = allow_smem(k_rest<4, kRest2U, 2>, rest_smem_bytes<4, 2>());
    if (e == cudaSuccess) e = allow_smem(k_rest<8, kRestHeadU, 2>, rest_smem_bytes<8, 2>());
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

#ifdef GF2_COUNT_OPS
cudaError_t read_update_ops(unsigned long long *acc, bool reset)
{
    unsigned long long h[kNumOps];
    cudaError_t e = cudaMemcpyFromSymbol(h, g_update_ops, sizeof(h));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < kNumOps; ++i) acc[i] += h[i];
    if (reset) {
        const unsigned long long z[kNumOps] = {};
        e = cudaMemcpyToSymbol(g_update_ops, z, sizeof(z));
    }
    return e;
}
#endif

#ifdef GF2_TRACE
cudaError_t read_update_trace(unsigned long long *out, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_update_trace, sizeof(g_update_trace));
    if (e == cudaSuccess && reset) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_update_trace);
        if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(g_update_trace));
    }
    return e;
}
#endif

cudaError_t launch_next(const DecompCtx &c, int j, cudaStream_t s)
{
    const int blocks = (c.n + kNextRows - 1) / kNextRows;
    k_next<<<blocks, kNextThreads, 0, s>>>(c, j);
    return cudaGetLastError();
}

int rest_tiles(const DecompCtx &c, int j, int np, int *tile_first)
{
    *tile_first = (j + 1 + np) / kTileWords + 1;
    const int tiles = (c.mu + kTileWords - 1) / kTileWords - *tile_first;
    return tiles > 0 ? tiles : 0;
}

cudaError_t launch_rest(const DecompCtx &c, int j, int np, int est_active_rows, cudaStream_t s, int skip, int limit)
{
    int tile_first = 0;
    int ntiles = rest_tiles(c, j, np, &tile_first) - skip;
    tile_first += skip;
    if (ntiles > limit) ntiles = limit;
    if (ntiles <= 0) return cudaSuccess;
    const int nchunks = (c.n + kRestChunk - 1) / kRestChunk;
    const int64_t items = (int64_t)ntiles * nchunks;
    // one SM is left free for the panel kernel (whose shared-memory request
    // keeps it off the SMs that hold a k_rest CTA): the panel is a serial,
    // latency-bound chain that slows down when it shares a scheduler
    int grid = num_sms() > 1 ? num_sms() - 1 : 1;
    if (items < grid) grid = (int)items;
    cudaError_t e = prepare_update_kernels();
    if (e != cudaSuccess) return e;
    // programmatic stream serialization: the launch may be scheduled while
    // the previous update runs (its CTAs wait in griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kRestThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // table size: the caller's choice (c.tab_c), else 8 bits, and 4 bits
    // for one panel with few rows below it (fewer rows to amortise the
    // tables over)
    if (np == 2) {
        if (c.tab_c == 4) {
            cfg.dynamicSmemBytes = rest_smem_bytes<4, 2>();
            return cudaLaunchKernelEx(&cfg, k_rest<4, kRest2U, 2>, c, j, tile_first, ntiles);
        }
        cfg.dynamicSmemBytes = rest_smem_bytes<8, 2>();
        // a head with at most one item per CTA (where CTAs take two or more,
        // the deeper row groups of kRest2U do better), and with at least
        // kRestHeadMinRows rows below the pair: there the update stream bounds
        // the decomposition and the head's latency delays the look-ahead
        // (measured: below, e.g. all of a 16384 x 16384 decomposition, the
        // deeper row groups do better here too)
        if (limit == 1 && skip == 0 && ntiles == 1 && est_active_rows >= kRestHeadMinRows &&
            (est_active_rows + kRestChunk - 1) / kRestChunk <= num_sms() - 1)
            return cudaLaunchKernelEx(&cfg, k_rest<8, kRestHeadU, 2>, c, j, tile_first, ntiles);
        return cudaLaunchKernelEx(&cfg, k_rest<8, kRest2U, 2>, c, j, tile_first, ntiles);
    }
    if (c.tab_c == 8 || (c.tab_c == 0 && est_active_rows >= 4096)) {
        cfg.dynamicSmemBytes = rest_smem_bytes<8, 1>();
        return cudaLaunchKernelEx(&cfg, k_rest<8, kRestU, 1>, c, j, tile_first, ntiles);
    }
    cfg.dynamicSmemBytes = rest_smem_bytes<4, 1>();
    return cudaLaunchKernelEx(&cfg, k_rest<4, kRestU, 1>, c, j, tile_first, ntiles);
}

}  // namespace gf2
