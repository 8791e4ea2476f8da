// The whole decomposition P*A = L*E in one persistent, cooperative launch
// (pairs of 64-column panels; Section 4's block elimination with the
// wide-panel update of Section 5).
//
// Why one launch.  The panel step of block j (Procedure buildZ, Sections
// 4.1-4.4) is a serial chain of 64 pivot decisions that no other work can
// shorten, and panel j+2 cannot start before the look-ahead of panel j has
// applied panel j to the next two column blocks.  As separate launches each
// of the mu panels pays a kernel launch and the placement of its CTA, and
// one panel CTA's shared memory keeps the next one from being resident
// early.  Here CTA 0 runs the panel chain for the whole decomposition on an
// SM it never gives up, and the other CTAs (the workers) run the look-ahead
// and the trailing updates as the chain releases them.
//
// Work and its order (the same dependencies as the separate launches):
//   PANEL(j)  CTA 0, threads 0..127; after NEXT(j-2).
//   NEXT(j)   the look-ahead of panel j (next_body, csrc/update_core.cuh), in
//             chunks of 512 list entries; after PANEL(j) and NEXT(j-1) (its
//             input list and F word), after the last pair update that covers
//             the tile holding word j+2 has finished that tile, and after the
//             pair update that read Y and the active list of panel j-8 (the
//             ring of eight buffers) has finished.
//   REST(p)   the update of the pair (2p, 2p+1) (rest_prepare / rest_pass),
//             after NEXT(2p+1) and after the previous pair's update has
//             finished (two updates of one word are ordered); in slots of
//             (tile, range of 256-entry chunks), each owned by one worker.
//             The first tile of the pair, which the next look-aheads wait
//             for, is split over every worker and claimed first.
// The look-ahead is the critical path: a worker looks for a look-ahead
// chunk before each batch of update chunks (kFBatch of them, a few
// microseconds), and its update tables live in shared memory apart from the
// look-ahead's, so it resumes its slot without rebuilding them.
//
// Progress counters in global memory order the work.  A producer's threads
// finish their writes, the CTA synchronises, and thread 0 fences and then
// increments (release); a consumer's thread 0 reads with acquire and fences,
// then the CTA synchronises before it touches the data.  Nothing is read
// through the read-only path.  Every wait polls with a short sleep and gives
// up after kFSpinLimit polls: it then sets the failure word, every CTA
// leaves, and the rank reads -1.  The cooperative launch puts all CTAs on
// the GPU at once, so a wait only ever waits for CTAs that are running.
#include <mutex>

#include "panel_core.cuh"
#include "update_core.cuh"

namespace gf2 {
namespace {

constexpr int kFThreads = 512;
constexpr int kFNextRows = 512;           // list entries per look-ahead round (one per thread)
constexpr int kFNextRounds = 1;           // rounds per look-ahead chunk (one table setup per chunk)
constexpr int kFRestU = 4;                // row groups of 16 rows per warp and pass iteration
constexpr int kFBatch = 16;               // update chunks between looks at the look-ahead queue
constexpr int kFSmemBytes = 200 * 1024;   // dynamic shared memory of every CTA (one per SM)
constexpr long long kFSpinLimit = 1ll << 22;  // default polls of one wait (~64-500 ns each) before it gives up

// progress words (int32, zeroed before the launch): a header, then the
// per-panel, per-pair and per-(pair, tile) counters
enum { kPgPanelDone = 0, kPgNextComplete = 1, kPgFail = 2, kPgHeader = 8 };

struct Progress {
    int32_t *hdr;
    int32_t *next_claim, *next_done;                          // [mu]: chunks claimed / finished
    int32_t *pair_claim, *pair_done;                          // [npairs]: slots claimed, chunks finished
    int32_t *pair_tf, *pair_nt, *pair_nch, *pair_prev;        // [npairs]: shape, published with NEXT(2p+1)
    int32_t *tile_done;                                       // [npairs][ntw]: chunks finished per tile
    int npairs, ntw;
    long long limit;                                          // polls of one wait before it gives up
};

__host__ __device__ inline Progress progress_at(int32_t *base, int mu)
{
    Progress g;
    g.npairs = mu / 2;
    g.ntw = (mu + kTileWords - 1) / kTileWords;
    g.hdr = base;
    int32_t *p = base + kPgHeader;
    g.limit = kFSpinLimit;
    g.next_claim = p; p += mu;
    g.next_done = p; p += mu;
    g.pair_claim = p; p += g.npairs;
    g.pair_done = p; p += g.npairs;
    g.pair_tf = p; p += g.npairs;
    g.pair_nt = p; p += g.npairs;
    g.pair_nch = p; p += g.npairs;
    g.pair_prev = p; p += g.npairs;
    g.tile_done = p;
    return g;
}

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int32_t *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: polls until *p >= v.  false: the run failed (here or elsewhere).
__device__ __forceinline__ bool wait_geq(const int32_t *p, int v, const Progress &g)
{
    for (long long it = 0;; ++it) {
        if (ld_acquire(p) >= v) return true;
        if (ld_relaxed(g.hdr + kPgFail)) return false;
        if (it >= g.limit) {
            atomicExch(g.hdr + kPgFail, 1);
            return false;
        }
        __nanosleep(64);
    }
}

// Look-ahead chunks of panel j: one per kFNextRows entries of the list of
// the rows active before it, at least one (chunk 0 also writes the pivot
// rows' factors).
__device__ __forceinline__ int next_chunks(const DecompCtx &c, int j)
{
    const int cnt = j == 0 ? c.n : ld_relaxed(c.nact + j - 1);
    return max(1, (cnt + kFNextRows * kFNextRounds - 1) / (kFNextRows * kFNextRounds));
}

// Slots of pair p: ranges of its items, (tile, 256-entry chunk) in
// tile-major order.  Its first tile (tile_first), which the next
// look-aheads wait for, is split into `head` slots claimed first; the other
// tiles' items are split into one equal range per worker (about as the
// separate update launch splits them over its CTAs), so that a worker builds
// its tables once or twice per pair.
constexpr int kFHeadSlots = 16;

struct PairSlots {
    int head, body, nslots;
    int64_t items;  // tiles x chunks
};

__device__ __forceinline__ PairSlots pair_slots(const Progress &g, int p, int workers)
{
    PairSlots ps{0, 0, 0, 0};
    const int nt = ld_relaxed(g.pair_nt + p), nch = ld_relaxed(g.pair_nch + p);
    if (nt <= 0 || nch <= 0) return ps;
    ps.items = (int64_t)nt * nch;
    ps.head = min(nch, kFHeadSlots);
    ps.body = nt > 1 ? workers : 0;
    ps.nslots = ps.head + ps.body;
    return ps;
}

// Thread 0, after NEXT(2p+1) finished: the shape of pair p's update and the
// latest earlier pair with an update (its tiles are ordered before p's).
__device__ __forceinline__ void publish_pair(const DecompCtx &c, const Progress &g, int p)
{
    const int tf = (2 * p + 1 + 2) / kTileWords + 1;
    const int nt = max(0, g.ntw - tf);
    const int r0 = c.info[2 * p].r, r1 = c.info[2 * p + 1].r;
    const int nact = ld_relaxed(c.nact + 2 * p + 1);
    int nch = 0;
    if ((r0 | r1) && nt > 0) nch = max((nact + kRestChunk - 1) / kRestChunk, c.Eint ? 1 : 0);
    g.pair_tf[p] = tf;
    g.pair_nt[p] = nch > 0 ? nt : 0;
    g.pair_nch[p] = nch;
    g.pair_prev[p] = p == 0 ? -1 : (ld_relaxed(g.pair_nch + p - 1) > 0 ? p - 1 : ld_relaxed(g.pair_prev + p - 1));
}

// Thread 0: may NEXT(j) start?  (Never waits.)  When not, *wp / *wv name
// the first unmet condition, "*wp >= *wv": the caller polls that one word
// instead of testing everything again.
__device__ __forceinline__ bool next_ready(const DecompCtx &c, const Progress &g, int j, const int32_t **wp, int *wv)
{
    *wp = g.hdr + kPgPanelDone;
    *wv = j + 1;
    if (ld_acquire(*wp) < *wv) return false;
    *wp = g.hdr + kPgNextComplete;
    *wv = j;
    if (ld_acquire(*wp) < *wv) return false;
    // the ring of Y buffers and active lists: the update that read panel
    // j-8's has finished
    if (j >= 8) {
        const int q = (j - 8) / 2;
        const int nch = ld_relaxed(g.pair_nch + q);
        *wp = g.pair_done + q;
        *wv = nch * ld_relaxed(g.pair_nt + q);
        if (nch > 0 && ld_acquire(*wp) < *wv) return false;
    }
    // the tile holding word j+2: the last pair update that covers it (pairs
    // up to (j-2, j-1)) has finished it
    if (j + 2 < c.mu && j >= 2) {
        const int T = (j + 2) / kTileWords;
        int q = (j - 2) / 2;
        if (ld_relaxed(g.pair_nch + q) == 0) q = ld_relaxed(g.pair_prev + q);
        while (q >= 0 && ld_relaxed(g.pair_tf + q) > T) q = ld_relaxed(g.pair_prev + q);
        if (q >= 0) {
            *wp = g.tile_done + (int64_t)q * g.ntw + T;
            *wv = ld_relaxed(g.pair_nch + q);
            if (ld_acquire(*wp) < *wv) return false;
        }
    }
    *wp = nullptr;
    return true;
}

#ifdef GF2_TRACE
__device__ unsigned long long g_factor_trace[kTrSlots * kTraceMaxPanels];  // the trace build's stamps
#endif

// what a worker CTA does next (decided by thread 0)
enum { kDoIdle = 0, kDoNext = 1, kDoRest = 2, kDoQuit = 3 };
struct WorkerCmd {
    int kind, j, chunk, p, tile, rb, re, prepare, first;
};

// Panels j_start.. (even j_start): the earlier panels, their look-aheads
// and the updates of their pairs are done (launch_factor_init marks them).
template <int C>
__global__ void __launch_bounds__(kFThreads, 1) k_factor(DecompCtx c, int32_t *progress, int j_start,
                                                           long long wait_limit)
{
    extern __shared__ __align__(16) unsigned char fsmem[];
    Progress g = progress_at(progress, c.mu);
    g.limit = wait_limit;
    const int tid = threadIdx.x;
    UpdOps ops;

    if (blockIdx.x == 0) {
        // ---------------------------------------------------- the panel chain
        if (tid >= kPanelThreads) return;
        PanelShared &sh = *reinterpret_cast<PanelShared *>(fsmem);
        constexpr int kShBytes = (int)((sizeof(PanelShared) + 15) / 16 * 16);
        constexpr int kListCap = (kFSmemBytes - kShBytes) / 12 / 8 * 8;
        uint64_t *zs = reinterpret_cast<uint64_t *>(fsmem + kShBytes);
        __shared__ int quit;
        for (int j = j_start; j < c.mu; ++j) {
            if (tid == 0) {
                quit = (j >= 2 && !wait_geq(g.hdr + kPgNextComplete, j - 1, g)) ? 1 : 0;
                __threadfence();
                GF2_TR(if (j < kTraceMaxPanels) g_factor_trace[kTrPanelStart * kTraceMaxPanels + j] = trace_clock();)
            }
            panel_sync();
            if (quit) return;
#ifdef GF2_TRACE
            panel_block(c, j, sh, zs, kListCap, j < kTraceMaxPanels ? g_factor_trace : nullptr);
#else
            panel_block(c, j, sh, zs, kListCap);
#endif
            panel_sync();
            if (tid == 0) {
                __threadfence();
                st_release(g.hdr + kPgPanelDone, j + 1);
            }
        }
        return;
    }

    // -------------------------------------------------------------- workers
    // shared memory: the update's tables and staged rows, then the
    // look-ahead's (apart, so that a look-ahead chunk leaves the tables of
    // the segment in progress intact)
    uint64_t *rest_smem = reinterpret_cast<uint64_t *>(fsmem);
    uint64_t *next_smem = reinterpret_cast<uint64_t *>(fsmem + rest_smem_bytes<C, 2>());
    int *keep_row = reinterpret_cast<int *>(next_smem + kNextSmemWords);
    int *keep_warp = keep_row + kFNextRows;
    __shared__ WorkerCmd cmd;
    __shared__ int kw[kFThreads / 32];  // per warp: the next iteration of the segment in progress
    __shared__ int stop;                // set by thread 0: leave the update pass (look-ahead work)
    const int workers = gridDim.x - 1;
    const int wid = blockIdx.x - 1;
    // every worker takes look-ahead chunks; the last kFHeadSlots also take
    // the head slots of every pair
    const int head_slot = wid - (workers - kFHeadSlots);  // >= 0: this worker's head slot
    // thread 0's state: the look-ahead cursor; the pair cursor, its phase
    // (0: head slot, 1: body slot) and the slot in progress (items [si, se),
    // tile-major, of pair sp; sprep: the tables of item si's tile are not
    // built yet)
    int jn = j_start, pr = j_start / 2, phase = head_slot >= 0 ? 0 : 1;
    int sp = -1, sprep = 0, s_tf = 0, s_nch = 1, s_nact = 0;
    int64_t si = 0, se = 0, seg_end = 0;
    long long idle = 0;
    // the condition NEXT(jn) waits for ("*watch >= watch_val"; null: test
    // everything) and its value, read before the previous work ran
    const int32_t *watch = nullptr;
    int watch_val = 0, watched = 0;
    for (;;) {
        if (tid == 0) {
            WorkerCmd w{};
            w.kind = kDoIdle;
            if (ld_relaxed(g.hdr + kPgFail)) {
                w.kind = kDoQuit;
            } else {
                // 1. a look-ahead chunk (only once the condition it last
                // waited for holds)
                // (a worker without a slot in progress tests everything)
                while (jn < c.mu && (!watch || watched >= watch_val || sp < 0) && next_ready(c, g, jn, &watch, &watch_val)) {
                    const int nch = next_chunks(c, jn);
                    if (ld_relaxed(g.next_claim + jn) >= nch) {
                        ++jn;
                        continue;
                    }
                    const int t = atomicAdd(g.next_claim + jn, 1);
                    if (t < nch) {
                        w.kind = kDoNext;
                        w.j = jn;
                        w.chunk = t;
                        break;
                    }
                    ++jn;
                }
                // 2. this worker's slots of the pairs in order: its head slot
                // (if it has one), then its range of the other tiles, once the
                // pair's look-ahead is done
                while (w.kind == kDoIdle && sp < 0 && pr < g.npairs &&
                       ld_acquire(g.hdr + kPgNextComplete) >= 2 * pr + 2) {
                    const int p_this = pr;
                    const PairSlots ps = pair_slots(g, p_this, workers);
                    const int64_t nch = ld_relaxed(g.pair_nch + p_this);
                    si = se = 0;
                    if (ps.nslots > 0 && phase == 0 && head_slot < ps.head) {
                        si = nch * head_slot / ps.head;
                        se = nch * (head_slot + 1) / ps.head;
                    } else if (ps.nslots > 0 && phase == 1 && ps.body > 0) {
                        si = nch + (ps.items - nch) * wid / ps.body;
                        se = nch + (ps.items - nch) * (wid + 1) / ps.body;
                    }
                    // the next slot of this worker: the body slot of this
                    // pair after its head slot, else the next pair
                    if (phase == 0) {
                        phase = 1;
                    } else {
                        phase = head_slot >= 0 ? 0 : 1;
                        ++pr;
                    }
                    if (si < se) {
                        sp = p_this;
                        s_tf = ld_relaxed(g.pair_tf + sp);
                        s_nch = (int)nch;
                        s_nact = ld_relaxed(c.nact + 2 * sp + 1);
                        sprep = 1;
                    }
                }
                if (w.kind == kDoIdle && sp >= 0) {
                    // the rest of item si's tile in this slot; a new tile
                    // first waits until the previous pair with an update has
                    // finished it (two updates of one word are ordered)
                    const int64_t t = si / s_nch, c0 = si % s_nch;
                    seg_end = min(se, (t + 1) * s_nch);
                    const int tile = s_tf + (int)t;
                    const int q = sprep ? ld_relaxed(g.pair_prev + sp) : -1;
                    if (q >= 0 && !wait_geq(g.tile_done + (int64_t)q * g.ntw + tile, ld_relaxed(g.pair_nch + q), g)) {
                        w.kind = kDoQuit;
                    } else {
                        w.kind = kDoRest;
                        w.p = sp;
                        w.tile = tile;
                        w.prepare = sprep;
                        w.first = c0 == 0;
                        w.rb = (int)(c0 * kRestChunk);
                        w.re = min(s_nact, (int)(((seg_end - 1) % s_nch + 1) * kRestChunk));
                        w.chunk = (int)(seg_end - si);  // chunks of this segment
                    }
                }
                if (w.kind == kDoIdle && jn >= c.mu && pr >= g.npairs && sp < 0) w.kind = kDoQuit;
            }
            if (w.kind != kDoIdle) __threadfence();
            cmd = w;
            stop = 0;
            // the watched word, loaded now and used at the next decision:
            // its latency overlaps the work of this one
            if (watch) watched = ld_relaxed(watch);
        }
        __syncthreads();
        const WorkerCmd w = cmd;
        if (w.kind == kDoQuit) break;
        if (w.kind == kDoIdle) {
            if (tid == 0) {
                if (++idle > g.limit) atomicExch(g.hdr + kPgFail, 1);
                __nanosleep(128);
            }
            __syncthreads();
            continue;
        }
        idle = 0;
        if (w.kind == kDoNext) {
            GF2_TR(if (tid == 0 && w.j < kTraceMaxPanels)
                       atomicMax(g_factor_trace + kTrNextStart * kTraceMaxPanels + w.j, ~trace_clock());)
            next_body<kFThreads, kFNextRows, kFNextRounds>(c, w.j, w.chunk, next_smem, keep_row, keep_warp);
            __syncthreads();
            if (tid == 0) {
                GF2_TR(if (w.j < kTraceMaxPanels) atomicMax(g_factor_trace + kTrNextEnd * kTraceMaxPanels + w.j, trace_clock());)
                __threadfence();
                const int nch = next_chunks(c, w.j);
                if (atomicAdd(g.next_done + w.j, 1) == nch - 1) {
                    // the last chunk: NEXT(j) is complete
                    __threadfence();
                    if (w.j & 1) publish_pair(c, g, w.j / 2);
                    __threadfence();
                    st_release(g.hdr + kPgNextComplete, w.j + 1);
                }
            }
        } else {  // kDoRest
            const int j = 2 * w.p;
            GF2_TR(if (tid == 0 && j + 1 < kTraceMaxPanels)
                       atomicMax(g_factor_trace + kTrRestStart * kTraceMaxPanels + j + 1, ~trace_clock());)
            if (w.prepare) {
                rest_prepare<C, 2, kFThreads>(c, j, w.tile, w.first != 0, rest_smem, ops);
                if (tid < kFThreads / 32) kw[tid] = 0;
                __syncthreads();
            }
            // (thread 0 of a look-ahead worker polls the word its look-ahead
            // waits for and stops the pass when it changes)
            const int done = w.rb < w.re ? rest_pass_from<C, kFRestU, 2, kFThreads>(c, j, w.tile, w.rb, w.re, rest_smem,
                                                                                     ops, kw, &stop, watch, watch_val)
                                         : 1;
            if (tid == 0) {
                GF2_TR(if (j + 1 < kTraceMaxPanels) atomicMax(g_factor_trace + kTrRestEnd * kTraceMaxPanels + j + 1, trace_clock());)
                if (done) {
                    __threadfence();
                    atomicAdd(g.tile_done + (int64_t)w.p * g.ntw + w.tile, w.chunk);
                    atomicAdd(g.pair_done + w.p, w.chunk);
                    si = seg_end;
                    sprep = 1;
                    if (si >= se) sp = -1;
                } else {
                    sprep = 0;  // stopped: the tables and kw stay for the resumption
                }
            }
        }
    }
    GF2_OPS(add_ops(g_update_ops, kOpUpdates, ops.upd); add_ops(g_update_ops, C == 8 ? kOpLookups8 : kOpLookups4, ops.lk);
            add_ops(g_update_ops, C == 8 ? kOpTable8 : kOpTable4, ops.tab);)
}

static_assert(rest_smem_bytes<8, 2>() + kNextSmemWords * 8 + (kFNextRows + kFThreads / 32 + 1) * 4 <= kFSmemBytes,
              "worker shared memory");

std::mutex g_factor_mutex;
int g_factor_ready[64];  // per device: 0 unknown, 1 usable, -1 not (one CTA per SM does not fit)

template <int C>
cudaError_t factor_prepare(int dev)
{
    cudaError_t e = cudaFuncSetAttribute(k_factor<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmemBytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor<C>, kFThreads, kFSmemBytes);
    if (e != cudaSuccess) return e;
    int coop = 0;
    e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return e;
    return (per_sm >= 1 && coop) ? cudaSuccess : cudaErrorNotSupported;
}

// The progress words before a run from panel j_start: all zero (the pairs
// before j_start / 2 read as having no update, which is complete), then
// j_start panels and look-aheads done.
__global__ void k_factor_init(int32_t *progress, int64_t ints, int j_start)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ints; i += (int64_t)gridDim.x * blockDim.x)
        progress[i] = i == kPgPanelDone || i == kPgNextComplete ? j_start : 0;
}

}  // namespace

cudaError_t launch_factor_init(int32_t *progress, int mu, int j_start, cudaStream_t s)
{
    const int64_t ints = factor_progress_ints(mu);
    const int blocks = (int)((ints + 255) / 256 < 1024 ? (ints + 255) / 256 : 1024);
    k_factor_init<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(progress, ints, j_start);
    return cudaGetLastError();
}

int64_t factor_progress_ints(int mu)
{
    const int64_t npairs = mu / 2, ntw = (mu + kTileWords - 1) / kTileWords;
    return kPgHeader + 2 * (int64_t)mu + 6 * npairs + npairs * ntw;
}

const int32_t *factor_fail_word(const int32_t *progress) { return progress + kPgFail; }

cudaError_t factor_available()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_factor_mutex);
        if (g_factor_ready[dev] == 0) {
            e = factor_prepare<8>(dev);
            if (e == cudaSuccess) e = factor_prepare<4>(dev);
            g_factor_ready[dev] = e == cudaSuccess ? 1 : -1;
            if (e != cudaSuccess && e != cudaErrorNotSupported) {
                g_factor_ready[dev] = 0;
                return e;
            }
        }
        if (g_factor_ready[dev] < 0) return cudaErrorNotSupported;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    return sms < 2 ? cudaErrorNotSupported : cudaSuccess;
}

cudaError_t launch_factor(const DecompCtx &c0, int32_t *progress, int j_start, cudaStream_t s)
{
    cudaError_t e = factor_available();
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (sms < 2) return cudaErrorNotSupported;
    DecompCtx c = c0;
    c.fail = progress + kPgFail;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sms);
    cfg.blockDim = dim3(kFThreads);
    cfg.dynamicSmemBytes = kFSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long limit = (long long)device_wait_limit(kFSpinLimit);
    if (c.tab_c == 4) return cudaLaunchKernelEx(&cfg, k_factor<4>, c, progress, j_start, limit);
    return cudaLaunchKernelEx(&cfg, k_factor<8>, c, progress, j_start, limit);
}

#ifdef GF2_COUNT_OPS
cudaError_t read_factor_ops(unsigned long long *acc, bool reset)
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
cudaError_t read_factor_trace(unsigned long long *out, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_factor_trace, sizeof(g_factor_trace));
    if (e == cudaSuccess && reset) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_factor_trace);
        if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(g_factor_trace));
    }
    return e;
}
#endif

}  // namespace gf2
