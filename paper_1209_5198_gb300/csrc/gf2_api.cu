// C ABI of the F2 library (declared in include/gf2.h): argument checks,
// workspace carving and the host-side sequence of kernel launches.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gf2.h"
#include "gf2_internal.cuh"

namespace gf2 {
// the autotuner's entry for (this device, the shape bucket of n x m), if any (csrc/tune.cu)
bool tuned_decompose_opts(int64_t n, int64_t m, gf2_opts *out);
// the decomposition over F_p (csrc/k_gfp.cu)
size_t fp_workspace_bytes(int64_t n, int64_t m);
int fp_decompose(const uint32_t *A, int64_t lda, int64_t n, int64_t m, uint32_t p, int32_t *perm, int32_t *pivcols,
                 int64_t *rank, uint32_t *L, int64_t ldl, uint32_t *E, int64_t lde, bool check, void *ws,
                 uint32_t wait_limit, cudaStream_t s);
}  // namespace gf2

using namespace gf2;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int64_t words_of(int64_t cols) { return (cols + 63) / 64; }
int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }
int64_t round_up_tiles(int64_t words) { return (words + kTileWords - 1) / kTileWords * kTileWords; }

uint64_t last_word_mask(int64_t cols)
{
    const int rem = (int)(cols % 64);
    return rem == 0 ? ~0ull : ((1ull << rem) - 1);
}

// ------------------------------------------------------------ workspace
struct OwnedWorkspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mutex;
std::vector<OwnedWorkspace> g_ws;  // one per device
uint32_t *g_flag_host = nullptr;   // pinned flag for padding checks
std::mutex g_flag_mutex;

int owned_workspace(size_t need, void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    if ((int)g_ws.size() <= dev) g_ws.resize(dev + 1);
    OwnedWorkspace &w = g_ws[dev];
    if (w.bytes < need) {
        if (w.ptr) {
            if (cudaDeviceSynchronize() != cudaSuccess) return GF2_ERR_CUDA;
            cudaFree(w.ptr);
            w.ptr = nullptr;
            w.bytes = 0;
        }
        if (cudaMalloc(&w.ptr, need) != cudaSuccess) {
            cudaGetLastError();
            return GF2_ERR_NOMEM;
        }
        w.bytes = need;
    }
    *out = w.ptr;
    return GF2_OK;
}

int get_workspace(void *user, size_t user_bytes, size_t need, void **out)
{
    if (user) {
        if (user_bytes < need) return GF2_ERR_NOMEM;
        *out = user;
        return GF2_OK;
    }
    if (need == 0) {
        *out = nullptr;
        return GF2_OK;
    }
    return owned_workspace(need, out);
}

// Reads the device flag back (synchronising the stream); GF2_ERR_PADDING if set.
int check_flag(const uint32_t *flag_dev, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_flag_mutex);
    if (!g_flag_host) {
        if (cudaHostAlloc(&g_flag_host, sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) return GF2_ERR_CUDA;
    }
    if (cudaMemcpyAsync(g_flag_host, flag_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GF2_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GF2_ERR_CUDA;
    return *g_flag_host ? GF2_ERR_PADDING : GF2_OK;
}

bool mat_ok(const gf2_mat *M)
{
    return M && M->rows >= 0 && M->cols >= 0 && (M->rows == 0 || M->cols == 0 || (M->w && M->ld >= M->rows));
}

#define CK(call)                                  \
    do {                                          \
        if ((call) != cudaSuccess) return GF2_ERR_CUDA; \
    } while (0)

// ------------------------------------------------------------ diagnostics
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};
std::atomic<int64_t> g_wait_limit{0};  // polls of a bounded device wait (0: each wait's default)
std::mutex g_timing_mutex;
struct TimedLaunch {
    int cls;
    cudaEvent_t a, b;
};
std::vector<TimedLaunch> g_timed;         // recorded since the last reset
std::vector<cudaEvent_t> g_event_pool;    // free events

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Runs one launch; counts it and, when timing is on, brackets it with events.
template <class F>
cudaError_t launch(int cls, cudaStream_t s, F &&f)
{
    if (!g_timing.load(std::memory_order_relaxed)) {
        cudaError_t e = f();
        if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
        return e;
    }
    std::lock_guard<std::mutex> lock(g_timing_mutex);
    TimedLaunch t{cls, take_event(), take_event()};
    if (!t.a || !t.b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(t.a, s);
    if (e == cudaSuccess) e = f();
    if (e == cudaSuccess) e = cudaEventRecord(t.b, s);
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    g_timed.push_back(t);
    return cudaSuccess;
}
#define LAUNCH(cls, expr) CK(launch((cls), s, [&]() { return (expr); }))
#define LAUNCH_ON(cls, strm, expr) CK(launch((cls), (strm), [&]() { return (expr); }))

// ------------------------------------------------------------ side stream
// Per device, kLanes sets of: high-priority non-blocking streams for the
// panel chain and for the look-ahead kernels, a low-priority one for the
// wide updates, and a pool of events for the cross-stream dependencies.
// Each decomposition takes the next lane in turn and holds that lane's mutex
// while it enqueues, so a lane's events are used by one call at a time (a
// wait captures the event's state when it is enqueued), and decompositions
// issued on different caller streams run side by side on the GPU.
constexpr int kLanes = 4;
struct SideResources {
    int device = 0;
    cudaStream_t main = nullptr;    // wide updates and outputs
    cudaStream_t stream = nullptr;  // the panel chain (high priority)
    cudaStream_t next = nullptr;    // the look-ahead kernels (high priority)
    std::vector<cudaEvent_t> events;
    std::mutex mu;                  // held while a decomposition is enqueued
};
struct DeviceLanes {
    SideResources lane[kLanes];
};
std::mutex g_lanes_mutex;  // guards the table below
std::vector<std::unique_ptr<DeviceLanes>> g_lanes;
std::atomic<unsigned> g_next_lane{0};

// The next lane of the current device, locked (lock owns its mutex).
int side_resources(int nevents, SideResources **out, std::unique_lock<std::mutex> &lock)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
    DeviceLanes *dl = nullptr;
    {
        std::lock_guard<std::mutex> g(g_lanes_mutex);
        if ((int)g_lanes.size() <= dev) g_lanes.resize(dev + 1);
        if (!g_lanes[dev]) g_lanes[dev].reset(new DeviceLanes);
        dl = g_lanes[dev].get();
    }
    SideResources &r = dl->lane[g_next_lane.fetch_add(1, std::memory_order_relaxed) % kLanes];
    lock = std::unique_lock<std::mutex>(r.mu);
    r.device = dev;
    if (!r.stream) {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return GF2_ERR_CUDA;
        if (cudaStreamCreateWithPriority(&r.stream, cudaStreamNonBlocking, hi) != cudaSuccess) return GF2_ERR_CUDA;
        if (cudaStreamCreateWithPriority(&r.next, cudaStreamNonBlocking, hi) != cudaSuccess) return GF2_ERR_CUDA;
        if (cudaStreamCreateWithPriority(&r.main, cudaStreamNonBlocking, lo) != cudaSuccess) return GF2_ERR_CUDA;
        if (prepare_update_kernels() != cudaSuccess) return GF2_ERR_CUDA;
        if (prepare_panel_kernel() != cudaSuccess) return GF2_ERR_CUDA;
    }
    while ((int)r.events.size() < nevents) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return GF2_ERR_CUDA;
        r.events.push_back(e);
    }
    *out = &r;
    return GF2_OK;
}

// ------------------------------------------------------------ graph cache
// One captured graph per (device, shape, every pointer the kernels see).
struct GraphKey {
    int32_t dev, pair, tab_c, jend;  // (no padding: the key is compared bytewise)
    int64_t n, m, lda, ldl, lde;
    const void *a, *perm, *piv, *rank, *L, *E, *ws;
};
struct GraphEntry {
    GraphKey key;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    uint64_t stamp;
    int64_t kernels;  // kernel nodes: the launches one replay makes
};
std::mutex g_graph_mutex;          // guards the graph cache
std::vector<GraphEntry> g_graphs;  // guarded by g_graph_mutex
uint64_t g_graph_clock = 0;
constexpr size_t kMaxGraphs = 16;
const bool g_use_graphs = [] {
    const char *e = getenv("GF2_GRAPHS");
    return !(e && e[0] == '0');
}();
// wide updates by pairs of panels (GF2_PAIRS=0: one update per panel)
const bool g_use_pairs = [] {
    const char *e = getenv("GF2_PAIRS");
    return !(e && e[0] == '0');
}();

// ------------------------------------------------------------ options
// A gf2_opts checked and resolved for one call (0 = the process-wide value,
// read where it is used).
struct CallOpts {
    int32_t automatic; // no decomposition option was given: the autotuner's entry applies, if any
    int32_t pair;      // wide updates by pairs of panels (panel_w 128) or one panel (64)
    int32_t tab_c;     // Four Russians table bits of the wide updates: 0 (automatic), 4 or 8
    int32_t schedule;  // GF2_SCHEDULE_*
    unsigned backend;  // product backend flag: 0, GF2_MMM_TABLES or GF2_MMM_TENSOR
    int64_t cutoff;    // Strassen cutoff of the product, 0 = the process one
    int64_t c8_from;   // batched: 8-bit tables from this size, 0 = the process one
};

int check_opts(const gf2_opts *o)
{
    if (!o) return GF2_OK;
    if (o->panel_w < 0 || o->panel_w % 64) return GF2_ERR_ARG;
    if (o->panel_w != 0 && o->panel_w != 64 && o->panel_w != 128) return GF2_ERR_UNSUPPORTED;
    if (o->table_c < 0 || o->table_c > 16) return GF2_ERR_ARG;
    if (o->table_c != 0 && o->table_c != 4 && o->table_c != 8) return GF2_ERR_UNSUPPORTED;
    if (o->tile_words < 0) return GF2_ERR_ARG;
    if (o->tile_words != 0 && o->tile_words != kTileWords) return GF2_ERR_UNSUPPORTED;
    if (o->backend < GF2_BACKEND_AUTO || o->backend > GF2_BACKEND_TENSOR) return GF2_ERR_ARG;
    if (o->schedule < GF2_SCHEDULE_AUTO || o->schedule > GF2_SCHEDULE_SPLIT || o->reserved) return GF2_ERR_ARG;
    if (o->strassen_cutoff < 0 || (o->strassen_cutoff > 0 && o->strassen_cutoff < 128)) return GF2_ERR_ARG;
    if (o->batched_c8_from < 0) return GF2_ERR_ARG;
    return GF2_OK;
}

CallOpts resolve_opts(const gf2_opts *o)
{
    CallOpts r{};
    r.automatic = !o || (o->panel_w == 0 && o->table_c == 0 && o->schedule == GF2_SCHEDULE_AUTO);
    r.pair = (o && o->panel_w) ? (o->panel_w == 128) : (g_use_pairs ? 1 : 0);
    r.tab_c = o ? o->table_c : 0;
    r.schedule = o ? o->schedule : GF2_SCHEDULE_AUTO;
    r.backend = !o ? 0u : o->backend == GF2_BACKEND_TABLES ? GF2_MMM_TABLES : o->backend == GF2_BACKEND_TENSOR ? GF2_MMM_TENSOR : 0u;
    r.cutoff = o ? o->strassen_cutoff : 0;
    r.c8_from = o ? o->batched_c8_from : 0;
    return r;
}

cudaGraphExec_t find_graph(const GraphKey &k, int64_t *kernels)
{
    for (auto &g : g_graphs)
        if (memcmp(&g.key, &k, sizeof(GraphKey)) == 0) {
            g.stamp = ++g_graph_clock;
            *kernels = g.kernels;
            return g.exec;
        }
    return nullptr;
}

int64_t kernel_nodes(cudaGraph_t graph)
{
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) != cudaSuccess) return 0;
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Keys of recent calls that ran without a graph (a second call captures one).
std::vector<GraphKey> g_seen;  // guarded by g_graph_mutex

bool seen_before(const GraphKey &k)
{
    for (auto &s : g_seen)
        if (memcmp(&s, &k, sizeof(GraphKey)) == 0) return true;
    if (g_seen.size() >= 4 * kMaxGraphs) g_seen.erase(g_seen.begin());
    g_seen.push_back(k);
    return false;
}

// Caches a captured graph and returns the one to launch: the cached one if
// another call captured the same key meanwhile (the new one is dropped).
cudaGraphExec_t remember_graph(const GraphKey &k, cudaGraph_t graph, cudaGraphExec_t exec)
{
    for (auto &g : g_graphs)
        if (memcmp(&g.key, &k, sizeof(GraphKey)) == 0) {
            cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            g.stamp = ++g_graph_clock;
            return g.exec;
        }
    if (g_graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < g_graphs.size(); ++i)
            if (g_graphs[i].stamp < g_graphs[old].stamp) old = i;
        cudaGraphExecDestroy(g_graphs[old].exec);
        cudaGraphDestroy(g_graphs[old].graph);
        g_graphs.erase(g_graphs.begin() + old);
    }
    g_graphs.push_back(GraphEntry{k, graph, exec, ++g_graph_clock, kernel_nodes(graph)});
    return exec;
}

void drop_graphs()
{
    g_seen.clear();
    for (auto &g : g_graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    g_graphs.clear();
}

// ------------------------------------------------------------ decompose
// Enqueues the factorization of an ingested matrix on the library streams:
// P runs the panels, N the look-ahead kernels, M the wide trailing updates
// and the outputs:
//   panel(j) waits for next(j-2), which wrote the F words it starts from and
//     applied panel j-2 to word j;
//   one panel at a time: next(j) waits for panel(j), for rest(j-2) (it reuses
//     Y and the active list of j-2) and, when word j+2 opens a new tile, for
//     rest(j-1) (which updated that tile); rest(j) waits for next(j);
//   by pairs (j even, j+1): next(j) waits for panel(j) and for the update
//     that last covered the tile it rewrites (the previous pair's for
//     j = 4k+2, the one before for j = 4k); next(j+1) follows next(j);
//     rest(j, j+1) waits for next(j+1); a lone last panel is updated alone.
// So panel j+1 runs while next(j) and the updates of earlier panels run.
// The factors out of the working buffers and the rank (after either schedule).
int enqueue_outputs(const DecompCtx &c, int64_t *rank, gf2_mat *L, gf2_mat *E, cudaStream_t s)
{
    LAUNCH(GF2_KCLASS_LAYOUT, launch_finish_scalars(c, rank, s));
    if (E) LAUNCH(GF2_KCLASS_LAYOUT, launch_finish_E(c, E->w, E->ld, s));
    if (L)
        LAUNCH(GF2_KCLASS_LAYOUT, launch_colblocks_from_rowmajor(c.Lint, c.ldl, c.perm, c.n, (int32_t)words_of(c.kmax),
                                                                   L->w, L->ld, s));
    return GF2_OK;
}

// The panels from j_start (even) on in one cooperative persistent launch
// (csrc/k_factor.cu) on s, after its progress words are set up.
int enqueue_persistent(const DecompCtx &c, int32_t *progress, int j_start, cudaStream_t s)
{
    CK(launch_factor_init(progress, c.mu, j_start, s));
    LAUNCH(GF2_KCLASS_FACTOR, launch_factor(c, progress, j_start, s));
    return GF2_OK;
}

// The factorization: panels [0, jend) as separate launches on the library's
// streams (below), then, when jend < mu, the panels from jend on in one
// persistent launch (progress: its counters; jend even), then the outputs.
int enqueue_factorization(DecompCtx c, int64_t *rank, gf2_mat *L, gf2_mat *E, SideResources *side, int jend,
                          int32_t *progress)
{
    cudaStream_t s = side->main, P = side->stream, N = side->next;
    const int mu = c.mu;
    cudaEvent_t *evPanel = side->events.data(), *evNext = evPanel + mu, *evRest = evNext + mu;
    cudaEvent_t evFork = evRest[mu], evJoinP = evRest[mu + 1], evJoinN = evRest[mu + 2];
    cudaEvent_t *evHead = evRest + mu + 5;  // after evIn / evOut of the caller
    std::vector<char> rest_launched(mu, 0), head_launched(mu, 0);
    // the event after which the tile a pair's update starts with is done
    auto first_tile_done = [&](int jr) -> cudaEvent_t {
        if (jr < 0 || jr >= mu || !rest_launched[jr]) return nullptr;
        return head_launched[jr] ? evHead[jr] : evRest[jr];
    };
    CK(cudaEventRecord(evFork, s));
    CK(cudaStreamWaitEvent(P, evFork, 0));
    CK(cudaStreamWaitEvent(N, evFork, 0));
    for (int j = 0; j < jend; ++j) {
        if (j >= 2) CK(cudaStreamWaitEvent(P, evNext[j - 2], 0));
        LAUNCH_ON(GF2_KCLASS_PANEL, P, launch_panel(c, j, P));
        CK(cudaEventRecord(evPanel[j], P));
        CK(cudaStreamWaitEvent(N, evPanel[j], 0));
        if (c.pair) {
            // next(j), j even, rewrites the tile of word j+2: tile k for
            // j = 4k, the first tile of the update of pair (j-4, j-3); tile
            // k+1 for j = 4k+2, the first tile of the previous pair's update.
            // Those updates run that tile in a launch of its own (the head),
            // so next(j) waits for the head only and runs beside the rest of
            // the update.  next(j+1) follows next(j) on N; its tile is that
            // of next(j), its active list one of four, and the first panel's
            // update of its pivot rows happens inside the pair's own update.
            // (The Y buffers and active lists form a ring of kRing, so those
            // of the update still running are not rewritten meanwhile.)
            if (!(j & 1)) {
                const cudaEvent_t ev = first_tile_done((j & 3) == 0 ? j - 3 : j - 1);
                if (ev) CK(cudaStreamWaitEvent(N, ev, 0));
            }
        } else {
            if (j >= 2 && rest_launched[j - 2]) CK(cudaStreamWaitEvent(N, evRest[j - 2], 0));
            if (j >= 1 && (j + 2) % kTileWords == 0 && rest_launched[j - 1]) CK(cudaStreamWaitEvent(N, evRest[j - 1], 0));
        }
        LAUNCH_ON(GF2_KCLASS_NEXT, N, launch_next(c, j, N));
        CK(cudaEventRecord(evNext[j], N));
        // the wide update: of this panel, of the pair ending here, or none
        // (first panel of a pair)
        const int np = !c.pair ? 1 : ((j & 1) ? 2 : (j == mu - 1 ? 1 : 0));
        const int jf = j - np + 1;
        int tile_first = 0;
        const int ntiles = np > 0 ? rest_tiles(c, jf, np, &tile_first) : 0;
        if (ntiles > 0) {
            CK(cudaStreamWaitEvent(s, evNext[j], 0));
            const int est = (int)(c.n - 64 * (int64_t)(j + 1));
            if (np == 2 && (jf & 3) == 0) {
                // pair (4k, 4k+1): its first tile (k+1) alone, then the others
                LAUNCH(GF2_KCLASS_UPDATE, launch_rest(c, jf, np, est, s, 0, 1));
                CK(cudaEventRecord(evHead[j], s));
                head_launched[j] = 1;
                if (ntiles > 1) LAUNCH(GF2_KCLASS_UPDATE, launch_rest(c, jf, np, est, s, 1));
            } else {
                LAUNCH(GF2_KCLASS_UPDATE, launch_rest(c, jf, np, est, s));
            }
            CK(cudaEventRecord(evRest[j], s));
            rest_launched[j] = 1;
        }
    }
    CK(cudaEventRecord(evJoinP, P));
    CK(cudaStreamWaitEvent(s, evJoinP, 0));
    CK(cudaEventRecord(evJoinN, N));
    CK(cudaStreamWaitEvent(s, evJoinN, 0));
    if (jend < mu) return GF2_OK;  // the caller continues with enqueue_tail
    return enqueue_outputs(c, rank, L, E, s);
}

// After the separate launches of panels [0, jend) (jend < mu): the panels
// from jend on in one persistent launch, then the outputs; on s.
int enqueue_tail(DecompCtx c, int64_t *rank, gf2_mat *L, gf2_mat *E, int jend, int32_t *progress, cudaStream_t s)
{
    const int st = enqueue_persistent(c, progress, jend, s);
    if (st) return st;
    c.fail = factor_fail_word(progress);
    return enqueue_outputs(c, rank, L, E, s);
}

struct DecompLayout {
    int64_t mu, ldw, kmax, ldl;
    size_t oW, oY, oF, oAct, oNact, oOrw, oPP, oInfo, oZpos, oZraw, oLint, oEint, oFlag, oProg, total;
};

DecompLayout decomp_layout(int64_t n, int64_t m, bool factors)
{
    DecompLayout d{};
    d.mu = words_of(m);
    d.ldw = round8(d.mu > 0 ? d.mu : 1);
    d.kmax = n < m ? n : m;
    d.ldl = words_of(d.kmax) > 0 ? words_of(d.kmax) : 1;
    size_t o = 0;
    d.oW = o; o += align_up((size_t)n * d.ldw * 8);
    d.oY = o; o += align_up((size_t)n * kRing * 8);
    d.oF = o; o += align_up((size_t)n * 2 * 8);
    d.oAct = o; o += align_up((size_t)n * kRing * 4);
    d.oNact = o; o += align_up((size_t)(d.mu > 0 ? d.mu : 1) * 4);
    d.oOrw = o; o += align_up((size_t)(d.mu > 0 ? d.mu : 1) * 4);
    d.oPP = o; o += align_up((size_t)n * 4);
    d.oInfo = o; o += align_up((size_t)(d.mu > 0 ? d.mu : 1) * sizeof(PanelInfo));
    d.oZpos = o; o += align_up((size_t)(n > 0 ? n : 1) * 4);
    d.oZraw = o; o += align_up((size_t)(n > 0 ? n : 1) * 8);
    d.oLint = o; if (factors) o += align_up((size_t)n * d.ldl * 8);
    d.oEint = o; if (factors) o += align_up((size_t)d.kmax * d.ldw * 8);
    d.oFlag = o; o += kAlign;
    d.oProg = o; o += align_up((size_t)factor_progress_ints((int)d.mu) * 4);  // the persistent run's counters
    d.total = o;
    return d;
}

int decompose_impl(const gf2_mat *A, int32_t *perm, int32_t *pivcols, int64_t *rank, gf2_mat *L, gf2_mat *E,
                   unsigned flags, const CallOpts &o_in, void *workspace, size_t ws_bytes, cudaStream_t s)
{
    if (!mat_ok(A) || !perm || !rank || (flags & ~GF2_NOCHECK)) return GF2_ERR_ARG;
    const int64_t n = A->rows, m = A->cols;
    CallOpts o = o_in;
    if (o.automatic) {
        // automatic options: the autotuner's choice for this shape bucket, when it has one
        gf2_opts t{};
        if (tuned_decompose_opts(n, m, &t)) {
            if (t.panel_w) o.pair = t.panel_w == 128;
            o.tab_c = t.table_c;
            o.schedule = t.schedule;
        }
    }
    if (n >= (1ll << 31) - 64 || m >= (1ll << 31) - 64) return GF2_ERR_UNSUPPORTED;
    const int64_t kmax = n < m ? n : m;
    if (kmax > 0 && !pivcols) return GF2_ERR_ARG;
    if (L && (!mat_ok(L) || L->rows != n || L->cols != kmax)) return GF2_ERR_SHAPE;
    if (E && (!mat_ok(E) || E->rows != kmax || E->cols != m)) return GF2_ERR_SHAPE;
    const bool factors = L || E;
    const DecompLayout d = decomp_layout(n, m, factors);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, d.total, &ws);
    if (st) return st;
    char *base = static_cast<char *>(ws);

    DecompCtx c{};
    c.W = reinterpret_cast<uint64_t *>(base + d.oW);
    c.tstride = n * kTileWords;
    c.lde = d.ldw;
    c.perm = perm;
    c.pivcols = pivcols;
    c.info = reinterpret_cast<PanelInfo *>(base + d.oInfo);
    c.Y = reinterpret_cast<uint64_t *>(base + d.oY);
    c.F = reinterpret_cast<uint64_t *>(base + d.oF);
    c.act = reinterpret_cast<int32_t *>(base + d.oAct);
    c.nact = reinterpret_cast<int32_t *>(base + d.oNact);
    c.orw = reinterpret_cast<int32_t *>(base + d.oOrw);
    c.pivpanel = reinterpret_cast<int32_t *>(base + d.oPP);
    c.zpos = reinterpret_cast<int32_t *>(base + d.oZpos);
    c.zraw = reinterpret_cast<uint64_t *>(base + d.oZraw);
    c.Lint = factors ? reinterpret_cast<uint64_t *>(base + d.oLint) : nullptr;
    c.ldl = d.ldl;
    c.Eint = factors ? reinterpret_cast<uint64_t *>(base + d.oEint) : nullptr;
    c.n = (int32_t)n;
    c.m = (int32_t)m;
    c.mu = (int32_t)d.mu;
    c.kmax = (int32_t)kmax;
    c.pair = o.pair;
    c.tab_c = o.tab_c;
    uint32_t *flag = reinterpret_cast<uint32_t *>(base + d.oFlag);

    if (n == 0 || m == 0) {
        if (n > 0) LAUNCH(GF2_KCLASS_LAYOUT, launch_ingest_tiled(A->w, A->ld > 0 ? A->ld : 1, (int32_t)n, 0, ~0ull, c.W, perm, nullptr, nullptr, s));
        CK(cudaMemsetAsync(rank, 0, sizeof(int64_t), s));
        if (L && n > 0 && L->cols > 0) CK(cudaMemsetAsync(L->w, 0, (size_t)L->ld * words_of(L->cols) * 8, s));
        return GF2_OK;
    }

    CK(cudaMemsetAsync(flag, 0, sizeof(uint32_t), s));
    LAUNCH(GF2_KCLASS_LAYOUT, launch_ingest_tiled(A->w, A->ld, (int32_t)n, (int32_t)d.mu, last_word_mask(m), c.W, perm, c.pivpanel, flag, s));
    if (!(flags & GF2_NOCHECK)) {
        st = check_flag(flag, s);
        if (st) return st;
    }
    if (c.Lint) CK(cudaMemsetAsync(c.Lint, 0, (size_t)n * d.ldl * 8, s));
    CK(cudaMemsetAsync(c.nact, 0, (size_t)c.mu * sizeof(int32_t), s));  // the active-list counts
    CK(cudaMemsetAsync(c.orw, 0, (size_t)c.mu * sizeof(int32_t), s));   // the look-ahead's zero-block flags

    // Which panels run as separate launches ([0, jend)) and which in one
    // persistent launch (csrc/k_factor.cu), by pairs of panels only:
    // PERSISTENT all of them; SPLIT the first three quarters as separate
    // launches and the last quarter persistent (the panel chain bounds the
    // end, and there the persistent launch runs a panel every ~17 us against
    // ~22 us); AUTO the separate launches (measured: SPLIT 13.01 ms against
    // 13.00 ms at 32768, the switch costs what the last quarter gains).
    // A device that cannot hold one CTA per SM keeps the separate launches.
    int jend = c.mu;
    if (c.pair && (o.schedule == GF2_SCHEDULE_PERSISTENT || o.schedule == GF2_SCHEDULE_SPLIT)) {
        const cudaError_t e = factor_available();
        if (e == cudaSuccess) jend = o.schedule == GF2_SCHEDULE_PERSISTENT ? 0 : 2 * ((3 * c.mu) / 8);
        else if (e != cudaErrorNotSupported) return GF2_ERR_CUDA;
        cudaGetLastError();
    }
    int32_t *progress = reinterpret_cast<int32_t *>(base + d.oProg);

    // The factorization runs on the library's three streams of this device
    // (M: wide updates and outputs, P: the panel chain, N: the look-ahead
    // kernels), joined to the caller's stream s by events; the whole
    // sequence is captured once into a CUDA graph per (shape, pointers) and
    // replayed on later calls.
    std::unique_lock<std::mutex> lane_lock;
    SideResources *side = nullptr;
    st = side_resources(4 * c.mu + 5, &side, lane_lock);
    if (st) return st;
    cudaEvent_t evIn = side->events[3 * c.mu + 3], evOut = side->events[3 * c.mu + 4];
    CK(cudaEventRecord(evIn, s));
    CK(cudaStreamWaitEvent(side->main, evIn, 0));
    GraphKey key{};
    key.dev = side->device;
    key.pair = c.pair;
    key.tab_c = c.tab_c;
    key.n = n; key.m = m; key.a = A->w; key.lda = A->ld;
    key.perm = perm; key.piv = pivcols; key.rank = rank;
    key.L = L ? L->w : nullptr; key.ldl = L ? L->ld : 0;
    key.E = E ? E->w : nullptr; key.lde = E ? E->ld : 0;
    key.ws = ws;
    key.jend = jend;
    // (the separate launches are captured into the graph; a persistent
    // launch after them is not: enqueue_tail follows the graph)
    if (g_timing.load() || !g_use_graphs || jend == 0) {
        st = enqueue_factorization(c, rank, L, E, side, jend, progress);
        if (st) return st;
    } else {
        bool replayed = false, seen = false;
        {
            // a cached graph is launched under the cache's lock, so that no
            // other call evicts (destroys) it in between
            std::lock_guard<std::mutex> glock(g_graph_mutex);
            int64_t kernels = 0;  // kernels of a graph captured earlier (a capture counts its own)
            cudaGraphExec_t exec = find_graph(key, &kernels);
            if (exec) {
                CK(cudaGraphLaunch(exec, side->main));
                g_launches.fetch_add(kernels, std::memory_order_relaxed);
                replayed = true;
            } else {
                seen = seen_before(key);
            }
        }
        if (replayed) {
            // done
        } else if (!seen) {
            // first call with this shape and these buffers: enqueue directly
            // (a capture and instantiation cost more than one run; a repeat
            // call is captured and every later one replays the graph)
            st = enqueue_factorization(c, rank, L, E, side, jend, progress);
            if (st) return st;
        } else {
            if (cudaStreamBeginCapture(side->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GF2_ERR_CUDA;
            st = enqueue_factorization(c, rank, L, E, side, jend, progress);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(side->main, &graph);
            if (st || ec != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return st ? st : GF2_ERR_CUDA;
            }
            cudaGraphExec_t exec = nullptr;
            if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                cudaGraphDestroy(graph);
                return GF2_ERR_CUDA;
            }
            std::lock_guard<std::mutex> glock(g_graph_mutex);
            exec = remember_graph(key, graph, exec);
            CK(cudaGraphLaunch(exec, side->main));
        }
    }
    if (jend < c.mu) {
        st = enqueue_tail(c, rank, L, E, jend, progress, side->main);
        if (st) return st;
    }
    CK(cudaEventRecord(evOut, side->main));
    CK(cudaStreamWaitEvent(s, evOut, 0));
    return GF2_OK;
}

// ------------------------------------------------------------ RREF
// Scratch of gf2_rref: the blocks' inverses (64 words per 64-row block) and
// the gathered left operand of the largest product of the recursion (the
// top level's: the top half's rows at the bottom half's pivot columns).
struct RrefLayout {
    size_t oV, oTmp, total;
};

int64_t rref_split(int64_t a, int64_t b) { return a + 64 * (((b - a + 63) / 64) / 2); }

RrefLayout rref_layout(int64_t k)
{
    RrefLayout d{};
    d.oV = 0;
    d.oTmp = align_up((size_t)((k + 63) / 64) * 64 * 8);
    size_t tmp = 0;
    if (k > 64) {
        const int64_t mid = rref_split(0, k);
        tmp = (size_t)mid * (size_t)words_of(k - mid) * 8;
    }
    d.total = d.oTmp + align_up(tmp > 0 ? tmp : 1);
    return d;
}

// Rows [a, b) of E, whose 64-row blocks are already reduced by their own
// pivot columns: the bottom half [mid, b) recursively, then the top half
// takes E_top ^= E_top[:, pivots of the bottom] * R_bottom -- which clears
// the top rows at the bottom's pivot columns and leaves the top's own
// pivot columns as they were -- then the top half recursively.
int rref_rec(const gf2_mat &E, const int32_t *piv, int64_t a, int64_t b, uint64_t *tmp, cudaStream_t s)
{
    if (b - a <= 64) return GF2_OK;
    const int64_t mid = rref_split(a, b);
    int st = rref_rec(E, piv, mid, b, tmp, s);
    if (st) return st;
    const int64_t rows = mid - a, kk = b - mid;
    LAUNCH(GF2_KCLASS_LAYOUT, launch_gather_cols(E.w, E.ld, E.cols, piv, a, rows, mid, kk, tmp, rows, s));
    MmmCtx c{tmp, rows, E.w + mid, E.ld, E.w + a, E.ld, (int32_t)rows, (int32_t)kk, (int32_t)words_of(E.cols), kMmmXor};
    LAUNCH(GF2_KCLASS_UPDATE, launch_mmm(c, s));
    return rref_rec(E, piv, a, mid, tmp, s);
}

}  // namespace

extern "C" {

const char *gf2_status_string(int status)
{
    switch (status) {
    case GF2_OK: return "ok";
    case GF2_ERR_ARG: return "invalid argument (null pointer, negative size or unknown flag)";
    case GF2_ERR_SHAPE: return "inconsistent shapes (inner dimensions, ld < rows, factor sizes, k > 64)";
    case GF2_ERR_PADDING: return "nonzero bit beyond the last column (padding must be zero)";
    case GF2_ERR_NOMEM: return "workspace too small or device allocation failed";
    case GF2_ERR_CUDA: return "a CUDA runtime call failed";
    case GF2_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case GF2_ERR_UNSUPPORTED: return "size not supported by this build";
    default: return "unknown status";
    }
}

int gf2_version(void) { return 3; }

int gf2_release_workspace(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    if ((int)g_ws.size() > dev && g_ws[dev].ptr) {
        if (cudaDeviceSynchronize() != cudaSuccess) return GF2_ERR_CUDA;
        {
            std::lock_guard<std::mutex> glock(g_graph_mutex);
            drop_graphs();  // graphs may point into the released workspace
        }
        cudaFree(g_ws[dev].ptr);
        g_ws[dev] = OwnedWorkspace{};
    }
    return GF2_OK;
}

size_t gf2_decompose_workspace_bytes(int64_t n, int64_t m, int want_factors)
{
    if (n < 0 || m < 0) return 0;
    return decomp_layout(n, m, want_factors != 0).total;
}

int gf2_decompose(const gf2_mat *A, int32_t *perm, int32_t *pivcols, int64_t *rank, gf2_mat *L, gf2_mat *E,
                  unsigned flags, void *workspace, size_t ws_bytes, void *stream)
{
    return decompose_impl(A, perm, pivcols, rank, L, E, flags, resolve_opts(nullptr), workspace, ws_bytes,
                          static_cast<cudaStream_t>(stream));
}

int gf2_decompose_ex(const gf2_mat *A, int32_t *perm, int32_t *pivcols, int64_t *rank, gf2_mat *L, gf2_mat *E,
                     unsigned flags, const gf2_opts *opts, void *workspace, size_t ws_bytes, void *stream)
{
    const int st = check_opts(opts);
    if (st) return st;
    return decompose_impl(A, perm, pivcols, rank, L, E, flags, resolve_opts(opts), workspace, ws_bytes,
                          static_cast<cudaStream_t>(stream));
}

int gf2_opts_check(const gf2_opts *o) { return check_opts(o); }

size_t gf2_nullspace_workspace_bytes(int64_t m, int64_t rank)
{
    if (m < 0 || rank < 0 || rank > m) return 0;
    return align_up((size_t)(m - rank > 0 ? m - rank : 1) * 4) + kAlign;
}

int gf2_nullspace(const gf2_mat *R, const int32_t *pivcols, int64_t rank, gf2_mat *N, void *workspace,
                  size_t ws_bytes, void *stream)
{
    if (!R || !N || R->rows < 0 || R->cols < 0 || rank < 0) return GF2_ERR_ARG;
    const int64_t k = R->rows, m = R->cols;
    if (rank > (k < m ? k : m)) return GF2_ERR_ARG;
    if (m >= (1ll << 31) - 64) return GF2_ERR_UNSUPPORTED;
    const int64_t nul = m - rank;
    if (!mat_ok(N) || N->rows != m || N->cols != nul) return GF2_ERR_SHAPE;
    if (nul == 0 || m == 0) return GF2_OK;
    if (rank > 0 && (!mat_ok(R) || !R->w || !pivcols)) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, gf2_nullspace_workspace_bytes(m, rank), &ws);
    if (st) return st;
    // (the free list is fully written for a valid pivot list; cleared first so
    // that any other list reads as -1 entries, which contribute nothing)
    CK(cudaMemsetAsync(ws, 0xff, (size_t)nul * 4, s));
    LAUNCH(GF2_KCLASS_LAYOUT, launch_nullspace(R->w, R->ld, pivcols, rank, m, static_cast<int32_t *>(ws), N->w,
                                               N->ld, s));
    return GF2_OK;
}

size_t gf2_rref_workspace_bytes(int64_t k, int64_t m)
{
    if (k < 0 || m < 0) return 0;
    return rref_layout(k).total;
}

int gf2_rref(gf2_mat *E, const int32_t *pivcols, void *workspace, size_t ws_bytes, void *stream)
{
    if (!E || E->rows < 0 || E->cols < 0) return GF2_ERR_ARG;
    const int64_t k = E->rows, m = E->cols;
    if (k == 0 || m == 0) return GF2_OK;
    if (!E->w || !pivcols) return GF2_ERR_ARG;
    if (E->ld < k) return GF2_ERR_SHAPE;
    if (k >= (1ll << 31) - 64 || m >= (1ll << 31) - 64) return GF2_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const RrefLayout d = rref_layout(k);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, d.total, &ws);
    if (st) return st;
    char *base = static_cast<char *>(ws);
    uint64_t *V = reinterpret_cast<uint64_t *>(base + d.oV), *tmp = reinterpret_cast<uint64_t *>(base + d.oTmp);
    LAUNCH(GF2_KCLASS_LAYOUT, launch_rref_diag(E->w, E->ld, pivcols, k, m, V, s));
    return rref_rec(*E, pivcols, 0, k, tmp, s);
}

}  // extern "C"
namespace {
// gf2_rank: a wide matrix (n < m) is ranked through its transpose (m x n,
// more rows than columns: fewer panels and a cheaper update, Section 7),
// which sits at the front of the workspace; then the decomposition's own
// workspace, perm (one entry per row of the matrix decomposed), pivcols and
// the rank.
struct RankLayout {
    bool transposed;
    int64_t rows, cols;  // of the matrix decomposed
    size_t oT, oDec, oPerm, oPiv, oRank, total;
};

RankLayout rank_layout(int64_t n, int64_t m)
{
    RankLayout d{};
    d.transposed = n > 0 && n < m;
    d.rows = d.transposed ? m : n;
    d.cols = d.transposed ? n : m;
    const int64_t kmax = n < m ? n : m;
    size_t o = 0;
    d.oT = o;
    if (d.transposed) o += align_up((size_t)words_of(n) * (size_t)m * 8);
    d.oDec = o;
    o += gf2_decompose_workspace_bytes(d.rows, d.cols, 0);
    d.oPerm = o;
    o += align_up((size_t)(d.rows > 0 ? d.rows : 1) * 4);
    d.oPiv = o;
    o += align_up((size_t)(kmax > 0 ? kmax : 1) * 4);
    d.oRank = o;
    o += kAlign;
    d.total = o + kAlign;  // + the padding flag of the transposed route
    return d;
}

int rank_impl(const gf2_mat *A, int64_t *rank_host, unsigned flags, const CallOpts &o, void *workspace, size_t ws_bytes,
              cudaStream_t s)
{
    if (!A || !rank_host || (flags & ~GF2_NOCHECK) || !mat_ok(A)) return GF2_ERR_ARG;
    const int64_t n = A->rows, m = A->cols;
    const RankLayout d = rank_layout(n, m);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, d.total, &ws);
    if (st) return st;
    char *base = static_cast<char *>(ws);
    int32_t *perm = reinterpret_cast<int32_t *>(base + d.oPerm);
    int32_t *piv = reinterpret_cast<int32_t *>(base + d.oPiv);
    int64_t *rk = reinterpret_cast<int64_t *>(base + d.oRank);
    const size_t dec = gf2_decompose_workspace_bytes(d.rows, d.cols, 0);
    if (!d.transposed) {
        st = decompose_impl(A, perm, piv, rk, nullptr, nullptr, flags, o, base + d.oDec, dec, s);
    } else {
        if (n >= (1ll << 31) - 64 || m >= (1ll << 31) - 64) return GF2_ERR_UNSUPPORTED;
        if (!(flags & GF2_NOCHECK) && (m % 64)) {
            // the padding bits of A's last column block (they would become
            // rows past m of the transpose, which are not written)
            uint32_t *flag = reinterpret_cast<uint32_t *>(base + d.total - kAlign);
            CK(cudaMemsetAsync(flag, 0, sizeof(uint32_t), s));
            LAUNCH(GF2_KCLASS_LAYOUT, launch_check_last_block(A->w + (words_of(m) - 1) * A->ld, (int)n,
                                                              last_word_mask(m), flag, s));
            st = check_flag(flag, s);
            if (st) return st;
        }
        uint64_t *T = reinterpret_cast<uint64_t *>(base + d.oT);
        LAUNCH(GF2_KCLASS_LAYOUT, launch_transpose_bits(A->w, A->ld, n, m, T, m, s));
        const gf2_mat At{T, m, n, m};
        st = decompose_impl(&At, perm, piv, rk, nullptr, nullptr, flags | GF2_NOCHECK, o, base + d.oDec, dec, s);
    }
    if (st) return st;
    CK(cudaMemcpyAsync(rank_host, rk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return *rank_host < 0 ? GF2_ERR_TIMEOUT : GF2_OK;  // (-1: a persistent run's device wait gave up)
}
}  // namespace
extern "C" {

size_t gf2_rank_workspace_bytes(int64_t n, int64_t m)
{
    if (n < 0 || m < 0) return 0;
    return rank_layout(n, m).total;
}

int gf2_rank(const gf2_mat *A, int64_t *rank_host, unsigned flags, void *workspace, size_t ws_bytes, void *stream)
{
    return rank_impl(A, rank_host, flags, resolve_opts(nullptr), workspace, ws_bytes, static_cast<cudaStream_t>(stream));
}

int gf2_rank_ex(const gf2_mat *A, int64_t *rank_host, unsigned flags, const gf2_opts *opts, void *workspace,
                size_t ws_bytes, void *stream)
{
    const int st = check_opts(opts);
    if (st) return st;
    return rank_impl(A, rank_host, flags, resolve_opts(opts), workspace, ws_bytes, static_cast<cudaStream_t>(stream));
}

size_t gf2_decompose_host_workspace_bytes(int64_t n, int64_t m, int want_factors)
{
    if (n < 0 || m < 0) return 0;
    const int64_t mu = words_of(m), kmax = n < m ? n : m;
    size_t t = align_up((size_t)n * mu * 8) + align_up((size_t)n * 4) + align_up((size_t)kmax * 4) + kAlign;
    if (want_factors) t += align_up((size_t)words_of(kmax) * n * 8) + align_up((size_t)mu * kmax * 8);
    return t + gf2_decompose_workspace_bytes(n, m, want_factors);
}

int gf2_decompose_host(int64_t n, int64_t m, const uint64_t *A_host, int64_t lda, int32_t *perm_host,
                       int32_t *pivcols_host, int64_t *rank_host, uint64_t *L_host, uint64_t *E_host,
                       unsigned flags, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 0 || m < 0 || !perm_host || !rank_host) return GF2_ERR_ARG;
    if (n > 0 && m > 0 && (!A_host || lda < n)) return GF2_ERR_SHAPE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t mu = words_of(m), kmax = n < m ? n : m, lw = words_of(kmax);
    const bool factors = L_host || E_host;
    if (flags & ~GF2_NOCHECK) return GF2_ERR_ARG;
    // the padding bits are checked here, on the host copy, before any device
    // work, so that the device work is not interrupted by a synchronisation
    // to read them back
    if (!(flags & GF2_NOCHECK) && n > 0 && (m % 64)) {
        const uint64_t keep = last_word_mask(m), *last = A_host + (mu - 1) * lda;
        uint64_t bad = 0;
        for (int64_t i = 0; i < n; ++i) bad |= last[i] & ~keep;
        if (bad) return GF2_ERR_PADDING;
    }
    const size_t need = gf2_decompose_host_workspace_bytes(n, m, factors);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, need, &ws);
    if (st) return st;
    char *p = static_cast<char *>(ws);
    uint64_t *Ad = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)n * mu * 8);
    int32_t *permd = reinterpret_cast<int32_t *>(p); p += align_up((size_t)n * 4);
    int32_t *pivd = reinterpret_cast<int32_t *>(p); p += align_up((size_t)kmax * 4);
    int64_t *rkd = reinterpret_cast<int64_t *>(p); p += kAlign;
    uint64_t *Ld = nullptr, *Ed = nullptr;
    if (factors) {
        Ld = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)lw * n * 8);
        Ed = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)mu * kmax * 8);
    }
    const size_t dec = gf2_decompose_workspace_bytes(n, m, factors);
    if (n > 0 && mu > 0) {
        if (lda == n) CK(cudaMemcpyAsync(Ad, A_host, (size_t)n * mu * 8, cudaMemcpyHostToDevice, s));
        else CK(cudaMemcpy2DAsync(Ad, (size_t)n * 8, A_host, (size_t)lda * 8, (size_t)n * 8, (size_t)mu,
                                  cudaMemcpyHostToDevice, s));
    }
    gf2_mat A{Ad, n, m, n > 0 ? n : 1};
    gf2_mat L{Ld, n, kmax, n > 0 ? n : 1};
    gf2_mat E{Ed, kmax, m, kmax > 0 ? kmax : 1};
    st = decompose_impl(&A, permd, pivd, rkd, factors ? &L : nullptr, factors ? &E : nullptr, flags | GF2_NOCHECK,
                        resolve_opts(nullptr), p, dec, s);
    if (st) return st;
    CK(cudaMemcpyAsync(rank_host, rkd, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (n > 0) CK(cudaMemcpyAsync(perm_host, permd, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    if (kmax > 0 && pivcols_host) CK(cudaMemcpyAsync(pivcols_host, pivd, (size_t)kmax * 4, cudaMemcpyDeviceToHost, s));
    if (L_host && lw > 0) CK(cudaMemcpyAsync(L_host, Ld, (size_t)lw * n * 8, cudaMemcpyDeviceToHost, s));
    if (E_host && kmax > 0) CK(cudaMemcpyAsync(E_host, Ed, (size_t)mu * kmax * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return *rank_host < 0 ? GF2_ERR_TIMEOUT : GF2_OK;
}

// ------------------------------------------------------------ solve
size_t gf2_solve_workspace_bytes(int64_t n, int64_t m)
{
    if (n < 0 || m < 0) return 0;
    const int64_t kmax = n < m ? n : m, mu = words_of(m), nbl = words_of(kmax);
    return align_up((size_t)(n > 0 ? n : 1) * 8) + align_up((size_t)(kmax > 0 ? kmax : 1) * 8) +
           align_up((size_t)(nbl > 0 ? nbl : 1) * 64 * 8) + align_up((size_t)(mu > 0 ? mu : 1) * 64 * 8) +
           align_up((size_t)(mu + 1) * 4) + kAlign;
}

int gf2_solve(const gf2_mat *L, const gf2_mat *E, const int32_t *perm, const int32_t *pivcols, const int64_t *rank,
              const gf2_mat *B, gf2_mat *X, uint64_t *consistent, unsigned flags, void *workspace, size_t ws_bytes,
              void *stream)
{
    if (!mat_ok(L) || !mat_ok(E) || !mat_ok(B) || !mat_ok(X) || !rank || !consistent || (flags & ~GF2_NOCHECK))
        return GF2_ERR_ARG;
    const int64_t n = B->rows, m = X->rows, kmax = n < m ? n : m, nrhs = B->cols;
    if (nrhs < 1 || nrhs > 64 || X->cols != nrhs) return GF2_ERR_SHAPE;
    if (L->rows != n || L->cols != kmax || E->rows != kmax || E->cols != m) return GF2_ERR_SHAPE;
    if (n >= (1ll << 31) || m >= (1ll << 31)) return GF2_ERR_UNSUPPORTED;
    if ((n > 0 && (!perm || !B->w)) || (kmax > 0 && !pivcols) || (m > 0 && !X->w)) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, gf2_solve_workspace_bytes(n, m), &ws);
    if (st) return st;
    const int64_t mu = words_of(m), nbl = words_of(kmax);
    char *p = static_cast<char *>(ws);
    SolveCtx c{};
    c.v = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)(n > 0 ? n : 1) * 8);
    c.y = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)(kmax > 0 ? kmax : 1) * 8);
    c.linv = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)(nbl > 0 ? nbl : 1) * 64 * 8);
    c.uinv = reinterpret_cast<uint64_t *>(p); p += align_up((size_t)(mu > 0 ? mu : 1) * 64 * 8);
    c.qstart = reinterpret_cast<int32_t *>(p); p += align_up((size_t)(mu + 1) * 4);
    c.sync = reinterpret_cast<uint32_t *>(p);
    c.bad = reinterpret_cast<uint64_t *>(p + 64);
    c.perm = perm;
    c.pivcols = pivcols;
    c.rank = rank;
    c.L = L->w;
    c.ldl = L->ld;
    c.E = E->w;
    c.lde = E->ld;
    c.B = B->w;
    c.X = X->w;
    c.consistent = consistent;
    c.rhs_mask = nrhs == 64 ? ~0ull : ((1ull << nrhs) - 1);
    c.n = (int32_t)n;
    c.m = (int32_t)m;
    c.check = (flags & GF2_NOCHECK) ? 0 : 1;
    c.wait_limit = (uint32_t)device_wait_limit(1ll << 24);
    CK(cudaMemsetAsync(p, 0, kAlign, s));
    LAUNCH(GF2_KCLASS_SOLVE, launch_solve(c, s));
    // the status of the bounded waits and of the padding check
    std::lock_guard<std::mutex> lock(g_flag_mutex);
    if (!g_flag_host) {
        if (cudaHostAlloc(&g_flag_host, sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) return GF2_ERR_CUDA;
    }
    CK(cudaMemcpyAsync(g_flag_host, c.sync + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*g_flag_host & 1u) return GF2_ERR_TIMEOUT;
    if (*g_flag_host & 2u) return GF2_ERR_PADDING;
    return GF2_OK;
}

// ------------------------------------------------------------ batched
}  // extern "C"

namespace {

constexpr int64_t kBatchMaxDim = 4096;

struct BatchLayout {
    int grid, c;
    int64_t nmax, mumax, kmax_max;
    int64_t off_y, off_info, off_pivpanel, off_lint, off_eint, slice_words;
    size_t off_items, off_order, off_sync, off_scratch, total;
};

int64_t round_words(int64_t w) { return (w + 31) / 32 * 32; }  // 256-byte slices

int batch_layout(int count, const int64_t *n, const int64_t *m, bool factors, int c, BatchLayout *L)
{
    BatchLayout d{};
    d.c = c;
    for (int i = 0; i < count; ++i) {
        d.nmax = n[i] > d.nmax ? n[i] : d.nmax;
        d.mumax = words_of(m[i]) > d.mumax ? words_of(m[i]) : d.mumax;
        const int64_t k = n[i] < m[i] ? n[i] : m[i];
        d.kmax_max = k > d.kmax_max ? k : d.kmax_max;
    }
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GF2_ERR_CUDA;
    const int want = sms * batch_ctas_per_sm(c);
    d.grid = count < want ? (count > 0 ? count : 1) : want;
    const int64_t nm = d.nmax > 0 ? d.nmax : 1;
    const int64_t ldw = round_up_tiles(d.mumax > 0 ? d.mumax : 1);
    const int64_t ldl = words_of(d.kmax_max) > 0 ? words_of(d.kmax_max) : 1;
    int64_t o = round_words(nm * ldw);                       // W (tiled)
    d.off_y = o; o += round_words(nm);                        // Y
    d.off_info = o; o += round_words(2 * (int64_t)((sizeof(PanelInfo) + 7) / 8));
    d.off_pivpanel = o; o += round_words((nm + 1) / 2);
    d.off_lint = o; if (factors) o += round_words(nm * ldl);
    d.off_eint = o; if (factors) o += round_words((d.kmax_max > 0 ? d.kmax_max : 1) * ldw);
    d.slice_words = o;
    size_t b = 0;
    d.off_items = b; b += align_up((size_t)(count > 0 ? count : 1) * sizeof(BatchItem));
    d.off_order = b; b += align_up((size_t)(count > 0 ? count : 1) * 4);
    d.off_sync = b; b += kAlign;
    d.off_scratch = b; b += (size_t)d.grid * (size_t)d.slice_words * 8;
    d.total = b;
    *L = d;
    return GF2_OK;
}

// Matrices whose larger dimension is at least this go to the c = 8 kernel,
// the others to the c = 4 one (gf2_batched_autotune measures it).
std::atomic<int64_t> g_batch_c8_from{1024};

// A batch split by table size: class 0 (c = 4) and class 1 (c = 8), each with
// its own items, order, counter and scratch, one status word for both.
struct BatchPlan {
    std::vector<int> idx[2];
    BatchLayout lay[2];
    size_t off[2];
    size_t flag_off, total;
};

int batch_plan(int count, const int64_t *n, const int64_t *m, bool factors, int64_t c8_from, BatchPlan *P)
{
    for (int i = 0; i < count; ++i) P->idx[(n[i] > m[i] ? n[i] : m[i]) >= c8_from ? 1 : 0].push_back(i);
    size_t o = 0;
    for (int cls = 0; cls < 2; ++cls) {
        P->off[cls] = o;
        P->lay[cls] = BatchLayout{};
        const size_t k = P->idx[cls].size();
        if (!k) continue;
        std::vector<int64_t> ns(k), ms(k);
        for (size_t t = 0; t < k; ++t) {
            ns[t] = n[P->idx[cls][t]];
            ms[t] = m[P->idx[cls][t]];
        }
        const int st = batch_layout((int)k, ns.data(), ms.data(), factors, cls ? 8 : 4, &P->lay[cls]);
        if (st) return st;
        o += align_up(P->lay[cls].total);
    }
    P->flag_off = o;
    P->total = o + kAlign;
    return GF2_OK;
}

// A second stream for the c = 4 kernel beside the c = 8 one (per device),
// with the events that fork it from and join it to the caller's stream;
// the mutex is held from the fork to the join's enqueue.
struct BatchSide {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_batch_side_mutex;
std::vector<BatchSide> g_batch_side;

int batch_side(BatchSide **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
    if ((int)g_batch_side.size() <= dev) g_batch_side.resize(dev + 1);
    BatchSide &b = g_batch_side[dev];
    if (!b.s) {
        if (cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming) != cudaSuccess)
            return GF2_ERR_CUDA;
    }
    *out = &b;
    return GF2_OK;
}

}  // namespace

namespace gf2 {
static int batched_with(int count, const BatchItem *items, bool factors, unsigned flags, void *workspace,
                        size_t ws_bytes, cudaStream_t s, int64_t c8_from);
}  // namespace gf2

extern "C" {

size_t gf2_decompose_batched_workspace_bytes_ex(int count, const int64_t *n, const int64_t *m, int want_factors,
                                                const gf2_opts *opts)
{
    if (count < 0 || (count > 0 && (!n || !m)) || check_opts(opts)) return 0;
    const int64_t from = resolve_opts(opts).c8_from;
    BatchPlan P;
    if (batch_plan(count, n, m, want_factors != 0, from > 0 ? from : g_batch_c8_from.load(), &P) != GF2_OK) return 0;
    return P.total;
}

size_t gf2_decompose_batched_workspace_bytes(int count, const int64_t *n, const int64_t *m, int want_factors)
{
    return gf2_decompose_batched_workspace_bytes_ex(count, n, m, want_factors, nullptr);
}

int gf2_decompose_batched(int count, const gf2_mat *A, int32_t *const *perm, int32_t *const *pivcols, int64_t *rank,
                          const gf2_mat *L, const gf2_mat *E, unsigned flags, void *workspace, size_t ws_bytes,
                          void *stream)
{
    return gf2_decompose_batched_ex(count, A, perm, pivcols, rank, L, E, flags, nullptr, workspace, ws_bytes, stream);
}

int gf2_decompose_batched_ex(int count, const gf2_mat *A, int32_t *const *perm, int32_t *const *pivcols, int64_t *rank,
                             const gf2_mat *L, const gf2_mat *E, unsigned flags, const gf2_opts *opts, void *workspace,
                             size_t ws_bytes, void *stream)
{
    const int ost = check_opts(opts);
    if (ost) return ost;
    const int64_t from = resolve_opts(opts).c8_from;
    if (count < 0 || (flags & ~GF2_NOCHECK)) return GF2_ERR_ARG;
    if (count == 0) return GF2_OK;
    if (!A || !perm || !rank || (count > 0 && !pivcols)) return GF2_ERR_ARG;
    const bool factors = L || E;
    if (factors && (!L || !E)) return GF2_ERR_ARG;
    std::vector<BatchItem> items(count);
    for (int i = 0; i < count; ++i) {
        if (!mat_ok(&A[i]) || !perm[i]) return GF2_ERR_ARG;
        const int64_t n = A[i].rows, m = A[i].cols, k = n < m ? n : m;
        if (n > kBatchMaxDim || m > kBatchMaxDim) return GF2_ERR_UNSUPPORTED;
        if (k > 0 && !pivcols[i]) return GF2_ERR_ARG;
        if (factors && (!mat_ok(&L[i]) || !mat_ok(&E[i]) || L[i].rows != n || L[i].cols != k || E[i].rows != k ||
                        E[i].cols != m))
            return GF2_ERR_SHAPE;
        items[i] = BatchItem{A[i].w, A[i].ld, (int32_t)n, (int32_t)m, perm[i], pivcols[i], rank + i,
                             factors ? L[i].w : nullptr, factors ? L[i].ld : 0,
                             factors ? E[i].w : nullptr, factors ? E[i].ld : 0};
    }
    return gf2::batched_with(count, items.data(), factors, flags, workspace, ws_bytes, static_cast<cudaStream_t>(stream),
                             from > 0 ? from : g_batch_c8_from.load());
}

}  // extern "C"

namespace gf2 {

size_t decompose_batched_items_bytes(int count, const BatchItem *items, bool factors)
{
    std::vector<int64_t> ns(count), ms(count);
    for (int i = 0; i < count; ++i) {
        ns[i] = items[i].n;
        ms[i] = items[i].m;
    }
    BatchPlan P;
    if (batch_plan(count, ns.data(), ms.data(), factors, g_batch_c8_from.load(), &P) != GF2_OK) return 0;
    return P.total;
}

// Enqueues one class of a batch (its items, largest work first) on stream s.
static int enqueue_batch_class(const BatchPlan &P, int cls, const BatchItem *items, bool factors, unsigned flags, char *ws,
                        cudaStream_t s)
{
    const std::vector<int> &idx = P.idx[cls];
    const int count = (int)idx.size();
    if (!count) return GF2_OK;
    const BatchLayout &d = P.lay[cls];
    char *p = ws + P.off[cls];
    std::vector<BatchItem> sub(count);
    for (int t = 0; t < count; ++t) sub[t] = items[idx[t]];
    std::vector<int32_t> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto work = [&](int t) {
        const int64_t n = sub[t].n, m = sub[t].m;
        return (double)n * words_of(m) * (n < m ? n : m);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    // (copies from pageable memory: the calls return once the host arrays
    // have been staged)
    CK(cudaMemcpyAsync(p + d.off_items, sub.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p + d.off_order, order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(p + d.off_sync, 0, kAlign, s));
    BatchCtx b{};
    b.items = reinterpret_cast<const BatchItem *>(p + d.off_items);
    b.order = reinterpret_cast<const int32_t *>(p + d.off_order);
    b.next_item = reinterpret_cast<int32_t *>(p + d.off_sync);
    b.err = reinterpret_cast<uint32_t *>(ws + P.flag_off);
    b.scratch = reinterpret_cast<uint64_t *>(p + d.off_scratch);
    b.scratch_words = d.slice_words;
    b.off_y = d.off_y;
    b.off_info = d.off_info;
    b.off_pivpanel = d.off_pivpanel;
    b.off_lint = d.off_lint;
    b.off_eint = d.off_eint;
    b.count = count;
    b.factors = factors ? 1 : 0;
    b.check = (flags & GF2_NOCHECK) ? 0 : 1;
    LAUNCH(GF2_KCLASS_PANEL, launch_batch(b, d.grid, d.c, s));
    return GF2_OK;
}

static int batched_with(int count, const BatchItem *items, bool factors, unsigned flags, void *workspace,
                        size_t ws_bytes, cudaStream_t s, int64_t c8_from)
{
    if (count <= 0) return GF2_OK;
    std::vector<int64_t> ns(count), ms(count);
    for (int i = 0; i < count; ++i) {
        ns[i] = items[i].n;
        ms[i] = items[i].m;
    }
    BatchPlan P;
    int st = batch_plan(count, ns.data(), ms.data(), factors, c8_from, &P);
    if (st) return st;
    void *ws = nullptr;
    st = get_workspace(workspace, ws_bytes, P.total, &ws);
    if (st) return st;
    char *p = static_cast<char *>(ws);
    CK(cudaMemsetAsync(p + P.flag_off, 0, kAlign, s));
    if (!P.idx[0].empty() && !P.idx[1].empty()) {
        // both classes: the c = 8 kernel on s, the c = 4 kernel beside it
        std::lock_guard<std::mutex> lock(g_batch_side_mutex);
        BatchSide *side = nullptr;
        st = batch_side(&side);
        if (st) return st;
        CK(cudaEventRecord(side->fork, s));
        CK(cudaStreamWaitEvent(side->s, side->fork, 0));
        st = enqueue_batch_class(P, 1, items, factors, flags, p, s);
        if (!st) st = enqueue_batch_class(P, 0, items, factors, flags, p, side->s);
        CK(cudaEventRecord(side->join, side->s));
        CK(cudaStreamWaitEvent(s, side->join, 0));
        if (st) return st;
    } else {
        st = enqueue_batch_class(P, P.idx[1].empty() ? 0 : 1, items, factors, flags, p, s);
        if (st) return st;
    }
    if (flags & GF2_NOCHECK) return GF2_OK;
    return check_flag(reinterpret_cast<uint32_t *>(p + P.flag_off), s);  // the padding status
}

// The batched decomposition of items already checked (each n, m <= 4096).
// With GF2_NOCHECK the call does not synchronise the stream.
int decompose_batched_items(int count, const BatchItem *items, bool factors, unsigned flags, void *workspace,
                            size_t ws_bytes, void *stream)
{
    return batched_with(count, items, factors, flags, workspace, ws_bytes, static_cast<cudaStream_t>(stream),
                        g_batch_c8_from.load());
}

void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int64_t device_wait_limit(int64_t dflt)
{
    const int64_t v = g_wait_limit.load();
    return v > 0 ? v : dflt;
}

}  // namespace gf2

extern "C" {

// ------------------------------------------------------------ product
}  // extern "C"

namespace {

// Strassen-Winograd over the Four Russians product (the recursion of the
// paper's Section 5 for C = A B): a level applies while n, k and m are at
// least the cutoff, n is even, k is a whole even number of words and m an
// even number of words.
std::atomic<int64_t> g_strassen_cutoff{int64_t(1) << 62};  // off until tuned or set

struct CBView {
    uint64_t *w;
    int64_t ld;
};

int strassen_levels(int64_t n, int64_t k, int64_t mw, int64_t cutoff)
{
    int levels = 0;
    while (levels < 8) {
        const int64_t kw = words_of(k), m = 64 * mw;
        if (n < cutoff || k < cutoff || m < cutoff) break;
        if ((n & 1) || (kw & 1) || (mw & 1) || k != 64 * kw) break;
        n /= 2;
        k /= 2;
        mw /= 2;
        ++levels;
    }
    return levels;
}

// temporaries of the levels: S1..S4 (n/2 x k/2), T1..T4 (k/2 x m/2), X (n/2 x m/2)
size_t strassen_level_words(int64_t n, int64_t k, int64_t mw)
{
    const int64_t n2 = n / 2, kw2 = words_of(k) / 2, k2 = 64 * kw2, mw2 = mw / 2;
    return (size_t)(4 * n2 * kw2 + 4 * k2 * mw2 + n2 * mw2);
}

size_t strassen_bytes(int64_t n, int64_t k, int64_t mw, int levels)
{
    size_t words = 0;
    for (int l = 0; l < levels; ++l) {
        words += strassen_level_words(n, k, mw);
        n /= 2;
        k /= 2;
        mw /= 2;
    }
    return words * 8;
}

int mmm_rec(CBView C, CBView A, CBView B, int64_t n, int64_t k, int64_t mw, bool acc, int levels, uint64_t *tmp,
            cudaStream_t s)
{
    if (levels == 0) {
        MmmCtx c{A.w, A.ld, B.w, B.ld, C.w, C.ld, (int32_t)n, (int32_t)k, (int32_t)mw, acc ? kMmmXor : kMmmStore};
        LAUNCH(GF2_KCLASS_UPDATE, launch_mmm(c, s));
        return GF2_OK;
    }
    const int64_t n2 = n / 2, kw2 = words_of(k) / 2, k2 = 64 * kw2, mw2 = mw / 2;
    if (!acc) CK(cudaMemset2DAsync(C.w, (size_t)C.ld * 8, 0, (size_t)n * 8, (size_t)mw, s));
    const CBView A11{A.w, A.ld}, A12{A.w + kw2 * A.ld, A.ld}, A21{A.w + n2, A.ld}, A22{A.w + kw2 * A.ld + n2, A.ld};
    const CBView B11{B.w, B.ld}, B12{B.w + mw2 * B.ld, B.ld}, B21{B.w + k2, B.ld}, B22{B.w + mw2 * B.ld + k2, B.ld};
    const CBView C11{C.w, C.ld}, C12{C.w + mw2 * C.ld, C.ld}, C21{C.w + n2, C.ld}, C22{C.w + mw2 * C.ld + n2, C.ld};
    uint64_t *p = tmp;
    auto take = [&](int64_t ld, int64_t words) {
        CBView v{p, ld};
        p += ld * words;
        return v;
    };
    const CBView S1 = take(n2, kw2), S2 = take(n2, kw2), S3 = take(n2, kw2), S4 = take(n2, kw2);
    const CBView T1 = take(k2, mw2), T2 = take(k2, mw2), T3 = take(k2, mw2), T4 = take(k2, mw2);
    const CBView X = take(n2, mw2);
    uint64_t *next = p;  // the sub-products' own temporaries
    auto add = [&](CBView D, CBView P, CBView Q, int64_t rows, int64_t words) {
        return launch_xor(D.w, D.ld, P.w, P.ld, Q.w, Q.ld, rows, words, s);
    };
    LAUNCH(GF2_KCLASS_LAYOUT, add(S1, A21, A22, n2, kw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(S2, S1, A11, n2, kw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(S3, A11, A21, n2, kw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(S4, A12, S2, n2, kw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(T1, B12, B11, k2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(T2, B22, T1, k2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(T3, B22, B12, k2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(T4, T2, B21, k2, mw2));
    int st;
    // C11 = P1 + P2
    if ((st = mmm_rec(X, A11, B11, n2, k2, mw2, false, levels - 1, next, s))) return st;  // X = P1
    LAUNCH(GF2_KCLASS_LAYOUT, add(C11, C11, X, n2, mw2));
    if ((st = mmm_rec(C11, A12, B21, n2, k2, mw2, true, levels - 1, next, s))) return st;  // + P2
    // U2 = P1 + P6 into C12, C21, C22
    if ((st = mmm_rec(X, S2, T2, n2, k2, mw2, true, levels - 1, next, s))) return st;
    LAUNCH(GF2_KCLASS_LAYOUT, add(C12, C12, X, n2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(C21, C21, X, n2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(C22, C22, X, n2, mw2));
    // P7 into C21, C22
    if ((st = mmm_rec(X, S3, T3, n2, k2, mw2, false, levels - 1, next, s))) return st;
    LAUNCH(GF2_KCLASS_LAYOUT, add(C21, C21, X, n2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(C22, C22, X, n2, mw2));
    // P5 into C12, C22
    if ((st = mmm_rec(X, S1, T1, n2, k2, mw2, false, levels - 1, next, s))) return st;
    LAUNCH(GF2_KCLASS_LAYOUT, add(C12, C12, X, n2, mw2));
    LAUNCH(GF2_KCLASS_LAYOUT, add(C22, C22, X, n2, mw2));
    // P3 into C12, P4 into C21
    if ((st = mmm_rec(C12, S4, B22, n2, k2, mw2, true, levels - 1, next, s))) return st;
    if ((st = mmm_rec(C21, A22, T4, n2, k2, mw2, true, levels - 1, next, s))) return st;
    return GF2_OK;
}

size_t mmm_tensor_bytes(int64_t n, int64_t k, int64_t m)
{
    const size_t rb = (size_t)mma_row_bytes(mma_pad(k > 0 ? k : 1));
    return align_up((size_t)mma_pad(n > 0 ? n : 1) * rb) + align_up((size_t)mma_pad(m > 0 ? m : 1) * rb) + kAlign;
}

// the tensor-core product only when the flags ask for it: measured on the
// GB300 the Four Russians product is faster at every size
bool mmm_use_tensor(int64_t k, unsigned flags)
{
    return (flags & GF2_MMM_TENSOR) && !(flags & GF2_MMM_TABLES) && k < (1ll << 24);
}

// cutoff 0: the process-wide one
int mmm_levels(int64_t n, int64_t k, int64_t m, unsigned flags, int64_t cutoff)
{
    if (flags & (GF2_MMM_TABLES | GF2_MMM_TENSOR)) return 0;
    return strassen_levels(n, k, words_of(m), cutoff > 0 ? cutoff : g_strassen_cutoff.load());
}

size_t mmm_bytes(int64_t n, int64_t k, int64_t m, unsigned flags, int64_t cutoff)
{
    if (n < 0 || k < 0 || m < 0) return 0;
    if (mmm_use_tensor(k, flags)) return mmm_tensor_bytes(n, k, m);
    return align_up(strassen_bytes(n, k, words_of(m), mmm_levels(n, k, m, flags, cutoff))) + kAlign;
}

int mmm_impl(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags, int64_t cutoff,
             void *workspace, size_t ws_bytes, void *stream);

// a backend flag and a backend option together are an error; otherwise the
// option's backend joins the flags
int mmm_opts_flags(unsigned flags, const gf2_opts *opts, unsigned *out, int64_t *cutoff)
{
    const int st = check_opts(opts);
    if (st) return st;
    const CallOpts o = resolve_opts(opts);
    if (o.backend && (flags & (GF2_MMM_TABLES | GF2_MMM_TENSOR))) return GF2_ERR_ARG;
    *out = flags | o.backend;
    *cutoff = o.cutoff;
    return GF2_OK;
}

}  // namespace

extern "C" {

size_t gf2_mmm_workspace_bytes(int64_t n, int64_t k, int64_t m, unsigned flags)
{
    return mmm_bytes(n, k, m, flags, 0);
}

size_t gf2_mmm_workspace_bytes_ex(int64_t n, int64_t k, int64_t m, unsigned flags, const gf2_opts *opts)
{
    unsigned f = 0;
    int64_t cutoff = 0;
    if (mmm_opts_flags(flags, opts, &f, &cutoff)) return 0;
    return mmm_bytes(n, k, m, f, cutoff);
}

int gf2_mmm(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags, void *workspace,
            size_t ws_bytes, void *stream)
{
    return mmm_impl(A, B, C, accumulate, flags, 0, workspace, ws_bytes, stream);
}

int gf2_mmm_ex(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags, const gf2_opts *opts,
               void *workspace, size_t ws_bytes, void *stream)
{
    unsigned f = 0;
    int64_t cutoff = 0;
    const int st = mmm_opts_flags(flags, opts, &f, &cutoff);
    if (st) return st;
    return mmm_impl(A, B, C, accumulate, f, cutoff, workspace, ws_bytes, stream);
}

}  // extern "C"

namespace {

int mmm_impl(const gf2_mat *A, const gf2_mat *B, gf2_mat *C, int accumulate, unsigned flags, int64_t cutoff,
             void *workspace, size_t ws_bytes, void *stream)
{
    if (!mat_ok(A) || !mat_ok(B) || !mat_ok(C) || (flags & ~(GF2_NOCHECK | GF2_MMM_TABLES | GF2_MMM_TENSOR)))
        return GF2_ERR_ARG;
    if ((flags & GF2_MMM_TABLES) && (flags & GF2_MMM_TENSOR)) return GF2_ERR_ARG;
    if (A->cols != B->rows || C->rows != A->rows || C->cols != B->cols) return GF2_ERR_SHAPE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = A->rows, k = A->cols, m = B->cols;
    if (n >= (1ll << 31) || k >= (1ll << 31) || m >= (1ll << 31)) return GF2_ERR_UNSUPPORTED;
    if (n == 0 || m == 0) return GF2_OK;
    const int64_t kw = words_of(k), mw = words_of(m);
    if (k == 0) {
        if (!accumulate) CK(cudaMemset2DAsync(C->w, (size_t)C->ld * 8, 0, (size_t)n * 8, (size_t)mw, s));
        return GF2_OK;
    }
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, mmm_bytes(n, k, m, flags, cutoff), &ws);
    if (st) return st;
    char *p = static_cast<char *>(ws);
    const bool tensor = mmm_use_tensor(k, flags);
    const int levels = tensor ? 0 : mmm_levels(n, k, m, flags, cutoff);
    uint32_t *flag = reinterpret_cast<uint32_t *>(
        p + (tensor ? mmm_tensor_bytes(n, k, m) - kAlign : align_up(strassen_bytes(n, k, mw, levels))));
    if (!(flags & GF2_NOCHECK)) {
        CK(cudaMemsetAsync(flag, 0, sizeof(uint32_t), s));
        LAUNCH(GF2_KCLASS_LAYOUT, launch_check_last_block(A->w + (kw - 1) * A->ld, (int)n, last_word_mask(k), flag, s));
        LAUNCH(GF2_KCLASS_LAYOUT, launch_check_last_block(B->w + (mw - 1) * B->ld, (int)k, last_word_mask(m), flag, s));
        if (accumulate)
            LAUNCH(GF2_KCLASS_LAYOUT, launch_check_last_block(C->w + (mw - 1) * C->ld, (int)n, last_word_mask(m), flag, s));
        st = check_flag(flag, s);
        if (st) return st;
    }
    if (tensor) {
        // expand to e2m1 entries, then the tcgen05 product; its device waits
        // are bounded and report through the word after the padding flag,
        // read back with one synchronisation of the stream
        const size_t kp = (size_t)mma_pad(k);
        uint8_t *A8 = reinterpret_cast<uint8_t *>(p);
        uint8_t *B8 = A8 + align_up((size_t)mma_pad(n) * (size_t)mma_row_bytes((int64_t)kp));
        uint32_t *err = flag + 1;
        CK(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
        LAUNCH(GF2_KCLASS_LAYOUT, launch_expand_operands(A->w, A->ld, B->w, B->ld, (int)n, (int)k, (int)m, A8, B8, s));
        LAUNCH(GF2_KCLASS_UPDATE, launch_umma_product(A8, B8, (int)mma_pad(n), (int)mma_pad(m), (int)kp, C->w, C->ld,
                                                      (int)n, (int)m, accumulate, err, s));
        st = check_flag(err, s);
        return st == GF2_ERR_PADDING ? GF2_ERR_TIMEOUT : st;
    }
    return mmm_rec(CBView{C->w, C->ld}, CBView{A->w, A->ld}, CBView{B->w, B->ld}, n, k, mw, accumulate != 0, levels,
                   reinterpret_cast<uint64_t *>(p), s);
}

}  // namespace

extern "C" {

int gf2_mmm_set_strassen_cutoff(int64_t cutoff)
{
    if (cutoff < 128) return GF2_ERR_ARG;
    g_strassen_cutoff.store(cutoff);
    return GF2_OK;
}

int64_t gf2_mmm_strassen_cutoff(void) { return g_strassen_cutoff.load(); }

}  // extern "C"

namespace {

__global__ void k_fill_words(uint64_t *w, int64_t count, uint64_t seed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);  // SplitMix64 finaliser
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        w[i] = z ^ (z >> 31);
    }
}

// best of `reps` timings (ms) of one square product of size d, at `levels`
int time_product(uint64_t *A, uint64_t *B, uint64_t *C, uint64_t *tmp, int64_t d, int levels, int reps, cudaStream_t s,
                 float *best)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GF2_ERR_CUDA;
    *best = 1e30f;
    int st = GF2_OK;
    for (int r = 0; r < reps + 1 && st == GF2_OK; ++r) {  // the first run warms up
        if (cudaEventRecord(e0, s) != cudaSuccess) st = GF2_ERR_CUDA;
        if (st == GF2_OK)
            st = mmm_rec(CBView{C, d}, CBView{A, d}, CBView{B, d}, d, d, d / 64, false, levels, tmp, s);
        if (st == GF2_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            st = GF2_ERR_CUDA;
        float ms = 0;
        if (st == GF2_OK && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < *best) *best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace

extern "C" {

size_t gf2_fp_decompose_workspace_bytes(int64_t n, int64_t m)
{
    if (n < 0 || m < 0) return 0;
    return fp_workspace_bytes(n, m);
}

int gf2_fp_is_prime(uint32_t p)
{
    if (p < 2) return 0;
    for (uint32_t d = 2; (uint64_t)d * d <= p; ++d)
        if (p % d == 0) return 0;
    return 1;
}

int gf2_fp_decompose(const uint32_t *A, int64_t lda, int64_t n, int64_t m, uint32_t p, int32_t *perm,
                     int32_t *pivcols, int64_t *rank, uint32_t *L, int64_t ldl, uint32_t *E, int64_t lde,
                     unsigned flags, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 0 || m < 0 || !rank || (flags & ~GF2_NOCHECK)) return GF2_ERR_ARG;
    if (p < 2 || p >= (1u << 31) || !gf2_fp_is_prime(p)) return GF2_ERR_ARG;
    if (n >= (1ll << 31) || m >= (1ll << 31)) return GF2_ERR_UNSUPPORTED;
    const int64_t k = n < m ? n : m;
    if ((n > 0 && !perm) || (k > 0 && !pivcols) || (n > 0 && m > 0 && !A)) return GF2_ERR_ARG;
    if (n > 0 && m > 0 && lda < m) return GF2_ERR_SHAPE;
    if (L && k > 0 && ldl < k) return GF2_ERR_SHAPE;
    if (E && k > 0 && lde < m) return GF2_ERR_SHAPE;
    void *ws = nullptr;
    int st = get_workspace(workspace, ws_bytes, fp_workspace_bytes(n, m), &ws);
    if (st) return st;
    return fp_decompose(A, lda, n, m, p, perm, pivcols, rank, L, ldl, E, lde, !(flags & GF2_NOCHECK), ws,
                        (uint32_t)device_wait_limit(1ll << 24), static_cast<cudaStream_t>(stream));
}

int gf2_tensor_peak(int64_t iters, double *tflops, void *stream)
{
    if (iters < 1 || iters > (1 << 30) || !tflops) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t *err = nullptr;
    CK(cudaMalloc(&err, sizeof(uint32_t)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = GF2_OK;
    if (cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || launch_umma_peak(sms, 16, err, s) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess || launch_umma_peak(sms, (int)iters, err, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        st = GF2_ERR_CUDA;
    float ms = 0.f;
    if (!st && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = GF2_ERR_CUDA;
    if (!st) {
        st = check_flag(err, s);
        if (st == GF2_ERR_PADDING) st = GF2_ERR_TIMEOUT;
    }
    if (!st) *tflops = (double)sms * (double)iters * umma_peak_flops_per_iter() / ((double)ms * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(err);
    return st;
}

int gf2_mmm_autotune(int64_t max_dim, int64_t *cutoff, void *stream)
{
    if (!cutoff || max_dim < 1024) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t top = 1024;
    while (top * 2 <= max_dim && top < 32768) top *= 2;
    const size_t mat = (size_t)top * (top / 64) * 8;
    const size_t tmp = strassen_bytes(top, top, top / 64, 1);
    char *buf = nullptr;
    if (cudaMalloc(&buf, 3 * mat + tmp) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ERR_NOMEM;
    }
    uint64_t *A = reinterpret_cast<uint64_t *>(buf), *B = A + mat / 8, *C = B + mat / 8, *T = C + mat / 8;
    int st = GF2_OK;
    k_fill_words<<<1024, 256, 0, s>>>(A, (int64_t)(2 * mat / 8), 0x1209519812095198ull);
    if (cudaGetLastError() != cudaSuccess) st = GF2_ERR_CUDA;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    // the smallest size from which one level is faster at that size and at
    // every larger size tried
    int64_t chosen = int64_t(1) << 62;
    for (int64_t d = top; d >= 2048 && st == GF2_OK; d /= 2) {
        float direct = 0, one = 0;
        const int reps = d >= 16384 ? 2 : 4;
        st = time_product(A, B, C, T, d, 0, reps, s, &direct);
        if (st == GF2_OK) st = time_product(A, B, C, T, d, 1, reps, s, &one);
        if (st != GF2_OK || one >= direct) break;
        chosen = d;
    }
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (st != GF2_OK) return st;
    g_strassen_cutoff.store(chosen);
    *cutoff = chosen;
    return GF2_OK;
}

int64_t gf2_launch_count(void) { return g_launches.load(); }

static_assert(GF2_OP_UPDATES == kOpUpdates && GF2_OP_YROWS == kOpYRows && GF2_OP_LOOKUPS8 == kOpLookups8 &&
                  GF2_OP_LOOKUPS4 == kOpLookups4 && GF2_OP_TABLE8 == kOpTable8 && GF2_OP_TABLE4 == kOpTable4 &&
                  GF2_OP_MMM_LOOKUPS == kOpMmmLookups && GF2_OP_MMM_TABLE == kOpMmmTable &&
                  GF2_OP_MMM_ADDS == kOpMmmAdds && GF2_NUM_OPS == kNumOps,
              "operation counter kinds of the ABI and of the kernels");

int gf2_op_counts(uint64_t *out, int count, int reset)
{
    if (!out || count < 0) return GF2_ERR_ARG;
#ifdef GF2_COUNT_OPS
    if (cudaDeviceSynchronize() != cudaSuccess) return GF2_ERR_CUDA;
    unsigned long long acc[kNumOps] = {};
    if (read_update_ops(acc, reset != 0) != cudaSuccess || read_mmm_ops(acc, reset != 0) != cudaSuccess ||
        read_factor_ops(acc, reset != 0) != cudaSuccess)
        return GF2_ERR_CUDA;
    for (int i = 0; i < count && i < kNumOps; ++i) out[i] = acc[i];
    return GF2_OK;
#else
    (void)reset;
    return GF2_ERR_UNSUPPORTED;
#endif
}

int gf2_debug_set_wait_limit(int64_t polls)
{
    if (polls < 0 || polls > UINT32_MAX) return GF2_ERR_ARG;
    g_wait_limit.store(polls);
    return GF2_OK;
}

int gf2_trace_read(uint64_t *out, int64_t count, int reset)
{
    if (!out || count < 0) return GF2_ERR_ARG;
#ifdef GF2_TRACE
    if (cudaDeviceSynchronize() != cudaSuccess) return GF2_ERR_CUDA;
    std::vector<unsigned long long> a(kTrSlots * kTraceMaxPanels), b(kTrSlots * kTraceMaxPanels),
        f(kTrSlots * kTraceMaxPanels);
    if (read_panel_trace(a.data(), reset != 0) != cudaSuccess || read_update_trace(b.data(), reset != 0) != cudaSuccess ||
        read_factor_trace(f.data(), reset != 0) != cudaSuccess)
        return GF2_ERR_CUDA;
    // each slot lives in one translation unit per schedule: the panel phases
    // in the panel kernel's, the launch spans in the update kernels', and
    // everything of a persistent run in its kernel's (a run writes one of
    // them; the larger value is the one written); start slots are kept
    // complemented on the device
    for (int64_t i = 0; i < count && i < (int64_t)a.size(); ++i) {
        const int slot = (int)(i / kTraceMaxPanels);
        unsigned long long v = trace_panel_slot(slot) ? a[i] : b[i];
        if (f[i] > v) v = f[i];
        if ((slot == kTrNextStart || slot == kTrRestStart) && v) v = ~v;
        out[i] = v;
    }
    return GF2_OK;
#else
    (void)reset;
    return GF2_ERR_UNSUPPORTED;
#endif
}

int gf2_timing_enable(int on)
{
    g_timing.store(on != 0);
    return GF2_OK;
}

int gf2_timing_reset(void)
{
    std::lock_guard<std::mutex> lock(g_timing_mutex);
    for (auto &t : g_timed) {
        g_event_pool.push_back(t.a);
        g_event_pool.push_back(t.b);
    }
    g_timed.clear();
    return GF2_OK;
}

int gf2_timing_read(int kernel_class, double *total_ms, int64_t *launches)
{
    if (!total_ms || !launches || kernel_class < 0 || kernel_class >= GF2_NUM_KCLASSES) return GF2_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_timing_mutex);
    double sum = 0;
    int64_t cnt = 0;
    for (auto &t : g_timed) {
        if (t.cls != kernel_class) continue;
        if (cudaEventSynchronize(t.b) != cudaSuccess) return GF2_ERR_CUDA;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) return GF2_ERR_CUDA;
        sum += ms;
        ++cnt;
    }
    *total_ms = sum;
    *launches = cnt;
    return GF2_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batched autotuner
extern "C" {

int gf2_batched_set_c8_from(int64_t dim)
{
    if (dim < 1) return GF2_ERR_ARG;
    g_batch_c8_from.store(dim);
    return GF2_OK;
}

int64_t gf2_batched_c8_from(void) { return g_batch_c8_from.load(); }

int gf2_batched_autotune(int64_t max_dim, int64_t *c8_from, float *times_ms, void *stream)
{
    if (!c8_from || max_dim < 128) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GF2_ERR_CUDA;
    const int64_t top = max_dim < kBatchMaxDim ? max_dim : kBatchMaxDim;
    std::vector<int64_t> dims;
    for (int64_t d = 128; d <= top; d *= 2) dims.push_back(d);
    // time both table sizes on a batch of square d x d matrices (random
    // words), the smallest d first; c = 8 wins from the first d at which it
    // is faster there and at every larger d
    std::vector<float> t4(dims.size(), 0.f), t8(dims.size(), 0.f);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GF2_ERR_CUDA;
    int st = GF2_OK;
    for (size_t di = 0; di < dims.size() && st == GF2_OK; ++di) {
        const int64_t d = dims[di], mu = d / 64;
        const int count = (int)(d >= 2048 ? 2 * sms : 4 * sms);
        const size_t mat = (size_t)d * mu * 8;
        std::vector<BatchItem> items(count);
        std::vector<int64_t> ns(count, d), ms(count, d);
        BatchPlan P4, P8;
        if ((st = batch_plan(count, ns.data(), ms.data(), true, int64_t(1) << 62, &P4)) != GF2_OK) break;
        if ((st = batch_plan(count, ns.data(), ms.data(), true, 0, &P8)) != GF2_OK) break;
        const size_t wsb = P4.total > P8.total ? P4.total : P8.total;
        const size_t per = 3 * align_up(mat) + align_up((size_t)d * 4) * 2 + kAlign;  // A, L, E, perm, pivcols
        char *buf = nullptr;
        if (cudaMalloc(&buf, per * count + (size_t)count * 8 + wsb) != cudaSuccess) {
            cudaGetLastError();
            st = GF2_ERR_NOMEM;
            break;
        }
        int64_t *ranks = reinterpret_cast<int64_t *>(buf + per * count);
        char *ws = buf + per * count + (size_t)count * 8;
        for (int i = 0; i < count; ++i) {
            char *q = buf + per * i;
            uint64_t *A = reinterpret_cast<uint64_t *>(q);
            uint64_t *L = reinterpret_cast<uint64_t *>(q + align_up(mat));
            uint64_t *E = reinterpret_cast<uint64_t *>(q + 2 * align_up(mat));
            int32_t *perm = reinterpret_cast<int32_t *>(q + 3 * align_up(mat));
            int32_t *piv = perm + align_up((size_t)d * 4) / 4;
            items[i] = BatchItem{A, d, (int32_t)d, (int32_t)d, perm, piv, ranks + i, L, d, E, d};
            k_fill_words<<<256, 256, 0, s>>>(A, (int64_t)(mat / 8), 0x5198ull * 1000003ull + (uint64_t)i);
        }
        if (cudaGetLastError() != cudaSuccess) st = GF2_ERR_CUDA;
        g_launches.fetch_add(count, std::memory_order_relaxed);
        for (int variant = 0; variant < 2 && st == GF2_OK; ++variant) {
            const int64_t from = variant ? 0 : (int64_t(1) << 62);
            float best = 1e30f;
            for (int r = 0; r < 3 && st == GF2_OK; ++r) {  // the first run warms up
                if (cudaEventRecord(e0, s) != cudaSuccess) st = GF2_ERR_CUDA;
                if (st == GF2_OK) st = gf2::batched_with(count, items.data(), true, GF2_NOCHECK, ws, wsb, s, from);
                if (st == GF2_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    st = GF2_ERR_CUDA;
                float ms = 0;
                if (st == GF2_OK && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
            }
            (variant ? t8 : t4)[di] = best;
        }
        cudaStreamSynchronize(s);
        cudaFree(buf);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GF2_OK) return st;
    int64_t chosen = int64_t(1) << 62;
    for (size_t di = dims.size(); di-- > 0;) {
        if (t8[di] < t4[di]) chosen = dims[di];
        else break;
    }
    if (times_ms)
        for (size_t di = 0; di < dims.size(); ++di) {
            times_ms[2 * di] = t4[di];
            times_ms[2 * di + 1] = t8[di];
        }
    g_batch_c8_from.store(chosen);
    *c8_from = chosen;
    return GF2_OK;
}

}  // extern "C"

// ------------------------------------------------------------ factor handle
namespace {

// What a gf2_factors owns: one device allocation holding perm, pivcols, the
// rank, L, E, the per-block data of the last decomposition (the block form's
// Z, T_j, T_j^-1, pivot rows and bits per 64-column block, as the
// decomposition leaves them) and the scratch of its calls (the largest of
// the decomposition's, the solve's, the reduced form's and the null
// space's workspaces); and, once a null space was asked for, a copy of the
// reduced form.
struct FactorsImpl {
    int device;
    void *mem;
    void *scratch;
    size_t scratch_bytes;
    PanelInfo *blocks;
    int64_t nblocks;
    size_t info_offset;  // of the decomposition's per-block data in its workspace
    uint64_t *R;         // k x m reduced form (ld k), for the null space
};

bool factors_ok(const gf2_factors *F)
{
    return F && F->impl && F->n >= 0 && F->m >= 0;
}

}  // namespace

extern "C" {

int gf2_factors_alloc(gf2_factors *F, int64_t n, int64_t m, unsigned flags)
{
    if (!F || n < 0 || m < 0 || (flags & ~GF2_FACTORS_RANK_ONLY)) return GF2_ERR_ARG;
    if (n >= (1ll << 31) - 64 || m >= (1ll << 31) - 64) return GF2_ERR_UNSUPPORTED;
    const bool factors = !(flags & GF2_FACTORS_RANK_ONLY);
    const int64_t kmax = n < m ? n : m, mu = words_of(m), lw = words_of(kmax);
    const int64_t ldl = n > 0 ? n : 1, lde = kmax > 0 ? kmax : 1;
    size_t scratch = gf2_decompose_workspace_bytes(n, m, factors);
    const size_t more[3] = {gf2_solve_workspace_bytes(n, m), gf2_rref_workspace_bytes(kmax, m),
                            gf2_nullspace_workspace_bytes(m, 0)};
    for (size_t x : more) scratch = x > scratch ? x : scratch;
    size_t o = 0;
    const size_t oPerm = o; o += align_up((size_t)(n > 0 ? n : 1) * 4);
    const size_t oPiv = o; o += align_up((size_t)(kmax > 0 ? kmax : 1) * 4);
    const size_t oRank = o; o += kAlign;
    const size_t oL = o; if (factors) o += align_up((size_t)lw * ldl * 8);
    const size_t oE = o; if (factors) o += align_up((size_t)mu * lde * 8);
    const size_t oBlk = o; o += align_up((size_t)(mu > 0 ? mu : 1) * sizeof(PanelInfo));
    const size_t oScr = o; o += align_up(scratch);
    auto *impl = new (std::nothrow) FactorsImpl{};
    if (!impl) return GF2_ERR_NOMEM;
    if (cudaGetDevice(&impl->device) != cudaSuccess) {
        delete impl;
        return GF2_ERR_CUDA;
    }
    if (cudaMalloc(&impl->mem, o) != cudaSuccess) {
        cudaGetLastError();
        delete impl;
        return GF2_ERR_NOMEM;
    }
    char *base = static_cast<char *>(impl->mem);
    impl->scratch = base + oScr;
    impl->scratch_bytes = align_up(scratch);
    impl->blocks = reinterpret_cast<PanelInfo *>(base + oBlk);
    impl->nblocks = mu;
    impl->info_offset = decomp_layout(n, m, factors).oInfo;
    impl->R = nullptr;
    gf2_factors f{};
    f.n = n;
    f.m = m;
    f.rank = -1;
    f.perm = reinterpret_cast<int32_t *>(base + oPerm);
    f.pivcols = reinterpret_cast<int32_t *>(base + oPiv);
    f.rank_dev = reinterpret_cast<int64_t *>(base + oRank);
    f.L = gf2_mat{factors ? reinterpret_cast<uint64_t *>(base + oL) : nullptr, n, kmax, ldl};
    f.E = gf2_mat{factors ? reinterpret_cast<uint64_t *>(base + oE) : nullptr, kmax, m, lde};
    f.flags = flags;
    f.impl = impl;
    // (zero factors: a decomposition writes them all; this keeps the padding
    // of L and E defined)
    if (cudaMemset(impl->mem, 0, o) != cudaSuccess) {
        cudaFree(impl->mem);
        delete impl;
        return GF2_ERR_CUDA;
    }
    *F = f;
    return GF2_OK;
}

int gf2_factors_free(gf2_factors *F)
{
    if (!F) return GF2_ERR_ARG;
    auto *impl = static_cast<FactorsImpl *>(F->impl);
    if (impl) {
        int cur = 0;
        const bool have = cudaGetDevice(&cur) == cudaSuccess;
        cudaSetDevice(impl->device);
        cudaDeviceSynchronize();
        cudaFree(impl->R);
        cudaFree(impl->mem);
        if (have) cudaSetDevice(cur);
        delete impl;
    }
    *F = gf2_factors{};
    return GF2_OK;
}

int gf2_factors_decompose(gf2_factors *F, const gf2_mat *A, unsigned flags, const gf2_opts *opts, void *stream)
{
    if (!factors_ok(F) || !A) return GF2_ERR_ARG;
    int st = check_opts(opts);
    if (st) return st;
    if (A->rows != F->n || A->cols != F->m) return GF2_ERR_SHAPE;
    auto *impl = static_cast<FactorsImpl *>(F->impl);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool factors = F->L.w != nullptr;
    F->rank = -1;
    st = decompose_impl(A, F->perm, F->pivcols, F->rank_dev, factors ? &F->L : nullptr, factors ? &F->E : nullptr,
                        flags, resolve_opts(opts), impl->scratch, impl->scratch_bytes, s);
    if (st) return st;
    if (impl->nblocks > 0 && F->n > 0)
        CK(cudaMemcpyAsync(impl->blocks, static_cast<char *>(impl->scratch) + impl->info_offset,
                           (size_t)impl->nblocks * sizeof(PanelInfo), cudaMemcpyDeviceToDevice, s));
    return GF2_OK;
}

int gf2_factors_rank(gf2_factors *F, int64_t *rank_host, void *stream)
{
    if (!factors_ok(F) || !rank_host) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(rank_host, F->rank_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    F->rank = *rank_host;
    return *rank_host < 0 ? GF2_ERR_TIMEOUT : GF2_OK;
}

int gf2_factors_solve(const gf2_factors *F, const gf2_mat *B, gf2_mat *X, uint64_t *consistent, unsigned flags,
                      void *stream)
{
    if (!factors_ok(F) || !F->L.w || !F->E.w || !B || !X) return GF2_ERR_ARG;
    if (B->rows != F->n || X->rows != F->m) return GF2_ERR_SHAPE;
    auto *impl = static_cast<FactorsImpl *>(F->impl);
    return gf2_solve(&F->L, &F->E, F->perm, F->pivcols, F->rank_dev, B, X, consistent, flags, impl->scratch,
                     impl->scratch_bytes, stream);
}

int gf2_factors_rref(const gf2_factors *F, gf2_mat *R, void *stream)
{
    if (!factors_ok(F) || !F->E.w || !R || !mat_ok(R)) return GF2_ERR_ARG;
    const int64_t k = F->E.rows, m = F->m;
    if (R->rows != k || R->cols != m) return GF2_ERR_SHAPE;
    if (k == 0 || m == 0) return GF2_OK;
    if (!R->w) return GF2_ERR_ARG;
    auto *impl = static_cast<FactorsImpl *>(F->impl);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpy2DAsync(R->w, (size_t)R->ld * 8, F->E.w, (size_t)F->E.ld * 8, (size_t)k * 8, (size_t)words_of(m),
                         cudaMemcpyDeviceToDevice, s));
    return gf2_rref(R, F->pivcols, impl->scratch, impl->scratch_bytes, stream);
}

int gf2_factors_nullspace(gf2_factors *F, gf2_mat *N, void *stream)
{
    if (!factors_ok(F) || !F->E.w || !N) return GF2_ERR_ARG;
    auto *impl = static_cast<FactorsImpl *>(F->impl);
    int64_t r = 0;
    int st = gf2_factors_rank(F, &r, stream);
    if (st) return st;
    const int64_t k = F->E.rows, m = F->m;
    if (!mat_ok(N) || N->rows != m || N->cols != m - r) return GF2_ERR_SHAPE;
    if (m == 0 || m == r) return GF2_OK;
    if (!impl->R && k > 0) {
        if (cudaMalloc(&impl->R, (size_t)k * words_of(m) * 8) != cudaSuccess) {
            cudaGetLastError();
            impl->R = nullptr;
            return GF2_ERR_NOMEM;
        }
    }
    gf2_mat R{impl->R, k, m, k > 0 ? k : 1};
    if (k > 0) {
        st = gf2_factors_rref(F, &R, stream);
        if (st) return st;
    }
    return gf2_nullspace(&R, F->pivcols, r, N, impl->scratch, impl->scratch_bytes, stream);
}

}  // extern "C"
