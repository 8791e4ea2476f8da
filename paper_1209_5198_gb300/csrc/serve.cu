// The serving engine (gf2_server_*, declared in include/gf2.h): rank and
// solve requests on many matrices, each matrix factored once (Lemma 4.1 in
// PLE form, as gf2_decompose) and its factors kept resident for the
// requests that follow (forward and back substitution, as gf2_solve).
//
// One host thread runs the loop below; callers only queue requests and take
// completions.  Per turn of the loop:
//   1. requests whose arrival time has come join the waiting list;
//   2. finished decompositions mark their factors ready and free their
//      staging; solve launches hand back every request whose CTA has raised
//      its done flag (results are in mapped host memory), and free their
//      device memory once the whole launch is over;
//   3. admission, in arrival order: a request on resident factors is
//      admitted at once; a miss reserves its factor block and the staging of
//      A in the device arena (evicting the least recently used factors that
//      no request holds) -- when that does not fit, later misses wait too,
//      so misses are admitted in order as memory frees up;
//   4. new misses are decomposed on four decomposition lanes in turn (a
//      stream and a workspace each; the library runs each plain
//      decomposition on its own set of streams, so lanes overlap on the
//      GPU): several small misses (up to 512 x 512) together in one batched
//      launch, every other one by the plain decomposition;
//   5. every admitted request whose factors are ready joins one solve
//      launch on a free slot (four slots: up to four launches in flight),
//      one CTA per request, largest first -- while that leaves SMs idle, a
//      system of 4096 rows or more gets a cluster of eight CTAs instead, in
//      a launch beside that one.
// With GF2_SERVE_SERIAL the loop instead takes one request at a time and
// runs gf2_decompose / gf2_solve on it to the end (the baseline).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gf2.h"
#include "gf2_internal.cuh"

using namespace gf2;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAl = 256;
constexpr int kSlots = 4;
constexpr int kDecLanes = 4;
// misses up to this size go to one batched decomposition (one CTA per
// matrix) when at least kBatchedDecompMin of them are new in the same turn;
// larger ones take the plain decomposition, which uses the whole GPU
constexpr int64_t kBatchedDecompMax = 512;
constexpr size_t kBatchedDecompMin = 4;
constexpr int kMaxBatchLimit = 4096;

size_t up(size_t x) { return (x + kAl - 1) / kAl * kAl; }
int64_t wordsof(int64_t cols) { return (cols + 63) / 64; }

// First-fit allocator over one device buffer; free blocks are kept by offset
// and merged with their neighbours on release.
class Arena {
  public:
    ~Arena()
    {
        if (base_) cudaFree(base_);
    }
    int init(size_t bytes)
    {
        bytes = up(bytes);
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return GF2_ERR_NOMEM;
        }
        cap_ = bytes;
        free_[0] = bytes;
        return GF2_OK;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[*off + bytes] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = up(bytes ? bytes : 1);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    char *at(size_t off) const { return base_ + off; }
    size_t capacity() const { return cap_; }

  private:
    char *base_ = nullptr;
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

// The resident factors of one matrix key.
struct Entry {
    uint64_t key = 0;
    int64_t n = 0, m = 0, kmax = 0;
    enum State { Building, Ready, Failed } state = Building;
    int status = GF2_OK;
    int refs = 0;  // admitted requests that still need it
    uint64_t stamp = 0;
    size_t off = 0, bytes = 0;           // factor block in the arena
    size_t a_off = 0, a_bytes = 0;       // staging of A while it is built
    const uint64_t *A_host = nullptr;    // source of the build
    int64_t lda = 0;
    int64_t *rank = nullptr;
    int32_t *perm = nullptr, *piv = nullptr;
    uint64_t *L = nullptr, *E = nullptr;  // ld n and ld max(kmax, 1)
};

struct Req {
    gf2_request r;
    double arrival = 0, admit = 0;
    Entry *e = nullptr;
    int hit = 0;
};

struct DecompJob {
    cudaEvent_t ev = nullptr;
    std::vector<Entry *> entries;
    bool has_ws = false;
    size_t ws_off = 0, ws_bytes = 0;
};

// One solve launch in flight (or a free slot).
struct Slot {
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;  // the cluster launch of the large systems, beside the other one
    cudaEvent_t ev = nullptr, fork = nullptr, join = nullptr;
    char *in_host = nullptr;   // pinned: the launch's items and right-hand sides
    size_t in_cap = 0;
    char *out_host = nullptr;  // pinned and mapped: per request done, rank, consistent, X
    char *out_dev = nullptr;
    size_t out_cap = 0;
    bool busy = false;
    size_t dev_off = 0, dev_bytes = 0;
    std::vector<Req *> reqs;
    std::vector<size_t> out_off;
    std::vector<char> seen;
    int remaining = 0;
};

// per request, at the start of its output record
struct OutHeader {
    uint32_t done;
    uint32_t pad;
    int64_t rank;
    uint64_t consistent;
    uint64_t pad2;
};

size_t factor_bytes(int64_t n, int64_t m)
{
    const int64_t k = n < m ? n : m;
    return up(8) + up((size_t)n * 4) + up((size_t)(k > 0 ? k : 1) * 4) + up((size_t)wordsof(k) * n * 8) +
           up((size_t)wordsof(m) * (k > 0 ? k : 1) * 8);
}

size_t solve_scratch_bytes(int64_t n, int64_t m)
{
    const int64_t k = n < m ? n : m, mu = wordsof(m), nbl = wordsof(k);
    return up((size_t)n * 8) + up((size_t)(k > 0 ? k : 1) * 8) + up((size_t)(nbl > 0 ? nbl : 1) * 64 * 8) +
           up((size_t)mu * 64 * 8) + up((size_t)(mu + 1) * 4) + kAl;
}

uint64_t low_mask(int bits) { return bits >= 64 ? ~0ull : ((1ull << bits) - 1); }

}  // namespace

struct gf2_server {
    int device = 0;
    unsigned flags = 0;
    int64_t max_n = 0, max_m = 0;
    int max_batch = 1;
    int sms = 1;
    Clock::time_point t0;
    Arena arena;        // factors, staging of A, batched-decomposition workspaces
    Arena solve_arena;  // right-hand sides and scratch of the solve launches in flight
    // decomposition lanes: a stream and a plain-decomposition workspace each,
    // so that up to kDecLanes misses are decomposed side by side
    void *dec_ws[kDecLanes] = {};
    size_t dec_ws_bytes = 0;
    cudaStream_t dec_stream[kDecLanes] = {};
    unsigned next_lane = 0;
    Slot slots[kSlots];
    std::unordered_map<uint64_t, Entry *> cache;
    uint64_t lru_clock = 0;
    size_t resident = 0;

    std::mutex mu;
    std::condition_variable cv_in, cv_done;
    std::vector<Req *> incoming;            // guarded by mu
    std::deque<gf2_completion> done;        // guarded by mu
    gf2_server_stats stats{};               // guarded by mu
    bool stop = false;                      // guarded by mu
    int64_t outstanding = 0;                // guarded by mu: queued, not completed

    // engine thread only
    std::vector<Req *> future;              // not arrived yet (min-heap on arrival)
    std::deque<Req *> waiting;              // arrived, not admitted
    std::deque<Req *> admitted;             // admitted, not yet in a solve launch
    std::vector<Entry *> to_build;
    std::vector<DecompJob> jobs;
    int sticky = GF2_OK;                    // a CUDA error ends all further work
    std::thread engine;

    double now() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
};

namespace {

bool later(const Req *a, const Req *b) { return a->arrival > b->arrival; }

void complete(gf2_server *S, Req *q, int status, int64_t rank, uint64_t consistent)
{
    gf2_completion c{};
    c.id = q->r.id;
    c.status = status;
    c.hit = q->hit;
    c.rank = rank;
    c.consistent = consistent;
    c.arrival_us = q->arrival;
    c.admit_us = q->admit;
    c.done_us = S->now();
    if (q->e) --q->e->refs;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->done.push_back(c);
        --S->outstanding;
        ++S->stats.completed;
        if (status == GF2_OK) {
            if (q->hit) ++S->stats.hits;
            else ++S->stats.misses;
        }
        S->stats.resident_bytes = (int64_t)S->resident;
    }
    S->cv_done.notify_all();
    delete q;
}

void evict(gf2_server *S, Entry *e)
{
    S->arena.release(e->off, e->bytes);
    S->resident -= e->bytes;
    S->cache.erase(e->key);
    delete e;
    std::lock_guard<std::mutex> lock(S->mu);
    ++S->stats.evictions;
}

// Allocates from the arena, evicting unreferenced factors (least recently
// used first) until the block fits.
bool alloc_evicting(gf2_server *S, size_t bytes, size_t *off)
{
    while (!S->arena.alloc(bytes, off)) {
        Entry *victim = nullptr;
        for (auto &kv : S->cache) {
            Entry *e = kv.second;
            if (e->refs == 0 && e->state != Entry::Building && (!victim || e->stamp < victim->stamp)) victim = e;
        }
        if (!victim) return false;
        evict(S, victim);
    }
    return true;
}

void carve_factors(gf2_server *S, Entry *e)
{
    char *p = S->arena.at(e->off);
    const int64_t k = e->kmax;
    e->rank = reinterpret_cast<int64_t *>(p); p += up(8);
    e->perm = reinterpret_cast<int32_t *>(p); p += up((size_t)e->n * 4);
    e->piv = reinterpret_cast<int32_t *>(p); p += up((size_t)(k > 0 ? k : 1) * 4);
    e->L = reinterpret_cast<uint64_t *>(p); p += up((size_t)wordsof(k) * e->n * 8);
    e->E = reinterpret_cast<uint64_t *>(p);
}

// A new entry for the miss q, with its factor block and A staging; false
// when the memory is not available now.
Entry *new_entry(gf2_server *S, Req *q, bool *never)
{
    const int64_t n = q->r.n, m = q->r.m;
    const size_t fb = factor_bytes(n, m), ab = (size_t)wordsof(m) * n * 8;
    *never = up(fb) + up(ab) > S->arena.capacity();
    if (*never) return nullptr;
    size_t off = 0, aoff = 0;
    if (!alloc_evicting(S, fb, &off)) return nullptr;
    if (!alloc_evicting(S, ab, &aoff)) {
        S->arena.release(off, fb);
        return nullptr;
    }
    Entry *e = new Entry;
    e->key = q->r.matrix;
    e->n = n;
    e->m = m;
    e->kmax = n < m ? n : m;
    e->off = off;
    e->bytes = fb;
    e->a_off = aoff;
    e->a_bytes = ab;
    e->A_host = q->r.A;
    e->lda = q->r.lda;
    carve_factors(S, e);
    S->cache[e->key] = e;
    S->resident += fb;
    return e;
}

int copy_a_in(gf2_server *S, Entry *e, int lane)
{
    const int64_t mu = wordsof(e->m);
    char *dst = S->arena.at(e->a_off);
    cudaError_t ce;
    if (e->lda == e->n)
        ce = cudaMemcpyAsync(dst, e->A_host, (size_t)mu * e->n * 8, cudaMemcpyHostToDevice, S->dec_stream[lane]);
    else
        ce = cudaMemcpy2DAsync(dst, (size_t)e->n * 8, e->A_host, (size_t)e->lda * 8, (size_t)e->n * 8, (size_t)mu,
                               cudaMemcpyHostToDevice, S->dec_stream[lane]);
    return ce == cudaSuccess ? GF2_OK : GF2_ERR_CUDA;
}

int plain_decompose(gf2_server *S, Entry *e, int lane)
{
    const int64_t k = e->kmax;
    gf2_mat A{reinterpret_cast<uint64_t *>(S->arena.at(e->a_off)), e->n, e->m, e->n};
    gf2_mat L{e->L, e->n, k, e->n};
    gf2_mat E{e->E, k, e->m, k > 0 ? k : 1};
    // separate launches: the engine overlaps up to four decompositions and
    // its solve launches on the GPU, which a launch holding every SM would
    // serialise
    gf2_opts o{};
    o.schedule = GF2_SCHEDULE_STREAMS;
    return gf2_decompose_ex(&A, e->perm, e->piv, e->rank, &L, &E, GF2_NOCHECK, &o, S->dec_ws[lane], S->dec_ws_bytes,
                            S->dec_stream[lane]);
}

void fail_entry(Entry *e, int status)
{
    e->state = Entry::Failed;
    e->status = status;
}

// ---- step 2a: decompositions that have finished
bool retire_jobs(gf2_server *S)
{
    bool progress = false;
    for (size_t i = 0; i < S->jobs.size();) {
        DecompJob &j = S->jobs[i];
        const cudaError_t q = cudaEventQuery(j.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess) S->sticky = GF2_ERR_CUDA;
        for (Entry *e : j.entries) {
            if (q == cudaSuccess) e->state = Entry::Ready;
            else fail_entry(e, GF2_ERR_CUDA);
            S->arena.release(e->a_off, e->a_bytes);
            e->a_bytes = 0;
        }
        if (j.has_ws) S->arena.release(j.ws_off, j.ws_bytes);
        cudaEventDestroy(j.ev);
        S->jobs.erase(S->jobs.begin() + i);
        progress = true;
    }
    return progress;
}

// ---- step 2b: requests whose CTA is done, launches that are over
bool scan_slot(gf2_server *S, Slot &sl)
{
    bool progress = false;
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        if (sl.seen[i]) continue;
        const OutHeader *h = reinterpret_cast<const OutHeader *>(sl.out_host + sl.out_off[i]);
        if (__atomic_load_n(&h->done, __ATOMIC_ACQUIRE) == 0) continue;
        Req *q = sl.reqs[i];
        if (q->r.nrhs > 0) std::memcpy(q->r.X, sl.out_host + sl.out_off[i] + sizeof(OutHeader), (size_t)q->r.m * 8);
        complete(S, q, GF2_OK, h->rank, q->r.nrhs > 0 ? h->consistent : 0);
        sl.seen[i] = 1;
        --sl.remaining;
        progress = true;
    }
    return progress;
}

bool retire_slots(gf2_server *S)
{
    bool progress = false;
    for (Slot &sl : S->slots) {
        if (!sl.busy) continue;
        progress |= scan_slot(S, sl);
        const cudaError_t st = cudaEventQuery(sl.ev);
        if (st == cudaErrorNotReady) continue;
        if (st == cudaSuccess) scan_slot(S, sl);  // every flag is visible once the launch is over
        else S->sticky = GF2_ERR_CUDA;
        for (size_t i = 0; i < sl.reqs.size(); ++i)
            if (!sl.seen[i]) complete(S, sl.reqs[i], GF2_ERR_CUDA, 0, 0);
        S->solve_arena.release(sl.dev_off, sl.dev_bytes);
        sl.busy = false;
        sl.reqs.clear();
        progress = true;
    }
    return progress;
}

// ---- step 3: admission in arrival order
bool gpu_busy(const gf2_server *S);

bool admit(gf2_server *S)
{
    bool progress = false, miss_blocked = false;
    const double now = S->now();
    // (continuous batching: a request may be admitted while earlier work of
    // the engine is still on the GPU)
    const bool in_flight = gpu_busy(S);
    auto count_admission = [&]() {
        if (!in_flight) return;
        std::lock_guard<std::mutex> lock(S->mu);
        ++S->stats.admitted_in_flight;
    };
    for (auto it = S->waiting.begin(); it != S->waiting.end();) {
        Req *q = *it;
        auto f = S->cache.find(q->r.matrix);
        if (f != S->cache.end()) {
            Entry *e = f->second;
            if (e->n != q->r.n || e->m != q->r.m) {
                it = S->waiting.erase(it);
                complete(S, q, GF2_ERR_SHAPE, 0, 0);
                progress = true;
                continue;
            }
            if (e->state == Entry::Failed) {
                it = S->waiting.erase(it);
                complete(S, q, e->status, 0, 0);
                progress = true;
                continue;
            }
            ++e->refs;
            e->stamp = ++S->lru_clock;
            q->e = e;
            q->hit = 1;
            q->admit = now;
            S->admitted.push_back(q);
            count_admission();
            it = S->waiting.erase(it);
            progress = true;
            continue;
        }
        if (miss_blocked) {
            ++it;
            continue;
        }
        bool never = false;
        Entry *e = new_entry(S, q, &never);
        if (!e) {
            if (never) {
                it = S->waiting.erase(it);
                complete(S, q, GF2_ERR_NOMEM, 0, 0);
                progress = true;
                continue;
            }
            miss_blocked = true;  // later misses wait behind this one
            ++it;
            continue;
        }
        e->refs = 1;
        e->stamp = ++S->lru_clock;
        q->e = e;
        q->hit = 0;
        q->admit = now;
        S->admitted.push_back(q);
        count_admission();
        S->to_build.push_back(e);
        it = S->waiting.erase(it);
        progress = true;
    }
    return progress;
}

// ---- step 4: decompositions of the new misses
// Records the end of a decomposition job on its lane and queues the job.
void queue_job(gf2_server *S, DecompJob &&job, int lane)
{
    if (cudaEventCreateWithFlags(&job.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(job.ev, S->dec_stream[lane]) != cudaSuccess) {
        cudaGetLastError();
        S->sticky = GF2_ERR_CUDA;
        cudaStreamSynchronize(S->dec_stream[lane]);
        if (!job.ev) cudaEventCreateWithFlags(&job.ev, cudaEventDisableTiming);
    }
    S->jobs.push_back(std::move(job));
}

bool launch_builds(gf2_server *S)
{
    if (S->to_build.empty()) return false;
    std::vector<Entry *> small, large;
    for (Entry *e : S->to_build) (e->n <= kBatchedDecompMax && e->m <= kBatchedDecompMax ? small : large).push_back(e);
    S->to_build.clear();
    if (small.size() >= kBatchedDecompMin) {
        // one batched launch for the small misses of this turn
        std::vector<BatchItem> items(small.size());
        for (size_t i = 0; i < small.size(); ++i) {
            Entry *e = small[i];
            items[i] = BatchItem{reinterpret_cast<const uint64_t *>(S->arena.at(e->a_off)), e->n, (int32_t)e->n,
                                 (int32_t)e->m, e->perm, e->piv, e->rank, e->L, e->n, e->E,
                                 e->kmax > 0 ? e->kmax : 1};
        }
        const size_t wb = decompose_batched_items_bytes((int)items.size(), items.data(), true);
        size_t off = 0;
        if (wb && alloc_evicting(S, wb, &off)) {
            const int lane = (int)(S->next_lane++ % kDecLanes);
            int st = GF2_OK;
            for (Entry *e : small)
                if (st == GF2_OK) st = copy_a_in(S, e, lane);
            if (st == GF2_OK)
                st = decompose_batched_items((int)items.size(), items.data(), true, GF2_NOCHECK, S->arena.at(off), wb,
                                             S->dec_stream[lane]);
            DecompJob job;
            job.has_ws = true;
            job.ws_off = off;
            job.ws_bytes = wb;
            for (Entry *e : small) {
                if (st != GF2_OK) fail_entry(e, st);
                job.entries.push_back(e);
            }
            queue_job(S, std::move(job), lane);
            std::lock_guard<std::mutex> lock(S->mu);
            ++S->stats.batched_decompositions;
            small.clear();
        }
        // no room for the batched workspace: the plain path below, one by one
    }
    for (Entry *e : small) large.push_back(e);
    // the larger misses, one plain decomposition each, lanes in turn
    for (Entry *e : large) {
        const int lane = (int)(S->next_lane++ % kDecLanes);
        int st = copy_a_in(S, e, lane);
        if (st == GF2_OK) st = plain_decompose(S, e, lane);
        if (st != GF2_OK) fail_entry(e, st);
        DecompJob job;
        job.entries.push_back(e);
        queue_job(S, std::move(job), lane);
        std::lock_guard<std::mutex> lock(S->mu);
        ++S->stats.plain_decompositions;
    }
    return true;
}

bool grow_pinned(char **p, size_t *cap, size_t need, bool mapped)
{
    if (*cap >= need) return true;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    size_t c = 1 << 20;
    while (c < need) c *= 2;
    if (cudaHostAlloc(reinterpret_cast<void **>(p), c, mapped ? cudaHostAllocMapped : cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    *cap = c;
    return true;
}

// ---- step 5: one solve launch with every ready request (up to max_batch)
bool launch_solves(gf2_server *S)
{
    Slot *sl = nullptr;
    for (Slot &s : S->slots)
        if (!s.busy) {
            sl = &s;
            break;
        }
    if (!sl || S->admitted.empty()) return false;
    std::vector<Req *> take;
    bool progress = false;
    for (auto it = S->admitted.begin(); it != S->admitted.end() && (int)take.size() < S->max_batch;) {
        Req *q = *it;
        if (q->e->state == Entry::Failed) {
            it = S->admitted.erase(it);
            complete(S, q, q->e->status, 0, 0);
            progress = true;
            continue;
        }
        if (q->e->state == Entry::Ready) {
            take.push_back(q);
            it = S->admitted.erase(it);
            continue;
        }
        ++it;
    }
    if (take.empty()) return progress;
    // largest first, so that the CTAs finish together
    std::stable_sort(take.begin(), take.end(), [](const Req *a, const Req *b) {
        return (double)a->r.n * wordsof(a->r.m) > (double)b->r.n * wordsof(b->r.m);
    });
    for (;;) {
        const size_t cnt = take.size();
        size_t in_bytes = kAl + up(cnt * sizeof(ServeItem)), scratch = 0, out_bytes = 0;
        for (Req *q : take) {
            in_bytes += up((size_t)q->r.n * 8);
            scratch += solve_scratch_bytes(q->r.n, q->r.m);
            out_bytes += up(sizeof(OutHeader) + (size_t)q->r.m * 8);
        }
        size_t off = 0;
        if (S->solve_arena.alloc(in_bytes + scratch, &off)) {
            if (!grow_pinned(&sl->in_host, &sl->in_cap, in_bytes, false) ||
                !grow_pinned(&sl->out_host, &sl->out_cap, out_bytes, true) ||
                cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl->out_dev), sl->out_host, 0) != cudaSuccess) {
                S->solve_arena.release(off, in_bytes + scratch);
                S->sticky = GF2_ERR_NOMEM;
                for (Req *q : take) complete(S, q, GF2_ERR_NOMEM, 0, 0);
                return true;
            }
            char *dev = S->solve_arena.at(off);
            char *hin = sl->in_host;
            std::memset(hin, 0, kAl);  // the CTAs' shared counter
            ServeItem *items = reinterpret_cast<ServeItem *>(hin + kAl);
            size_t bpos = kAl + up(cnt * sizeof(ServeItem)), spos = in_bytes, opos = 0;
            sl->out_off.assign(cnt, 0);
            for (size_t i = 0; i < cnt; ++i) {
                Req *q = take[i];
                Entry *e = q->e;
                const int64_t n = q->r.n, m = q->r.m, k = e->kmax, mu = wordsof(m), nbl = wordsof(k);
                ServeItem it{};
                SolveCtx &c = it.c;
                c.perm = e->perm;
                c.pivcols = e->piv;
                c.rank = e->rank;
                c.L = e->L;
                c.ldl = n;
                c.E = e->E;
                c.lde = k > 0 ? k : 1;
                if (q->r.nrhs > 0) std::memcpy(hin + bpos, q->r.B, (size_t)n * 8);
                else std::memset(hin + bpos, 0, (size_t)n * 8);
                c.B = reinterpret_cast<const uint64_t *>(dev + bpos);
                bpos += up((size_t)n * 8);
                char *sc = dev + spos;
                c.v = reinterpret_cast<uint64_t *>(sc); sc += up((size_t)n * 8);
                c.y = reinterpret_cast<uint64_t *>(sc); sc += up((size_t)(k > 0 ? k : 1) * 8);
                c.linv = reinterpret_cast<uint64_t *>(sc); sc += up((size_t)(nbl > 0 ? nbl : 1) * 64 * 8);
                c.uinv = reinterpret_cast<uint64_t *>(sc); sc += up((size_t)mu * 64 * 8);
                c.qstart = reinterpret_cast<int32_t *>(sc); sc += up((size_t)(mu + 1) * 4);
                c.sync = reinterpret_cast<uint32_t *>(sc);
                c.bad = reinterpret_cast<uint64_t *>(sc + 64);
                spos += solve_scratch_bytes(n, m);
                OutHeader *h = reinterpret_cast<OutHeader *>(sl->out_host + opos);
                std::memset(h, 0, sizeof(OutHeader));
                char *od = sl->out_dev + opos;
                c.X = reinterpret_cast<uint64_t *>(od + sizeof(OutHeader));
                c.consistent = reinterpret_cast<uint64_t *>(od + offsetof(OutHeader, consistent));
                c.rhs_mask = low_mask(q->r.nrhs > 0 ? q->r.nrhs : 1);
                c.n = (int32_t)n;
                c.m = (int32_t)m;
                c.check = 0;  // the right-hand sides were checked on submission
                it.rank_out = reinterpret_cast<int64_t *>(od + offsetof(OutHeader, rank));
                it.done = reinterpret_cast<uint32_t *>(od + offsetof(OutHeader, done));
                it.nrhs = q->r.nrhs;
                items[i] = it;
                sl->out_off[i] = opos;
                opos += up(sizeof(OutHeader) + (size_t)m * 8);
            }
            // (the host wrote the done words before the launch is enqueued)
            std::atomic_thread_fence(std::memory_order_seq_cst);
            // the large systems (first: the items are sorted by size) take one
            // cluster each on the second stream, the others one CTA each
            // -- while the SMs would otherwise idle: with a cluster per large
            // system the launch must still fit in one wave (a full launch is
            // served best by one CTA per system, all SMs busy)
            size_t nl = 0;
            while (nl < cnt && serve_by_cluster(take[nl]->r.n)) ++nl;
            if ((int64_t)cnt + (int64_t)nl * (kServeClusterCTAs - 1) > S->sms) nl = 0;
            const ServeItem *dev_items = reinterpret_cast<const ServeItem *>(dev + kAl);
            cudaError_t ce = cudaMemcpyAsync(dev, hin, in_bytes, cudaMemcpyHostToDevice, sl->stream);
            int launches = 0;
            if (ce == cudaSuccess && nl > 0) {
                ce = cudaEventRecord(sl->fork, sl->stream);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(sl->stream2, sl->fork, 0);
                if (ce == cudaSuccess) ce = launch_serve_cluster(dev_items, (int)nl, take[0]->r.n, sl->stream2);
                if (ce == cudaSuccess) ce = cudaEventRecord(sl->join, sl->stream2);
                ++launches;
            }
            if (ce == cudaSuccess && nl < cnt) {
                ce = launch_serve_solve(dev_items + nl, (int)(cnt - nl), reinterpret_cast<int32_t *>(dev),
                                        take[nl]->r.n, sl->stream);
                ++launches;
            }
            if (ce == cudaSuccess && nl > 0) ce = cudaStreamWaitEvent(sl->stream, sl->join, 0);
            if (ce == cudaSuccess) ce = cudaEventRecord(sl->ev, sl->stream);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                cudaStreamSynchronize(sl->stream);
                cudaStreamSynchronize(sl->stream2);
                S->solve_arena.release(off, in_bytes + scratch);
                S->sticky = GF2_ERR_CUDA;
                for (Req *q : take) complete(S, q, GF2_ERR_CUDA, 0, 0);
                return true;
            }
            add_launches(launches);
            const bool overlapped = gpu_busy(S);  // (before this slot counts as busy)
            sl->busy = true;
            sl->dev_off = off;
            sl->dev_bytes = in_bytes + scratch;
            sl->reqs = take;
            sl->seen.assign(cnt, 0);
            sl->remaining = (int)cnt;
            std::lock_guard<std::mutex> lock(S->mu);
            ++S->stats.solve_launches;
            if (overlapped) ++S->stats.overlapped_launches;
            if ((int64_t)cnt > S->stats.max_batch) S->stats.max_batch = (int64_t)cnt;
            return true;
        }
        if (take.size() == 1) break;
        // no room for all of them now: the smaller half goes back to the front
        const size_t keep = take.size() / 2;
        for (size_t i = take.size(); i-- > keep;) S->admitted.push_front(take[i]);
        take.resize(keep);
    }
    S->admitted.push_front(take[0]);  // waits for a launch in flight to end
    return progress;
}

// ---- the one-at-a-time baseline: gf2_decompose and gf2_solve, each waited for
bool serial_step(gf2_server *S)
{
    if (S->waiting.empty()) return false;
    Req *q = S->waiting.front();
    S->waiting.pop_front();
    q->admit = S->now();
    const int64_t n = q->r.n, m = q->r.m;
    auto f = S->cache.find(q->r.matrix);
    Entry *e = f == S->cache.end() ? nullptr : f->second;
    if (e && (e->n != n || e->m != m)) {
        complete(S, q, GF2_ERR_SHAPE, 0, 0);
        return true;
    }
    if (!e) {
        bool never = false;
        e = new_entry(S, q, &never);
        if (!e) {
            complete(S, q, GF2_ERR_NOMEM, 0, 0);
            return true;
        }
        int st = copy_a_in(S, e, 0);
        if (st == GF2_OK) st = plain_decompose(S, e, 0);
        if (st == GF2_OK && cudaStreamSynchronize(S->dec_stream[0]) != cudaSuccess) st = GF2_ERR_CUDA;
        S->arena.release(e->a_off, e->a_bytes);
        e->a_bytes = 0;
        if (st != GF2_OK) {
            fail_entry(e, st);
            S->sticky = st == GF2_ERR_CUDA ? st : S->sticky;
        } else {
            e->state = Entry::Ready;
        }
        std::lock_guard<std::mutex> lock(S->mu);
        ++S->stats.plain_decompositions;
        q->hit = 0;
    } else {
        q->hit = 1;
    }
    q->e = e;
    ++e->refs;
    e->stamp = ++S->lru_clock;
    if (e->state == Entry::Failed) {
        complete(S, q, e->status, 0, 0);
        return true;
    }
    int64_t rank = 0;
    uint64_t cons = 0;
    int st = GF2_OK;
    if (q->r.nrhs > 0) {
        const int64_t k = e->kmax;
        const size_t wb = gf2_solve_workspace_bytes(n, m);
        const size_t need = up(wb) + up((size_t)n * 8) + up((size_t)m * 8) + kAl;
        size_t off = 0;
        if (!alloc_evicting(S, need, &off)) {
            complete(S, q, GF2_ERR_NOMEM, 0, 0);
            return true;
        }
        char *p = S->arena.at(off);
        uint64_t *Bd = reinterpret_cast<uint64_t *>(p + up(wb));
        uint64_t *Xd = reinterpret_cast<uint64_t *>(p + up(wb) + up((size_t)n * 8));
        uint64_t *cd = reinterpret_cast<uint64_t *>(p + up(wb) + up((size_t)n * 8) + up((size_t)m * 8));
        gf2_mat L{e->L, n, k, n}, E{e->E, k, m, k > 0 ? k : 1}, B{Bd, n, q->r.nrhs, n}, X{Xd, m, q->r.nrhs, m};
        cudaStream_t ds = S->dec_stream[0];
        if (cudaMemcpyAsync(Bd, q->r.B, (size_t)n * 8, cudaMemcpyHostToDevice, ds) != cudaSuccess)
            st = GF2_ERR_CUDA;
        if (st == GF2_OK)
            st = gf2_solve(&L, &E, e->perm, e->piv, e->rank, &B, &X, cd, GF2_NOCHECK, p, wb, ds);
        if (st == GF2_OK &&
            (cudaMemcpyAsync(q->r.X, Xd, (size_t)m * 8, cudaMemcpyDeviceToHost, ds) != cudaSuccess ||
             cudaMemcpyAsync(&cons, cd, 8, cudaMemcpyDeviceToHost, ds) != cudaSuccess))
            st = GF2_ERR_CUDA;
        if (st == GF2_OK &&
            (cudaMemcpyAsync(&rank, e->rank, 8, cudaMemcpyDeviceToHost, ds) != cudaSuccess ||
             cudaStreamSynchronize(ds) != cudaSuccess))
            st = GF2_ERR_CUDA;
        S->arena.release(off, need);
    } else if (cudaMemcpyAsync(&rank, e->rank, 8, cudaMemcpyDeviceToHost, S->dec_stream[0]) != cudaSuccess ||
               cudaStreamSynchronize(S->dec_stream[0]) != cudaSuccess) {
        st = GF2_ERR_CUDA;
    }
    if (st == GF2_ERR_CUDA) S->sticky = st;
    complete(S, q, st, rank, cons);
    return true;
}

bool gpu_busy(const gf2_server *S)
{
    if (!S->jobs.empty()) return true;
    for (const Slot &s : S->slots)
        if (s.busy) return true;
    return false;
}

void fail_all_waiting(gf2_server *S)
{
    for (Req *q : S->waiting) complete(S, q, S->sticky, 0, 0);
    S->waiting.clear();
    for (Req *q : S->admitted) complete(S, q, S->sticky, 0, 0);
    S->admitted.clear();
}

void engine_main(gf2_server *S)
{
    cudaSetDevice(S->device);
    const bool serial = (S->flags & GF2_SERVE_SERIAL) != 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(S->mu);
            for (Req *q : S->incoming) {
                S->future.push_back(q);
                std::push_heap(S->future.begin(), S->future.end(), later);
            }
            S->incoming.clear();
            if (S->stop && S->outstanding == 0) break;
        }
        bool progress = false;
        const double now = S->now();
        while (!S->future.empty() && S->future.front()->arrival <= now) {
            std::pop_heap(S->future.begin(), S->future.end(), later);
            S->waiting.push_back(S->future.back());
            S->future.pop_back();
            progress = true;
        }
        if (serial) {
            progress |= serial_step(S);
        } else {
            progress |= retire_jobs(S);
            progress |= retire_slots(S);
            if (S->sticky != GF2_OK) {
                if (!gpu_busy(S)) fail_all_waiting(S);
            } else {
                progress |= admit(S);
                progress |= launch_builds(S);
                progress |= launch_solves(S);
            }
        }
        if (progress) continue;
        if (gpu_busy(S)) {
            std::this_thread::yield();
            continue;
        }
        // idle: sleep until a submission or shortly before the next arrival
        std::unique_lock<std::mutex> lock(S->mu);
        if (!S->incoming.empty() || (S->stop && S->outstanding == 0)) continue;
        double wait_us = 2000;
        if (!S->future.empty()) wait_us = std::min(wait_us, S->future.front()->arrival - S->now() - 50.0);
        if (!S->waiting.empty()) wait_us = std::min(wait_us, 20.0);  // blocked on memory
        if (wait_us <= 0) {
            lock.unlock();
            std::this_thread::yield();
            continue;
        }
        S->cv_in.wait_for(lock, std::chrono::microseconds((int64_t)wait_us));
    }
    // every request is complete; wait for the GPU before the memory goes
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.stream2) cudaStreamSynchronize(s.stream2);
    }
    for (cudaStream_t d : S->dec_stream)
        if (d) cudaStreamSynchronize(d);
}

// host-side checks of one request; GF2_OK or its error
int check_request(const gf2_server *S, const gf2_request &r)
{
    if (r.n < 1 || r.m < 1 || r.nrhs < 0 || r.nrhs > 64) return r.nrhs > 64 ? GF2_ERR_SHAPE : GF2_ERR_ARG;
    if (r.n > S->max_n || r.m > S->max_m) return GF2_ERR_UNSUPPORTED;
    if (!r.A || r.lda < r.n) return r.A ? GF2_ERR_SHAPE : GF2_ERR_ARG;
    if (r.nrhs > 0 && (!r.B || !r.X)) return GF2_ERR_ARG;
    if (r.m % 64) {
        const uint64_t keep = low_mask((int)(r.m % 64));
        const uint64_t *last = r.A + (wordsof(r.m) - 1) * r.lda;
        uint64_t bad = 0;
        for (int64_t i = 0; i < r.n; ++i) bad |= last[i] & ~keep;
        if (bad) return GF2_ERR_PADDING;
    }
    if (r.nrhs > 0 && r.nrhs < 64) {
        const uint64_t keep = low_mask(r.nrhs);
        uint64_t bad = 0;
        for (int64_t i = 0; i < r.n; ++i) bad |= r.B[i] & ~keep;
        if (bad) return GF2_ERR_PADDING;
    }
    return GF2_OK;
}

void destroy_resources(gf2_server *S)
{
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.stream2) cudaStreamDestroy(s.stream2);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.fork) cudaEventDestroy(s.fork);
        if (s.join) cudaEventDestroy(s.join);
        if (s.in_host) cudaFreeHost(s.in_host);
        if (s.out_host) cudaFreeHost(s.out_host);
    }
    for (int l = 0; l < kDecLanes; ++l) {
        if (S->dec_stream[l]) cudaStreamDestroy(S->dec_stream[l]);
        if (S->dec_ws[l]) cudaFree(S->dec_ws[l]);
    }
    for (auto &kv : S->cache) delete kv.second;
    S->cache.clear();
}

}  // namespace

extern "C" {

int gf2_server_create(int64_t device_bytes, int64_t max_n, int64_t max_m, int max_batch, unsigned flags,
                      gf2_server **out)
{
    if (!out || device_bytes <= 0 || max_n < 1 || max_m < 1 || max_n >= (1ll << 31) - 64 ||
        max_m >= (1ll << 31) - 64 || max_batch < 1 || max_batch > kMaxBatchLimit || (flags & ~GF2_SERVE_SERIAL))
        return GF2_ERR_ARG;
    *out = nullptr;
    gf2_server *S = new (std::nothrow) gf2_server;
    if (!S) return GF2_ERR_NOMEM;
    S->flags = flags;
    S->max_n = max_n;
    S->max_m = max_m;
    S->max_batch = max_batch;
    S->t0 = Clock::now();
    int st = GF2_OK;
    int sms = 1, lo = 0, hi = 0;
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess)
        st = GF2_ERR_CUDA;
    S->sms = sms;
    // the solve launches get their own arena, so that resident factors can
    // never crowd out the solves that release them
    const size_t one = solve_scratch_bytes(max_n, max_m) + up((size_t)max_n * 8) + 2 * kAl + up(sizeof(ServeItem));
    size_t solve_bytes = std::max<size_t>((size_t)device_bytes / 8, 8 * one);
    solve_bytes = std::max<size_t>(std::min<size_t>(solve_bytes, (size_t)1 << 30), 2 * one);
    if ((size_t)device_bytes <= solve_bytes) st = GF2_ERR_ARG;
    if (st == GF2_OK) st = S->solve_arena.init(solve_bytes);
    if (st == GF2_OK) st = S->arena.init((size_t)device_bytes - solve_bytes);
    if (st == GF2_OK) {
        S->dec_ws_bytes = gf2_decompose_workspace_bytes(max_n, max_m, 1);
        const int lanes = (flags & GF2_SERVE_SERIAL) ? 1 : kDecLanes;
        for (int l = 0; l < lanes && st == GF2_OK; ++l) {
            if (cudaMalloc(&S->dec_ws[l], S->dec_ws_bytes) != cudaSuccess) {
                cudaGetLastError();
                S->dec_ws[l] = nullptr;
                st = GF2_ERR_NOMEM;
            } else if (cudaStreamCreateWithFlags(&S->dec_stream[l], cudaStreamNonBlocking) != cudaSuccess) {
                st = GF2_ERR_CUDA;
            }
        }
    }
    for (Slot &s : S->slots) {
        if (st != GF2_OK) break;
        if (cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s.stream2, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming) != cudaSuccess)
            st = GF2_ERR_CUDA;
    }
    if (st != GF2_OK) {
        destroy_resources(S);
        delete S;
        return st;
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stats.arena_bytes = (int64_t)S->arena.capacity();
    }
    try {
        S->engine = std::thread(engine_main, S);
    } catch (...) {
        destroy_resources(S);
        delete S;
        return GF2_ERR_NOMEM;
    }
    *out = S;
    return GF2_OK;
}

int gf2_server_submit(gf2_server *S, const gf2_request *requests, int count)
{
    if (!S || count < 0 || (count > 0 && !requests)) return GF2_ERR_ARG;
    const double now = S->now();
    std::vector<Req *> ok;
    std::vector<gf2_completion> bad;
    ok.reserve(count);
    for (int i = 0; i < count; ++i) {
        const gf2_request &r = requests[i];
        const int st = check_request(S, r);
        const double arrival = r.arrival_us > now ? r.arrival_us : now;
        if (st != GF2_OK) {
            gf2_completion c{};
            c.id = r.id;
            c.status = st;
            c.arrival_us = arrival;
            c.admit_us = now;
            c.done_us = now;
            bad.push_back(c);
            continue;
        }
        Req *q = new (std::nothrow) Req;
        if (!q) {
            for (Req *p : ok) delete p;
            return GF2_ERR_NOMEM;
        }
        q->r = r;
        q->arrival = arrival;
        ok.push_back(q);
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            for (Req *p : ok) delete p;
            return GF2_ERR_ARG;
        }
        for (Req *q : ok) S->incoming.push_back(q);
        S->outstanding += (int64_t)ok.size();
        for (auto &c : bad) S->done.push_back(c);
        S->stats.completed += (int64_t)bad.size();
    }
    S->cv_in.notify_one();
    if (!bad.empty()) S->cv_done.notify_all();
    return GF2_OK;
}

int gf2_server_poll(gf2_server *S, gf2_completion *out, int max, int64_t wait_us, int *count)
{
    if (!S || !count || max < 0 || (max > 0 && !out)) return GF2_ERR_ARG;
    *count = 0;
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->done.empty() && wait_us > 0)
        S->cv_done.wait_for(lock, std::chrono::microseconds(wait_us), [&] { return !S->done.empty(); });
    int k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    *count = k;
    return GF2_OK;
}

double gf2_server_clock_us(const gf2_server *S) { return S ? S->now() : 0.0; }

int gf2_server_stats_read(const gf2_server *S, gf2_server_stats *stats)
{
    if (!S || !stats) return GF2_ERR_ARG;
    std::lock_guard<std::mutex> lock(const_cast<gf2_server *>(S)->mu);
    *stats = S->stats;
    return GF2_OK;
}

int gf2_server_destroy(gf2_server *S)
{
    if (!S) return GF2_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_in.notify_one();
    if (S->engine.joinable()) S->engine.join();
    destroy_resources(S);
    delete S;
    return GF2_OK;
}

}  // extern "C"
