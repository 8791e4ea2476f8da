// Panel kernel: selection of the pivot rows of one 64-column block and the
// pseudo-inverse that expresses every other row of the block through them.
//
// What it computes (Sections 4.1-4.4 of the paper, Procedure buildZ): for
// bit k = 0..63 of column block j, the first row at or after the current
// pivot slot (in the current row order) whose entry k, reduced by the pivots
// already chosen in this block, is one -- the non-singularity condition
// (eq. cond:nonsing:Bk) -- is exchanged with the pivot slot.  A bit with no
// such row gets no pivot (the paper inserts the virtual row (0,1,0) there,
// Section 4.4); no column is ever exchanged.
//
// How (GB300 design, not the paper's CPU loop): warp 0 keeps a window of up
// to 32 rows (one per lane, lane = position mod 32) already REDUCED by the
// pivots found so far, so the test for bit k is one ballot over the window
// and the first qualifying row is a find-first-set on the ballot rotated to
// the pivot slot.  A new pivot row E_s (reduced) is broadcast with shuffles
// and eliminated from the window rows.  64 "probe" rows e_0..e_63 (two per
// lane) go through the same eliminations; at the end they give the linear
// maps Zp (B-coordinates, the paper's Z of eq. pre:W) and Comp
// (E-coordinates) for every other row of the block, and during the loop they
// reduce rows entering the window and give the test mask for rows outside
// it.  Rows outside the window are only scanned when the window has no
// qualifying row; those scans use all 8 warps of the CTA.
#include <climits>

#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
enum { kReqDone = 0, kReqFind = 1, kReqOr = 2 };

__device__ __forceinline__ void bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src)
{
    return __shfl_sync(kFull, v, src);
}

__device__ __forceinline__ uint64_t warp_xor(uint64_t v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v ^= __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ uint64_t warp_or(uint64_t v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v |= __shfl_xor_sync(kFull, v, off);
    return v;
}

struct PanelShared {
    uint64_t pred[64], ptinv[64], plcoef[64];  // probe rows (published for the scans)
    uint64_t tab[kNumTables * 256];            // tables of pred for full reductions
    uint64_t E[64], TI[64], T[64];
    int32_t pb[64];
    uint64_t mask;
    unsigned long long orv;
    int req, from, found;
};

// Positions [from, n): first one whose panel word w has parity(w & mask) = 1.
__device__ void scan_find(const DecompCtx &c, const uint64_t *Wj, PanelShared &sh)
{
    constexpr int U = 4;
    const int tid = threadIdx.x;
    const int from = sh.from, n = c.n;
    const uint64_t mask = sh.mask;
    for (int base = from; base < n; base += kPanelThreads * U) {
        int srow[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * kPanelThreads + tid;
            srow[u] = q < n ? c.perm[q] : -1;
        }
        uint64_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = srow[u] >= 0 ? Wj[(int64_t)srow[u] * c.ldw] : 0;
        int hit = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!hit && (__popcll(v[u] & mask) & 1)) {
                atomicMin(&sh.found, base + u * kPanelThreads + tid);
                hit = 1;
            }
        }
        if (__syncthreads_or(hit)) break;
    }
}

// OR over positions [from, n) of the fully reduced panel words (reduction by
// the current pivots through the probe rows: red(w) = XOR_{p in w} pred[p]).
__device__ void scan_or(const DecompCtx &c, const uint64_t *Wj, PanelShared &sh)
{
    constexpr int U = 4;
    const int tid = threadIdx.x;
    for (int e = tid; e < kNumTables * 256; e += kPanelThreads) {
        const int g = e >> 8, x = e & 255;
        uint64_t acc = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if ((x >> b) & 1) acc ^= sh.pred[8 * g + b];
        sh.tab[e] = acc;
    }
    __syncthreads();
    const int from = sh.from, n = c.n;
    uint64_t acc = 0;
    for (int base = from; base < n; base += kPanelThreads * U) {
        int srow[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * kPanelThreads + tid;
            srow[u] = q < n ? c.perm[q] : -1;
        }
        uint64_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = srow[u] >= 0 ? Wj[(int64_t)srow[u] * c.ldw] : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint64_t r = 0;
#pragma unroll
            for (int g = 0; g < kNumTables; ++g) r ^= sh.tab[g * 256 + ((v[u] >> (8 * g)) & 255)];
            acc |= r;
        }
    }
    acc = warp_or(acc);
    if ((tid & 31) == 0 && acc) atomicOr(&sh.orv, (unsigned long long)acc);
}

__global__ void __launch_bounds__(kPanelThreads, 1) k_panel(DecompCtx c, int j)
{
    __shared__ PanelShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = j == 0 ? 0 : c.info[j - 1].R + c.info[j - 1].r;
    const int n = c.n;
    const int nbits = min(64, c.m - 64 * j);
    PanelInfo *pi = c.info + j;
    const uint64_t *Wj = c.W + j;

    if (R >= n || nbits <= 0) {
        if (tid == 0) {
            pi->R = R;
            pi->r = 0;
        }
        return;
    }

    if (warp != 0) {  // helpers: serve scan requests of warp 0
        for (;;) {
            bar_sync(1, kPanelThreads);
            const int req = sh.req;
            if (req == kReqDone) return;
            if (req == kReqFind) scan_find(c, Wj, sh);
            else scan_or(c, Wj, sh);
            bar_sync(2, kPanelThreads);
        }
    }

    // ---------------------------------------------------------------- warp 0
    bool wv = false;        // window slot holds a row
    int wsrow = 0;          // its storage row
    uint64_t wred = 0;      // its panel word reduced by the pivots so far
    uint64_t wtinv = 0;     // B-coordinates of what was added to it
    uint64_t wlc = 0;       // E-coordinates of what was added to it
    uint64_t pr0 = 1ull << lane, pr1 = 1ull << (lane + 32);  // probes e_lane, e_{lane+32}
    uint64_t pt0 = 0, pt1 = 0, pl0 = 0, pl1 = 0;
    int ib = R;    // current pivot slot (head of the window)
    int fill = R;  // first position not loaded into the window
    int s = 0;     // pivots found

    auto publish = [&]() {
        sh.pred[lane] = pr0;
        sh.pred[lane + 32] = pr1;
        sh.ptinv[lane] = pt0;
        sh.ptinv[lane + 32] = pt1;
        sh.plcoef[lane] = pl0;
        sh.plcoef[lane + 32] = pl1;
        __syncwarp();
    };
    auto refill = [&]() {
        const int end = min(ib + 32, n);
        if (fill >= end) return;
        publish();
        const int pos = fill + ((lane - fill) & 31);
        if (pos < end) {
            const int srow = c.perm[pos];
            const uint64_t v = Wj[(int64_t)srow * c.ldw];
            uint64_t rd = 0, ti = 0, lc = 0;
            for (uint64_t x = v; x; x &= x - 1) {
                const int p = __ffsll((long long)x) - 1;
                rd ^= sh.pred[p];
                ti ^= sh.ptinv[p];
                lc ^= sh.plcoef[p];
            }
            wv = true;
            wsrow = srow;
            wred = rd;
            wtinv = ti;
            wlc = lc;
        }
        fill = end;
        __syncwarp();
    };
    auto request = [&](int req, int from, uint64_t mask, unsigned long long orv) {
        if (lane == 0) {
            sh.req = req;
            sh.from = from;
            sh.mask = mask;
            sh.found = INT_MAX;
            sh.orv = orv;
        }
        __syncwarp();
        bar_sync(1, kPanelThreads);
        if (req == kReqFind) scan_find(c, Wj, sh);
        else scan_or(c, Wj, sh);
        bar_sync(2, kPanelThreads);
    };

    refill();
    int k = 0;
    while (k < nbits && ib < n) {
        unsigned hit = __ballot_sync(kFull, wv && ((wred >> k) & 1));
        if (!hit && fill < n && fill < ib + 32) {
            refill();
            hit = __ballot_sync(kFull, wv && ((wred >> k) & 1));
        }
        const int h = ib & 31;
        int pivpos, psrow, hsrow = 0;
        uint64_t Es, TIs, Ts;
        if (hit) {
            const unsigned rot = h ? ((hit >> h) | (hit << (32 - h))) : hit;
            const int f = __ffs((int)rot) - 1;
            const int lf = (h + f) & 31;
            pivpos = ib + f;
            Es = shfl64(wred, lf);
            const uint64_t ti = shfl64(wtinv, lf), lc = shfl64(wlc, lf);
            psrow = __shfl_sync(kFull, wsrow, lf);
            const uint64_t hred = shfl64(wred, h), hti = shfl64(wtinv, h), hlc = shfl64(wlc, h);
            hsrow = __shfl_sync(kFull, wsrow, h);
            TIs = ti ^ (1ull << s);
            Ts = lc ^ (1ull << s);
            if (lane == lf && lf != h) {  // the row in the pivot slot moves to the pivot's place
                wred = hred;
                wtinv = hti;
                wlc = hlc;
                wsrow = hsrow;
            }
            if (lane == h) wv = false;
        } else if (fill < n) {
            // The window (full) has no candidate: scan the rows behind it.
            const unsigned lo = __ballot_sync(kFull, (pr0 >> k) & 1);
            const unsigned hi = __ballot_sync(kFull, (pr1 >> k) & 1);
            const uint64_t ck = (uint64_t)lo | ((uint64_t)hi << 32);
            request(kReqFind, fill, ck, 0);
            const int q = sh.found;
            if (q == INT_MAX) {
                // Bit k has no pivot.  The next bit that can have one is the
                // lowest bit above k set in some reduced remaining row.
                publish();
                const uint64_t worv = warp_or(wv ? wred : 0);
                request(kReqOr, fill, 0, worv);
                const uint64_t above = k + 1 < 64 ? (sh.orv & (~0ull << (k + 1))) : 0;
                k = above ? __ffsll((long long)above) - 1 : 64;
                continue;
            }
            pivpos = q;
            psrow = c.perm[q];
            const uint64_t v = Wj[(int64_t)psrow * c.ldw];
            uint64_t a = 0, b = 0, cc = 0;
            if ((v >> lane) & 1) { a ^= pr0; b ^= pt0; cc ^= pl0; }
            if ((v >> (lane + 32)) & 1) { a ^= pr1; b ^= pt1; cc ^= pl1; }
            Es = warp_xor(a);
            TIs = warp_xor(b) ^ (1ull << s);
            Ts = warp_xor(cc) ^ (1ull << s);
            hsrow = __shfl_sync(kFull, wsrow, h);
            if (lane == h) wv = false;  // the row in the pivot slot moves behind the window
        } else {
            // Every remaining row is in the window and none has bit k.
            const uint64_t worv = warp_or(wv ? wred : 0);
            const uint64_t above = k + 1 < 64 ? (worv & (~0ull << (k + 1))) : 0;
            k = above ? __ffsll((long long)above) - 1 : 64;
            continue;
        }
        if (lane == 0) {
            c.perm[ib] = psrow;
            if (pivpos != ib) c.perm[pivpos] = hsrow;
            sh.E[s] = Es;
            sh.TI[s] = TIs;
            sh.T[s] = Ts;
            sh.pb[s] = k;
        }
        ++ib;
        const uint64_t bk = 1ull << k, es = 1ull << s;
        if (wv && (wred & bk)) { wred ^= Es; wtinv ^= TIs; wlc ^= es; }
        if (pr0 & bk) { pr0 ^= Es; pt0 ^= TIs; pl0 ^= es; }
        if (pr1 & bk) { pr1 ^= Es; pt1 ^= TIs; pl1 ^= es; }
        ++s;
        ++k;
    }
    // release the helpers
    if (lane == 0) sh.req = kReqDone;
    __syncwarp();
    bar_sync(1, kPanelThreads);

    if (lane == 0) {
        pi->R = R;
        pi->r = s;
    }
    pi->Zp[lane] = pt0;
    pi->Zp[lane + 32] = pt1;
    pi->Comp[lane] = pl0;
    pi->Comp[lane + 32] = pl1;
    __syncwarp();
    for (int t = lane; t < s; t += 32) {
        pi->Tinv[t] = sh.TI[t];
        pi->T[t] = sh.T[t];
        pi->Erow[t] = sh.E[t];
        pi->pivbit[t] = sh.pb[t];
        c.pivcols[R + t] = 64 * j + sh.pb[t];
    }
}

}  // namespace

cudaError_t launch_panel(const DecompCtx &c, int j, cudaStream_t s)
{
    k_panel<<<1, kPanelThreads, 0, s>>>(c, j);
    return cudaGetLastError();
}

}  // namespace gf2
