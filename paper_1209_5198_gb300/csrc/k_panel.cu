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
// How (GB300 design, not the paper's CPU loop).  Warp 0 holds a window of up
// to 64 consecutive rows (positions ib..ib+63, slot = position mod 64),
// already reduced by the pivots found so far, TRANSPOSED: lane l owns the
// columns (bits) l and l+32, each a 64-bit mask over the window slots.  For
// bit k the owner broadcasts column k; the first qualifying row is a
// find-first-set on it, circularly from the pivot slot; eliminating the
// pivot row E_s from the rows that have bit k is one masked XOR per column;
// each lane keeps bit s of its two columns of E_s, and the pivot's (bit,
// offset) is recorded in a register.  The row exchanges themselves (perm,
// slot tables) are replayed from those records before the window is
// refilled and at the end, off the per-bit path.
// At the end the coordinate maps are derived from those bits and the raw
// pivot words B_s:
//   U    = E restricted to the pivot columns (unit upper triangular),
//   Comp = rows of U^-1 at the pivot bits: E-coordinates, d = lambda(d) E,
//   T[s] = lambda(B_s) (B = T E),  T^-1,  Zp = Comp T^-1: B-coordinates, the
//          paper's pseudo-inverse Z (eq. pre:W) with B Z = I, D Z = Y.
// Rows outside the window are only scanned when the window has no
// qualifying row; those scans use all warps of the CTA.
#include <climits>

#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWin = 64;  // window slots
enum { kReqDone = 0, kReqFind = 1, kReqOr = 2 };

__device__ __forceinline__ void bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint64_t warp_or(uint64_t v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v |= __shfl_xor_sync(kFull, v, off);
    return v;
}

// 32 x 32 bit transpose across a warp: lane i holds row i (bit j = A[i][j]);
// afterwards lane i holds column i (bit j = A[j][i]).  Recursive exchange of
// the off-diagonal m x m blocks, m = 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t v, int lane)
{
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int m = 16 >> st;
        const uint32_t M = masks[st];
        const uint32_t p = __shfl_xor_sync(kFull, v, m);
        v = (lane & m) ? ((v & ~M) | ((p & ~M) >> m)) : ((v & M) | ((p & M) << m));
    }
    return v;
}

// 64 x 64 transpose: lane l holds a[0] = row l, a[1] = row l + 32 (64 bits
// each); afterwards a[0] = column l, a[1] = column l + 32.
__device__ __forceinline__ void transpose64(uint64_t a[2], int lane)
{
    const uint32_t r0l = transpose32((uint32_t)a[0], lane), r0h = transpose32((uint32_t)(a[0] >> 32), lane);
    const uint32_t r1l = transpose32((uint32_t)a[1], lane), r1h = transpose32((uint32_t)(a[1] >> 32), lane);
    a[0] = (uint64_t)r0l | ((uint64_t)r1l << 32);
    a[1] = (uint64_t)r0h | ((uint64_t)r1h << 32);
}

struct PanelShared {
    uint64_t pred[64];               // reduced unit rows red(e_p), for the scans
    uint64_t tab[kNumTables * 256];  // tables of pred for full reductions
    uint64_t E[64], B[64], T[64], TI[64], Comp[64], Ucol[64];
    int32_t pb[64];                  // pivot s -> its bit
    int32_t sidx[64];                // bit -> its pivot (or -1)
    int32_t slot_srow[kWin];
    uint64_t slot_raw[kWin];
    uint32_t rec32[64];  // fast path: pivot t -> bit | offset << 8
    uint64_t Lpr[64];    // fast path: probes that received E_t
    uint64_t nrow[32];   // fast path: rows entering the window
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
// the current pivots: red(w) = XOR_{p in w} pred[p]).
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

// <= 128 registers: 128 x 128 fits next to a 512 x 96 k_rest CTA on one SM
__global__ void __launch_bounds__(kPanelThreads, 4) k_panel(DecompCtx c, int j)
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
    uint64_t A = 0, B = 0;    // columns lane and lane+32 over the window slots
    uint64_t EA = 0, EB = 0;  // bit s: entry (s, column) of E_s
    uint64_t valid = 0;       // window slots holding a row
    uint32_t recA = 0, recB = 0;  // pivot lane / lane+32: its bit | offset << 8
    int ib = R, fill = R, s = 0, s_done = 0;
    sh.sidx[lane] = -1;
    sh.sidx[lane + 32] = -1;

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

    // The per-pivot bookkeeping is deferred out of the bit loop: pivot t
    // recorded (bit, offset f); the exchange of positions R+t and R+t+f is
    // replayed here, in order, on the slot -> row tables (before any refill
    // or spill changes the slots, and at the end).
    auto replay = [&]() {
        for (int t = s_done; t < s; ++t) {
            const uint32_t rec = __shfl_sync(kFull, t < 32 ? recA : recB, t & 31);
            if (lane == 0) {
                const int k = rec & 255, f = rec >> 8;
                const int pos = R + t, hs = pos & (kWin - 1), fs = (pos + f) & (kWin - 1);
                const int psrow = sh.slot_srow[fs];
                sh.B[t] = sh.slot_raw[fs];
                sh.pb[t] = k;
                sh.sidx[k] = t;
                c.perm[pos] = psrow;
                c.pivpanel[psrow] = j;
                if (f) {
                    const int hsrow = sh.slot_srow[hs];
                    c.perm[pos + f] = hsrow;
                    sh.slot_srow[fs] = hsrow;
                    sh.slot_raw[fs] = sh.slot_raw[hs];
                }
            }
        }
        s_done = s;
        __syncwarp();
    };

    // Loads positions [fill, min(ib + 64, n)) into their slots and reduces
    // the new rows by the pivots found so far, in pivot order.
    auto refill = [&]() {
        const int end = min(ib + kWin, n);
        if (fill >= end) return;
        replay();
        uint64_t raw[2];
        uint32_t isnew[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int slot = 32 * u + lane;
            const int p = fill + ((slot - fill) & (kWin - 1));
            isnew[u] = p < end;
            raw[u] = 0;
            if (isnew[u]) {
                const int srow = c.perm[p];
                raw[u] = Wj[(int64_t)srow * c.ldw];
                sh.slot_srow[slot] = srow;
                sh.slot_raw[slot] = raw[u];
            }
        }
        const uint64_t newm = (uint64_t)__ballot_sync(kFull, isnew[0]) | ((uint64_t)__ballot_sync(kFull, isnew[1]) << 32);
        transpose64(raw, lane);  // raw[0] = column lane, raw[1] = column lane+32 of the new rows
        uint64_t na = raw[0], nb = raw[1];
        __syncwarp();
        for (int t = 0; t < s; ++t) {
            const int k = sh.pb[t];
            const uint64_t m = __shfl_sync(kFull, k < 32 ? na : nb, k & 31);
            if ((EA >> t) & 1) na ^= m;
            if ((EB >> t) & 1) nb ^= m;
        }
        A |= na;
        B |= nb;
        valid |= newm;
        fill = end;
    };

    // E rows and the reduced unit rows red(e_p) into shared memory (rare paths)
    auto publish_reduced_units = [&]() {
        uint64_t e2[2] = {EA, EB};
        transpose64(e2, lane);  // e2[h] = E_{lane + 32h}
        sh.E[lane] = e2[0];
        sh.E[lane + 32] = e2[1];
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint64_t x = 1ull << (lane + 32 * h);
            for (int t = 0; t < s; ++t)
                if ((x >> sh.pb[t]) & 1) x ^= sh.E[t];
            sh.pred[lane + 32 * h] = x;
        }
        __syncwarp();
    };

    // ------------------------------------------------------------ fast path
    // The common case: the pivots of the block come from the first 96 rows.
    // Those rows are loaded once into registers (lane l: positions
    // R + l, R + 32 + l, R + 64 + l); the window has 32 slots (slot = position
    // - R mod 32, the lane that holds the row), so every column is a 32-bit
    // mask.  Each column also carries the 64 probe rows e_p (bit p of the
    // column's probe word = entry of the reduced e_p): a row v entering the
    // window is reduced by parity(v & probe word), with no serial chain, and
    // the probe bits of the broadcast column are the probe part of the L
    // column of the pivot, which gives Comp directly.  The exchanges are
    // recorded as (bit, offset) and resolved at the end by tracking the
    // position of every register row through them, one lane per row.  Any
    // other situation leaves the fast path after resolving what it did, and
    // the general loop below takes over.
    int k = 0;
    bool fast_complete = false;
    {
        const int fend = min(R + 3 * 32, n);  // rows available in registers
        uint64_t raw[3];
        int srw[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int p = R + 32 * u + lane;
            srw[u] = p < fend ? c.perm[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) raw[u] = srw[u] >= 0 ? Wj[(int64_t)srw[u] * c.ldw] : 0;
        uint32_t fA = 0, fB = 0, fvalid = 0;
        uint64_t Apr = 1ull << lane, Bpr = 1ull << (lane + 32);
        int hs = 0;                      // slot of the pivot slot ib
        uint32_t hsm = 1u, hmask = ~0u;  // its bit, and the slots at or after it
        uint64_t smask = 1ull;           // bit s
        auto fast_refill = [&]() {
            const int end = min(ib + 32, fend);
            if (fill >= end) return;
            const int p = fill + ((R + lane - fill) & 31);
            const bool isnew = p < end;
            const int u = (p - R) >> 5;
            const uint64_t v = isnew ? (u == 0 ? raw[0] : (u == 1 ? raw[1] : raw[2])) : 0;
            sh.nrow[lane] = v;
            const uint32_t newm = __ballot_sync(kFull, isnew);
            __syncwarp();
            uint32_t na = 0, nb = 0;
#pragma unroll 8
            for (int sl = 0; sl < 32; ++sl) {
                const uint64_t w = sh.nrow[sl];
                na |= (uint32_t)(__popcll(w & Apr) & 1) << sl;
                nb |= (uint32_t)(__popcll(w & Bpr) & 1) << sl;
            }
            fA |= na & newm;
            fB |= nb & newm;
            fvalid |= newm;
            fill = end;
            __syncwarp();
        };
        fast_refill();
        bool leave = false;
        while (k < nbits && ib < n) {
            if (fill < fend && fill - ib <= 16) fast_refill();
            const uint32_t ckw = __shfl_sync(kFull, k < 32 ? fA : fB, k & 31);
            const uint64_t ckp = __shfl_sync(kFull, k < 32 ? Apr : Bpr, k & 31);
            const uint32_t h = ckw & fvalid;
            const uint32_t after = h & hmask;
            const uint32_t pick = after ? after : h;
            if (!pick) {
                if (fill < fend && fill < ib + 32) {
                    fast_refill();
                    continue;
                }
                if (fill >= n) {  // every remaining row is in the window, none has bit k
                    const uint64_t worv = (uint64_t)__ballot_sync(kFull, (fA & fvalid) != 0) |
                                          ((uint64_t)__ballot_sync(kFull, (fB & fvalid) != 0) << 32);
                    const uint64_t above = k + 1 < 64 ? (worv & (~0ull << (k + 1))) : 0;
                    k = above ? __ffsll((long long)above) - 1 : 64;
                    continue;
                }
                leave = true;
                break;
            }
            const uint32_t fm = pick & (0u - pick);
            const bool moved = fm != hsm;
            const bool eA = (fA & fm) != 0, eB = (fB & fm) != 0;
            const uint32_t keep = ~(fm | hsm);
            fA = (fA & keep) | ((moved && (fA & hsm)) ? fm : 0u);
            fB = (fB & keep) | ((moved && (fB & hsm)) ? fm : 0u);
            fvalid &= ~hsm;
            const uint32_t ck1 = ckw & keep & fvalid;
            if (eA) {
                fA ^= ck1;
                Apr ^= ckp;
            }
            if (eB) {
                fB ^= ck1;
                Bpr ^= ckp;
            }
            EA |= eA ? smask : 0ull;
            EB |= eB ? smask : 0ull;
            sh.rec32[s] = (uint32_t)k | ((uint32_t)((__ffs((int)fm) - 1 - hs) & 31) << 8);
            sh.Lpr[s] = ckp;
            hs = (hs + 1) & 31;
            hsm = hs ? (hsm << 1) : 1u;
            hmask = hs ? (hmask << 1) : ~0u;
            smask <<= 1;
            ++ib;
            ++s;
            ++k;
        }
        __syncwarp();
        // resolve the recorded exchanges: final position of every register row
        int pos[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) pos[u] = R + 32 * u + lane;
        for (int t = 0; t < s; ++t) {
            const uint32_t rec = sh.rec32[t];
            const int a = R + t, b = a + (int)(rec >> 8);
#pragma unroll
            for (int u = 0; u < 3; ++u) pos[u] = pos[u] == a ? b : (pos[u] == b ? a : pos[u]);
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (srw[u] < 0) continue;
            if (pos[u] != R + 32 * u + lane) c.perm[pos[u]] = srw[u];
            if (pos[u] < R + s) {
                sh.B[pos[u] - R] = raw[u];
                c.pivpanel[srw[u]] = j;
            }
        }
        for (int t = lane; t < s; t += 32) {
            const int kt = (int)(sh.rec32[t] & 255);
            sh.pb[t] = kt;
            sh.sidx[kt] = t;
        }
        __syncwarp();
        s_done = s;
        fill = ib;  // the general loop starts from an empty window
        if (!leave) {
            fast_complete = true;
            uint64_t l2[2] = {s > lane ? sh.Lpr[lane] : 0ull, s > lane + 32 ? sh.Lpr[lane + 32] : 0ull};
            transpose64(l2, lane);  // Comp[p] bit t = probe p received E_t
            sh.Comp[lane] = l2[0];
            sh.Comp[lane + 32] = l2[1];
        }
    }

    if (!fast_complete) refill();
    while (!fast_complete && k < nbits && ib < n) {
        if (fill < n && fill - ib <= kWin / 2) refill();  // keep the window at least half full
        const uint64_t ck0 = __shfl_sync(kFull, k < 32 ? A : B, k & 31);
        // first window row with bit k, from the pivot slot on (circularly)
        const int hs = ib & (kWin - 1);
        const uint64_t h = ck0 & valid;
        const uint64_t after = h & (~0ull << hs);
        const uint64_t pick = after ? after : h;

        if (!pick) {
            if (fill < n && fill < ib + kWin) {  // room in the window: load more rows
                refill();
                continue;
            }
            replay();
            if (fill < n) {
                // the window is full and has no candidate: scan the rows behind it
                publish_reduced_units();
                uint64_t ck = 0;  // bit p: entry k of red(e_p)
                for (int p = 0; p < 64; ++p) ck |= ((sh.pred[p] >> k) & 1) << p;
                request(kReqFind, fill, ck, 0);
                const int q = sh.found;
                if (q != INT_MAX) {
                    // pivot outside the window; the row in the pivot slot
                    // moves there and leaves the window
                    const int psrow = c.perm[q];
                    const uint64_t v = Wj[(int64_t)psrow * c.ldw];
                    uint64_t red = 0;
                    for (uint64_t b = v; b; b &= b - 1) red ^= sh.pred[__ffsll((long long)b) - 1];
                    const uint32_t eA = (red >> lane) & 1, eB = (red >> (lane + 32)) & 1;
                    const uint64_t hm = 1ull << hs;
                    const uint64_t ck1 = ck0 & valid & ~hm;
                    if (eA) A ^= ck1;
                    if (eB) B ^= ck1;
                    A &= ~hm;
                    B &= ~hm;
                    EA |= (uint64_t)eA << s;
                    EB |= (uint64_t)eB << s;
                    if (lane == 0) {
                        c.perm[ib] = psrow;
                        c.perm[q] = sh.slot_srow[hs];
                        c.pivpanel[psrow] = j;
                        sh.B[s] = v;
                        sh.pb[s] = k;
                        sh.sidx[k] = s;
                    }
                    __syncwarp();
                    valid &= ~hm;
                    ++ib;
                    ++s;
                    s_done = s;
                    ++k;
                    continue;
                }
                // Bit k has no pivot.  The next bit that can have one is the
                // lowest bit above k set in some reduced remaining row.
                const uint64_t worv = (uint64_t)__ballot_sync(kFull, (A & valid) != 0) |
                                      ((uint64_t)__ballot_sync(kFull, (B & valid) != 0) << 32);
                request(kReqOr, fill, 0, worv);
                const uint64_t above = k + 1 < 64 ? (sh.orv & (~0ull << (k + 1))) : 0;
                k = above ? __ffsll((long long)above) - 1 : 64;
                continue;
            }
            // every remaining row is in the window and none has bit k
            const uint64_t worv = (uint64_t)__ballot_sync(kFull, (A & valid) != 0) |
                                  ((uint64_t)__ballot_sync(kFull, (B & valid) != 0) << 32);
            const uint64_t above = k + 1 < 64 ? (worv & (~0ull << (k + 1))) : 0;
            k = above ? __ffsll((long long)above) - 1 : 64;
            continue;
        }

        // pivot: slot fs, f places after the pivot slot.  The pivot row
        // leaves the window; the row in the pivot slot (when f > 0) takes
        // its slot.  The head row has bit k = 0 when f > 0.
        const int fs = __ffsll((long long)pick) - 1;
        const int f = (fs - hs) & (kWin - 1);
        const uint64_t fm = 1ull << fs, hm = 1ull << hs;
        const bool eA = (A & fm) != 0, eB = (B & fm) != 0;
        const uint64_t keep = ~(fm | hm);
        const uint64_t mvA = (f && (A & hm)) ? fm : 0, mvB = (f && (B & hm)) ? fm : 0;
        A = (A & keep) | mvA;
        B = (B & keep) | mvB;
        valid &= ~hm;
        const uint64_t ck1 = ck0 & keep & valid;
        if (eA) A ^= ck1;
        if (eB) B ^= ck1;
        EA |= (uint64_t)eA << s;
        EB |= (uint64_t)eB << s;
        const uint32_t rec = (uint32_t)k | ((uint32_t)f << 8);
        recA = (lane == s) ? rec : recA;
        recB = (lane + 32 == s) ? rec : recB;
        ++ib;
        ++s;
        ++k;
    }
    replay();
    // release the helpers
    if (lane == 0) sh.req = kReqDone;
    __syncwarp();
    bar_sync(1, kPanelThreads);

    // ---- coordinate maps from E (bits EA/EB) and the raw pivot words B
    {
        uint64_t e2[2] = {EA, EB};
        transpose64(e2, lane);
        sh.E[lane] = e2[0];
        sh.E[lane + 32] = e2[1];
        // column s' of U = column pb[s'] of E
        const int sa = sh.sidx[lane], sb = sh.sidx[lane + 32];
        if (sa >= 0) sh.Ucol[sa] = EA;
        if (sb >= 0) sh.Ucol[sb] = EB;
    }
    __syncwarp();
    const int c0 = lane, c1 = lane + 32;
    // rows c0, c1 of U^-1: U^T y = e_c, forward over t > c (fixed trip count);
    // Comp at the pivot bits.  (The fast path already has Comp from its probes.)
    if (!fast_complete) {
        uint64_t y0 = c0 < s ? (1ull << c0) : 0, y1 = c1 < s ? (1ull << c1) : 0;
#pragma unroll 8
        for (int t = 1; t < 64; ++t) {
            const uint64_t u = sh.Ucol[t];
            const bool ok = t < s;
            const uint64_t b0 = (uint64_t)(__popcll(u & y0) & 1) << t;
            const uint64_t b1 = (uint64_t)(__popcll(u & y1) & 1) << t;
            if (ok && t > c0) y0 |= b0;
            if (ok && t > c1) y1 |= b1;
        }
        sh.TI[c0] = y0;  // staging: rows of U^-1
        sh.TI[c1] = y1;
        __syncwarp();
        const int t0 = sh.sidx[c0], t1 = sh.sidx[c1];
        sh.Comp[c0] = t0 >= 0 ? sh.TI[t0] : 0;
        sh.Comp[c1] = t1 >= 0 ? sh.TI[t1] : 0;
    }
    __syncwarp();
    // T[t] = lambda(B_t) = XOR over the bits p of B_t of Comp[p]
    {
        const uint64_t b0 = c0 < s ? sh.B[c0] : 0, b1 = c1 < s ? sh.B[c1] : 0;
        uint64_t a0 = 0, a1 = 0;
#pragma unroll 8
        for (int p = 0; p < 64; ++p) {
            const uint64_t cp = sh.Comp[p];
            if ((b0 >> p) & 1) a0 ^= cp;
            if ((b1 >> p) & 1) a1 ^= cp;
        }
        sh.T[c0] = a0;
        sh.T[c1] = a1;
    }
    __syncwarp();
    // T^-1 by columns: T x = e_c, x[t] = parity(T[t] & x) for t > c
    uint64_t x2[2];
    {
        uint64_t x0 = c0 < s ? (1ull << c0) : 0, x1 = c1 < s ? (1ull << c1) : 0;
#pragma unroll 8
        for (int t = 1; t < 64; ++t) {
            const uint64_t tt = sh.T[t];
            const bool ok = t < s;
            const uint64_t b0 = (uint64_t)(__popcll(tt & x0) & 1) << t;
            const uint64_t b1 = (uint64_t)(__popcll(tt & x1) & 1) << t;
            if (ok && t > c0) x0 |= b0;
            if (ok && t > c1) x1 |= b1;
        }
        x2[0] = x0;
        x2[1] = x1;
    }
    transpose64(x2, lane);  // rows of T^-1
    sh.TI[c0] = x2[0];
    sh.TI[c1] = x2[1];
    __syncwarp();
    if (lane == 0) {
        pi->R = R;
        pi->r = s;
    }
    {
        const uint64_t m0 = sh.Comp[c0], m1 = sh.Comp[c1];
        uint64_t z0 = 0, z1 = 0;
#pragma unroll 8
        for (int t = 0; t < 64; ++t) {
            const uint64_t ti = sh.TI[t];
            if ((m0 >> t) & 1) z0 ^= ti;
            if ((m1 >> t) & 1) z1 ^= ti;
        }
        pi->Zp[c0] = z0;
        pi->Zp[c1] = z1;
        pi->Comp[c0] = m0;
        pi->Comp[c1] = m1;
    }
    for (int t = lane; t < s; t += 32) {
        pi->Tinv[t] = sh.TI[t];
        pi->T[t] = sh.T[t];
        pi->Erow[t] = sh.E[t];
        pi->pivbit[t] = sh.pb[t];
        c.pivcols[R + t] = 64 * j + sh.pb[t];
    }
}

// Unused dynamic shared memory that keeps a panel CTA off any SM holding a
// persistent k_rest CTA (about 133 KB): the panel runs on the SM k_rest
// leaves free, without other warps competing for its scheduler.
constexpr int kPanelReserveBytes = 110 * 1024;

}  // namespace

cudaError_t prepare_panel_kernel()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelReserveBytes);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t launch_panel(const DecompCtx &c, int j, cudaStream_t s)
{
    const cudaError_t e = prepare_panel_kernel();
    if (e != cudaSuccess) return e;
    k_panel<<<1, kPanelThreads, kPanelReserveBytes, s>>>(c, j);
    return cudaGetLastError();
}

}  // namespace gf2
