// Device code of the panel step: selection of the pivot rows of one 64-column
// block and the pseudo-inverse that expresses every other row of the block
// through them.  Shared by the panel kernel of the decomposition and by the
// batched decomposition (one CTA per matrix); every definition is internal to
// the translation unit that includes this file.
//
// What it computes (Sections 4.1-4.4 of the paper, Procedure buildZ): for
// bit k = 0..63 of column block j, the first row at or after the current
// pivot slot (in the current row order) whose entry k, reduced by the pivots
// already chosen in this block, is one -- the non-singularity condition
// (eq. cond:nonsing:Bk) -- is exchanged with the pivot slot.  A bit with no
// such row gets no pivot (the paper inserts the virtual row (0,1,0) there,
// Section 4.4); no column is ever exchanged.
//
// How (GB300 design, not the paper's CPU loop).  Warp 0 holds rows reduced
// by the pivots found so far TRANSPOSED: lane l owns the columns (bits) l and
// l+32 as masks over row slots.  For bit k the owner broadcasts column k; the
// first qualifying row is a find-first-set on it; eliminating the pivot row
// E_s from the rows that have bit k is one masked XOR per column, and each
// lane keeps bit s of its two columns of E_s.  The common case (the fast
// path) holds the first 96 rows for the whole block with the exchanges
// applied to the masks themselves; the general loop keeps a circular window
// of 64 rows (slot = position mod 64), refilled as pivots consume it, and
// replays the recorded exchanges on its slot tables off the per-bit path.
// At the end the coordinate maps are derived from those bits and the raw
// pivot words B_s:
//   U    = E restricted to the pivot columns (unit upper triangular),
//   Comp = rows of U^-1 at the pivot bits: E-coordinates, d = lambda(d) E,
//   T[s] = lambda(B_s) (B = T E),  T^-1,  Zp = Comp T^-1: B-coordinates, the
//          paper's pseudo-inverse Z (eq. pre:W) with B Z = I, D Z = Y.
// Rows outside the window are only scanned when the window has no
// qualifying row; those scans use all warps of the CTA.
#pragma once
#include <climits>

#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWin = 64;  // window slots
enum { kReqDone = 0, kReqFind = 1 };

__device__ __forceinline__ void bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Barrier of the panel's kPanelThreads threads (named barrier kBarPanel).
// The panel step synchronises its own threads only, so that it also runs in
// the first kPanelThreads threads of a larger CTA (the persistent
// decomposition kernel, whose other warps of that CTA have left).
constexpr int kBarPanel = 3;

__device__ __forceinline__ void panel_sync() { bar_sync(kBarPanel, kPanelThreads); }

// panel_sync that also returns whether any of the panel's threads passed p != 0
__device__ __forceinline__ int panel_sync_or(int p)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred pin, pout;\n\tsetp.ne.s32 pin, %1, 0;\n\t"
        "bar.red.or.pred pout, %2, %3, pin;\n\tselp.s32 %0, 1, 0, pout;\n\t}"
        : "=r"(r)
        : "r"(p), "n"(kBarPanel), "n"(kPanelThreads)
        : "memory");
    return r;
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
    uint64_t fraw[96];   // fast path: raw word and storage row of each register row
    int32_t fsrow[96];
    int32_t prow[64];    // pivot s -> its storage row
    uint64_t zt[256];    // 16 tables of 16: y = F * Zp of the previous panel
    uint64_t ct[256];    // 16 tables of 16: y * C, C = word j of the previous panel's pivot rows
    uint64_t mask;
    unsigned long long orv;
    int req, from, found;
    // the panel's list of nonzero rows behind the window (general path, when
    // the context provides zpos / zraw): entries [0, zn) are the positions
    // with a nonzero panel word among [zfrom, zto), in position order, and
    // their raw words; zhead: the first entry at or after the current scan's
    // start; found_idx: the entry of the row a scan found
    int zn, zfrom, zto, zhead, found_idx;
    uint64_t found_raw;  // the raw word of the row found (with the list)
    int wcnt[kPanelThreads / 32];
    uint64_t basis[64];  // end phase: the 8-bit blocks' basis effects of a triangular sweep
    int ns;              // end phase: pivots found in the panel
};

// Word j of storage row i with the updates of every panel < j.  W holds it
// without the update of panel j-1, which is added here from the row's
// finished word j-1 (Fp[i * fstride]: F, or W itself for j = 1): y = that
// word * Zp, then word ^= y * C through the tables zt / ct (Fp = null when
// panel j-1 left nothing to apply).
struct PrevPanel {
    const uint64_t *Fp;
    int64_t fstride;
};

// The update of panel j-1 for a row whose finished word j-1 is f: (f Zp) C.
__device__ __forceinline__ uint64_t prev_update(const PanelShared &sh, uint64_t f)
{
    uint64_t y = 0, u = 0;
#pragma unroll
    for (int g = 0; g < 16; ++g) y ^= sh.zt[g * 16 + (int)((f >> (4 * g)) & 15)];
#pragma unroll
    for (int g = 0; g < 16; ++g) u ^= sh.ct[g * 16 + (int)((y >> (4 * g)) & 15)];
    return u;
}

__device__ __forceinline__ uint64_t panel_word(const uint64_t *Wj, const PrevPanel &pv, const PanelShared &sh, int i)
{
    uint64_t w = Wj[(int64_t)i * kTileWords];
    if (pv.Fp) w ^= prev_update(sh, pv.Fp[(int64_t)i * pv.fstride]);
    return w;
}

// Tables of the reduction by the current pivots (red(w) = XOR_{p in w}
// pred[p]), 8 bits at a time.
__device__ __forceinline__ void build_reduction_tables(PanelShared &sh)
{
    for (int e = threadIdx.x; e < kNumTables * 256; e += kPanelThreads) {
        const int g = e >> 8, x = e & 255;
        uint64_t acc = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if ((x >> b) & 1) acc ^= sh.pred[8 * g + b];
        sh.tab[e] = acc;
    }
    panel_sync();
}

__device__ __forceinline__ uint64_t reduce_word(const PanelShared &sh, uint64_t v)
{
    uint64_t r = 0;
#pragma unroll
    for (int g = 0; g < kNumTables; ++g) r ^= sh.tab[g * 256 + ((v >> (8 * g)) & 255)];
    return r;
}

// Storage of the row list: entries below cap in shared memory (the panel
// kernel's otherwise unused dynamic shared memory), the rest in c.zpos /
// c.zraw (same index).
struct RowList {
    uint64_t *raw;
    int32_t *pos;
    int cap;
};

__device__ __forceinline__ int32_t list_pos(const DecompCtx &c, const RowList &L, int e)
{
    return e < L.cap ? L.pos[e] : c.zpos[e];
}

__device__ __forceinline__ uint64_t list_raw(const DecompCtx &c, const RowList &L, int e)
{
    return e < L.cap ? L.raw[e] : c.zraw[e];
}

__device__ __forceinline__ void list_put(const DecompCtx &c, const RowList &L, int e, int32_t p, uint64_t v)
{
    if (e < L.cap) {
        L.pos[e] = p;
        L.raw[e] = v;
    } else {
        c.zpos[e] = p;
        c.zraw[e] = v;
    }
}

// Positions [from, n): first one whose panel word w has parity(w & mask) = 1.
// The same pass ORs the fully reduced words into sh.orv, so that when no
// position qualifies sh.orv holds the OR over all of them (a block whose
// remaining rows are zero, as once the rank is used up, costs one pass).
//
// With a row list (c.zpos): the rows already read in this panel are tested
// from the list of the nonzero ones (a zero row never qualifies and adds
// nothing to the OR), and the pass over the rows behind the list appends the
// nonzero rows it reads.  So every row is read from memory at most once per
// panel, however many bits need a scan -- sparse blocks, where most rows are
// zero and most bits find no candidate in the window, scan for nearly every
// bit.  A raw word does not change during the panel (the parity test takes
// the current pivots through the mask); the exchange that moves the pivot
// slot's row to a listed position updates that entry.
__device__ __noinline__ void scan_find(const DecompCtx &c, const uint64_t *Wj, const PrevPanel pv, PanelShared &sh,
                                       const RowList L)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int from = sh.from, n = c.n;
    const uint64_t mask = sh.mask;
    uint64_t acc = 0;
    if (!c.zpos) {
        build_reduction_tables(sh);
        constexpr int U = 4;
        for (int base = from; base < n; base += kPanelThreads * U) {
            int srow[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = base + u * kPanelThreads + tid;
                srow[u] = q < n ? c.perm[q] : -1;
            }
            uint64_t v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = srow[u] >= 0 ? panel_word(Wj, pv, sh, srow[u]) : 0;
            int hit = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc |= reduce_word(sh, v[u]);
                if (!hit && (__popcll(v[u] & mask) & 1)) {
                    atomicMin(&sh.found, base + u * kPanelThreads + tid);
                    hit = 1;
                }
            }
            if (panel_sync_or(hit)) break;
        }
        acc = warp_or(acc);
        if (lane == 0 && acc) atomicOr(&sh.orv, (unsigned long long)acc);
        return;
    }

    // the list: started by the panel's first scan; its head moved to `from`
    if (tid == 0) {
        if (sh.zfrom < 0) {
            sh.zfrom = sh.zto = from;
            sh.zn = 0;
            sh.zhead = 0;
        }
        int h = sh.zhead;
        while (h < sh.zn && list_pos(c, L, h) < from) ++h;
        sh.zhead = h;
    }
    panel_sync();
    bool found = false;
    {
        // (2 entries per thread between barriers: the qualifying row is
        // usually near the head of the list, and larger steps test rows past
        // it -- 16 per thread measured 12% slower on S_n, 4 about 1% slower)
        constexpr int UL = 2;
        const int zn = sh.zn;
        for (int b = sh.zhead; b < zn && !found; b += kPanelThreads * UL) {
            int hit = 0;
#pragma unroll
            for (int u = 0; u < UL; ++u) {
                const int e = b + u * kPanelThreads + tid;
                if (e < zn) {
                    const uint64_t v = list_raw(c, L, e);
                    if (!hit && (__popcll(v & mask) & 1)) {
                        atomicMin(&sh.found_idx, e);
                        hit = 1;
                    }
                }
            }
            found = panel_sync_or(hit);
        }
    }
    // the rows behind the list, appended in position order
    constexpr int U = 8;
    const int p0 = max(from, sh.zto);
    for (int base = p0; base < n && !found; base += kPanelThreads * U) {
        int srow[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * kPanelThreads + tid;
            srow[u] = q < n ? c.perm[q] : -1;
        }
        uint64_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = srow[u] >= 0 ? panel_word(Wj, pv, sh, srow[u]) : 0;
        uint64_t any = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) any |= v[u];
        int hit = 0;
        if (panel_sync_or(any != 0)) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool nz = v[u] != 0;
                const unsigned bal = __ballot_sync(kFull, nz);
                if (lane == 0) sh.wcnt[warp] = __popc(bal);
                panel_sync();
                int off = sh.zn, total = 0;
#pragma unroll
                for (int w = 0; w < kPanelThreads / 32; ++w) {
                    off += w < warp ? sh.wcnt[w] : 0;
                    total += sh.wcnt[w];
                }
                if (nz) {
                    const int e = off + __popc(bal & ((1u << lane) - 1));
                    list_put(c, L, e, base + u * kPanelThreads + tid, v[u]);
                    if (!hit && (__popcll(v[u] & mask) & 1)) {
                        atomicMin(&sh.found_idx, e);
                        hit = 1;
                    }
                }
                panel_sync();  // every thread has read sh.zn and the counts
                if (tid == 0) sh.zn += total;
            }
        }
        if (tid == 0) sh.zto = min(base + kPanelThreads * U, n);
        found = panel_sync_or(hit);
    }
    // no row qualifies: every nonzero row behind the window is now listed, so
    // their OR comes from the list (only this case needs the reduction
    // tables; a scan that finds its row skips them)
    if (!found) {
        build_reduction_tables(sh);
        const int zh = sh.zhead, zn = sh.zn;
        for (int e = zh + tid; e < zn; e += kPanelThreads) acc |= reduce_word(sh, list_raw(c, L, e));
        acc = warp_or(acc);
        if (lane == 0 && acc) atomicOr(&sh.orv, (unsigned long long)acc);
    }
    panel_sync();
    if (tid == 0 && found) {
        sh.found = list_pos(c, L, sh.found_idx);
        sh.found_raw = list_raw(c, L, sh.found_idx);
    }
}

// Fast-path state of warp 0.  The 96 rows of positions R..R+95 are held
// transposed: lane l owns the columns (bits) l (A) and l+32 (B) of the block,
// each as three 32-bit masks over the slots (slot = position - R; word w
// covers slots 32w..32w+31).  Lanes 0..6 also own the identity columns: bit b
// of the original slot of the row now in each slot, moved with the rows so
// that the exchanges need no other bookkeeping.  EA / EB bit s: entry of E_s
// in column l / l+32.
struct FastCols {
    uint32_t A[3], B[3], ID[3];
    uint64_t EA, EB;
    int k, s;
};

// Word u of identity column b (lane b < 7): bit i is bit b of slot 32u + i.
__device__ __forceinline__ uint32_t slot_index_bits(int u, int b)
{
    switch (b) {
    case 0: return 0xAAAAAAAAu;
    case 1: return 0xCCCCCCCCu;
    case 2: return 0xF0F0F0F0u;
    case 3: return 0xFF00FF00u;
    case 4: return 0xFFFF0000u;
    case 5: return (u & 1) ? ~0u : 0u;
    case 6: return (u & 2) ? ~0u : 0u;
    default: return 0u;
    }
}

// Pivot s for bit k: its first qualifying row sits in the slot of the one-hot
// mask fm0..fm2 (words 0..2; W2 = false when it is in word 0 or 1); the pivot
// slot s is in word P.  Slots s and f exchange their rows, the pivot row
// leaves the window (slot s is cleared) and its bits E_s are XORed into every
// row with bit k: ck = column k without the pivot row (the row moved out of
// slot s has bit k = 0 whenever f != s).
template <int P, bool W2>
__device__ __forceinline__ void fast_pivot(FastCols &st, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t fm0,
                                           uint32_t fm1, uint32_t fm2)
{
    const uint32_t hsm = 1u << (st.s & 31);
    const uint32_t ck0 = c0 ^ fm0, ck1 = c1 ^ fm1, ck2 = c2 ^ fm2;
    auto at_f = [&](const uint32_t (&X)[3]) -> bool {
        return (W2 ? ((X[0] & fm0) | (X[1] & fm1) | (X[2] & fm2)) : ((X[0] & fm0) | (X[1] & fm1))) != 0;
    };
    auto eliminate = [&](uint32_t (&X)[3]) -> bool {
        const bool e = at_f(X);
        const bool hb = (X[P] & hsm) != 0;
        if (e != hb) {  // the head row's bit moves to slot f
            X[0] ^= fm0;
            X[1] ^= fm1;
            if (W2) X[2] ^= fm2;
        }
        X[P] &= ~hsm;
        if (e) {
            X[0] ^= ck0;
            X[1] ^= ck1;
            X[2] ^= ck2;
        }
        return e;
    };
    const bool eA = eliminate(st.A), eB = eliminate(st.B);
    {  // identity bits: exchange only
        const bool e = at_f(st.ID);
        const bool hb = (st.ID[P] & hsm) != 0;
        if (e != hb) {
            st.ID[0] ^= fm0;
            st.ID[1] ^= fm1;
            if (W2) st.ID[2] ^= fm2;
            st.ID[P] ^= hsm;
        }
    }
    const uint64_t sm = 1ull << st.s;
    st.EA |= eA ? sm : 0ull;
    st.EB |= eB ? sm : 0ull;
    ++st.s;
    ++st.k;
}

// Pivots with the pivot slot in word P (s < 32 for P = 0, s < 64 for P = 1),
// up to smax pivots.  Returns true when bit k has no qualifying row among the
// registers while more rows exist (the general loop takes over).
template <int P>
__device__ __forceinline__ bool fast_phase(FastCols &st, int nbits, int smax, bool more_rows)
{
    const int send = min(smax, 32 * (P + 1));
    while (st.k < nbits && st.s < send) {
        const int src = st.k & 31;
        const bool lo = st.k < 32;
        const uint32_t c0 = __shfl_sync(kFull, lo ? st.A[0] : st.B[0], src);
        const uint32_t c1 = __shfl_sync(kFull, lo ? st.A[1] : st.B[1], src);
        const uint32_t c2 = __shfl_sync(kFull, lo ? st.A[2] : st.B[2], src);
        if (c0 | c1) {
            const uint32_t fm0 = c0 & (0u - c0);
            const uint32_t fm1 = c0 ? 0u : (c1 & (0u - c1));
            fast_pivot<P, false>(st, c0, c1, c2, fm0, fm1, 0u);
        } else if (c2) {
            fast_pivot<P, true>(st, c0, c1, c2, 0u, 0u, c2 & (0u - c2));
        } else {
            if (more_rows) return true;
            ++st.k;  // every remaining row is held and none has bit k
        }
    }
    return false;
}

// ---------------------------------------------------------------- end phase
// The coordinate maps of a panel, from E (rows in sh.E), U = E at the pivot
// columns (columns in sh.Ucol, unit upper triangular) and the raw pivot
// words B (sh.B):
//   Comp = rows of U^-1 at the pivot bits (lambda(d) = d Comp),
//   T    = B Comp (lambda of every pivot word, unit lower triangular),
//   T^-1, and Zp = Comp T^-1 (the paper's Z: y(d) = d Zp).
// Every map is linear over F2 and taken 8 bits at a time with 256-entry
// tables (Section 6's Four Russians method on 64 x 64 matrices): a product
// is 8 independent lookups per row; a triangular solve (M x = e_c, M unit
// upper triangular with column t in Mcol[t]) is 8 dependent lookups, one
// per 8-row block from the top: the backward sweep of one block (for t in
// the block, downwards: if x_t then x ^= the part of column t above the
// diagonal) changes x by a linear function of the block's 8 entries of x,
// tabulated from its 8 basis effects.  All kPanelThreads threads take part.

// tab[256 g + x] = XOR of basis[8 g + i] over the bits i of x, for the 8
// tables g: thread (g, q) fills entries 16 q .. 16 q + 15 of table g by a
// Gray walk (one XOR per entry) that starts at position q of the cyclic
// 4-bit Gray sequence, so that at every step the 16 threads of one table
// write 16 different bank pairs (no shared-memory bank conflicts).
__device__ __forceinline__ void fill_tables(const uint64_t *basis, uint64_t *tab)
{
    static_assert(kPanelThreads == 128, "8 tables x 16 threads");
    const int tid = threadIdx.x;
    const int g = tid >> 4, q = tid & 15;
    const uint64_t *bs = basis + 8 * g;
    uint64_t v = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if ((q >> i) & 1) v ^= bs[4 + i];
    const int gq = q ^ (q >> 1);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if ((gq >> i) & 1) v ^= bs[i];
    uint64_t *tb = tab + 256 * g + 16 * q;
    tb[gq] = v;
#pragma unroll 4
    for (int step = 1; step < 16; ++step) {
        const int p = (q + step) & 15;
        v ^= bs[p ? __ffs(p) - 1 : 3];  // (from 15 to 0 the cyclic sequence changes bit 3)
        tb[p ^ (p >> 1)] = v;
    }
}

// Tables of the block sweeps of M (columns Mcol, zero past the rank) in tab.
__device__ __forceinline__ void sweep_tables(const uint64_t *Mcol, PanelShared &sh)
{
    const int tid = threadIdx.x;
    if (tid < 64) {  // the effect of entry tid alone in its block
        const int lo = tid & ~7;
        uint64_t x = 1ull << tid;
        for (int t = tid; t >= lo; --t)
            if ((x >> t) & 1) x ^= Mcol[t] & ((1ull << t) - 1);
        sh.basis[tid] = x ^ (1ull << tid);
    }
    panel_sync();
    fill_tables(sh.basis, sh.tab);
    panel_sync();
}

// x = M^-1 x by the block sweeps (tables of sweep_tables)
__device__ __forceinline__ uint64_t sweep_apply(const PanelShared &sh, uint64_t x)
{
#pragma unroll
    for (int b = 7; b >= 0; --b) x ^= sh.tab[256 * b + (int)((x >> (8 * b)) & 255)];
    return x;
}

// Tables of the rows R[0..64): tab[256 g + x] = XOR of R[8 g + i] over the bits i of x.
__device__ __forceinline__ void product_tables(const uint64_t *R, PanelShared &sh)
{
    fill_tables(R, sh.tab);
    panel_sync();
}

// w R (the XOR of the rows R[p] over the bits p of w), tables of product_tables
__device__ __forceinline__ uint64_t product_apply(const PanelShared &sh, uint64_t w)
{
    uint64_t r = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) r ^= sh.tab[256 * g + (int)((w >> (8 * g)) & 255)];
    return r;
}

__device__ __forceinline__ void panel_end_phase(const DecompCtx &c, int j, int R, PanelInfo *pi, PanelShared &sh,
                                                unsigned long long *tr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = sh.ns;
    (void)tr;
    // U^-1 by columns (warp 0: columns lane, lane + 32), then its rows and Comp
    sweep_tables(sh.Ucol, sh);
    if (warp == 0) {
        uint64_t x[2];
        x[0] = sweep_apply(sh, lane < s ? 1ull << lane : 0);
        x[1] = sweep_apply(sh, lane + 32 < s ? 1ull << (lane + 32) : 0);
        transpose64(x, lane);  // x[h] = row lane + 32h of U^-1
        sh.TI[lane] = x[0];
        sh.TI[lane + 32] = x[1];
        __syncwarp();
        const int t0 = sh.sidx[lane], t1 = sh.sidx[lane + 32];
        sh.Comp[lane] = t0 >= 0 ? sh.TI[t0] : 0;
        sh.Comp[lane + 32] = t1 >= 0 ? sh.TI[t1] : 0;
    }
    panel_sync();
    GF2_TR(if (tr && tid == 0) tr[kTrPanelUinv * kTraceMaxPanels + j] = trace_clock();)
    // T[t] = lambda(B_t) = B_t Comp
    product_tables(sh.Comp, sh);
    uint64_t Tt = 0;
    if (tid < 64) Tt = tid < s ? product_apply(sh, sh.B[tid]) : 0;
    panel_sync();  // (every lookup into the tables done)
    if (tid < 64) sh.T[tid] = Tt;
    panel_sync();
    GF2_TR(if (tr && tid == 0) tr[kTrPanelT * kTraceMaxPanels + j] = trace_clock();)
    // T^-1 by rows: T^T y = e_c (column t of T^T = row t of T) gives row c
    sweep_tables(sh.T, sh);
    uint64_t Yc = 0;
    if (tid < 64) Yc = sweep_apply(sh, tid < s ? 1ull << tid : 0);
    panel_sync();
    if (tid < 64) sh.TI[tid] = Yc;
    panel_sync();
    GF2_TR(if (tr && tid == 0) tr[kTrPanelTinv * kTraceMaxPanels + j] = trace_clock();)
    // Zp = Comp T^-1
    product_tables(sh.TI, sh);
    if (tid < 64) {
        const uint64_t m = sh.Comp[tid];
        const uint64_t z = product_apply(sh, m);
        GF2_TR(if (tr && tid == 0) {
            asm volatile("" ::"l"(z));
            tr[kTrPanelZp * kTraceMaxPanels + j] = trace_clock();
        })
        pi->Zp[tid] = z;
        pi->Comp[tid] = m;
    }
    if (tid == 0) {
        pi->R = R;
        pi->r = s;
    }
    for (int t = tid; t < s; t += kPanelThreads) {
        pi->Tinv[t] = sh.TI[t];
        pi->T[t] = sh.T[t];
        pi->Erow[t] = sh.E[t];
        pi->pivbit[t] = sh.pb[t];
        pi->prow[t] = sh.prow[t];
        c.pivcols[R + t] = 64 * j + sh.pb[t];
    }
    GF2_TR(if (tr && tid == 0) tr[kTrPanelEnd * kTraceMaxPanels + j] = trace_clock();)
}

// The panel step of block j, run by one CTA of kPanelThreads threads (warp 0
// searches, warps 1..3 serve the scans of the general path).
// zs / zcap: shared memory for the first zcap entries of the row list (zcap
// words of raw rows, then zcap int32 positions), or none.
// tr: the trace build's timeline of the decomposition (null: no stamps).
__device__ __forceinline__ void panel_block(const DecompCtx &c, int j, PanelShared &sh, uint64_t *zs = nullptr,
                                            int zcap = 0, unsigned long long *tr = nullptr)
{
    const RowList L{zs, zs ? reinterpret_cast<int32_t *>(zs + zcap) : nullptr, zs ? zcap : 0};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = j == 0 ? 0 : panel_info(c, j - 1)->R + panel_info(c, j - 1)->r;
    const int n = c.n;
    const int nbits = min(64, c.m - 64 * j);
    PanelInfo *pi = panel_info(c, j);
    const uint64_t *Wj = c.W + (int64_t)(j / kTileWords) * c.tstride + (j % kTileWords);  // word j of row i: Wj[T i]

    if (tid == 0) sh.zfrom = -1;  // no row list yet in this panel
    // no pivot: no rows or columns left, or (panel j-1 had none and the
    // look-ahead of panel j-2 looked and saw only zero words j in the rows
    // still active) every row's word j is zero -- the rank is used up,
    // nothing to scan
    const bool zero_block = c.orw && j >= 2 && panel_info(c, j - 1)->r == 0 &&
                            *reinterpret_cast<volatile const int32_t *>(c.orw + j) == 2;
    if (R >= n || nbits <= 0 || zero_block) {
        if (tid == 0) {
            pi->R = R;
            pi->r = 0;
        }
        return;
    }

    // the update of panel j-1 that W does not hold yet (see panel_word)
    PrevPanel pv{nullptr, 1};
    const int rp = j > 0 ? panel_info(c, j - 1)->r : 0;
    if (rp > 0 && c.F) {
        if (j == 1) {  // word 0 has no earlier update: W holds it
            pv.Fp = c.W;
            pv.fstride = kTileWords;
        } else {
            pv.Fp = c.F + (int64_t)((j - 1) & 1) * n;
        }
    }
    // warp 0: the storage rows and words of the fast path's 96 rows, issued
    // before anything waits (the fast path combines them once the tables
    // of panel j-1 are built)
    const int fend = min(R + 3 * 32, n);  // rows held in registers: [R, fend)
    int srw[3];
    uint64_t wv[3] = {0, 0, 0}, fv[3] = {0, 0, 0};
    if (warp == 0) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int p = R + 32 * u + lane;
            srw[u] = p < fend ? c.perm[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (srw[u] < 0) continue;
            wv[u] = Wj[(int64_t)srw[u] * kTileWords];
            if (pv.Fp) fv[u] = pv.Fp[(int64_t)srw[u] * pv.fstride];
        }
    }
    if (pv.Fp) {
        const PanelInfo *pp = panel_info(c, j - 1);
        if (tid < 64) {
            sh.T[tid] = pp->Zp[tid];
            sh.TI[tid] = tid < rp ? Wj[(int64_t)pp->prow[tid] * kTileWords] : 0;
        }
        panel_sync();
        for (int e = tid; e < 256; e += kPanelThreads) {
            const int g = e >> 4, x = e & 15;
            uint64_t a = 0, b = 0;
#pragma unroll
            for (int bit = 0; bit < 4; ++bit)
                if ((x >> bit) & 1) {
                    a ^= sh.T[4 * g + bit];
                    b ^= sh.TI[4 * g + bit];
                }
            sh.zt[e] = a;
            sh.ct[e] = b;
        }
        panel_sync();
    }

    if (warp != 0) {  // helpers: serve scan requests of warp 0
        for (;;) {
            bar_sync(1, kPanelThreads);
            const int req = sh.req;
            if (req == kReqDone) break;  // (to the end phase, with warp 0)
            scan_find(c, Wj, pv, sh, L);
            bar_sync(2, kPanelThreads);
        }
    }

    // ---------------------------------------------------------------- warp 0
    if (warp == 0) {
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
            sh.found_idx = INT_MAX;
            sh.orv = orv;
        }
        __syncwarp();
        bar_sync(1, kPanelThreads);
        scan_find(c, Wj, pv, sh, L);
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
                sh.prow[t] = psrow;
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
                raw[u] = panel_word(Wj, pv, sh, srow);
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
    // The common case: the pivots of the block come from the first 96 rows
    // (positions R..R+95), held in registers for the whole block (see
    // FastCols).  Every column is kept fully reduced by the pivots found so
    // far and a row's bits move with the row when it is exchanged, so slots
    // below the pivot slot are empty and the first qualifying row for bit k
    // is the lowest set bit of column k.  When more than 96 rows would be
    // needed the general loop below takes over.
    int k = 0;
    bool fast_complete = false;
    {
        const int nrows = fend - R;
        uint64_t raw[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) raw[u] = (srw[u] >= 0 && pv.Fp) ? wv[u] ^ prev_update(sh, fv[u]) : wv[u];
        GF2_TR(if (tr && lane == 0) {
            asm volatile("" ::"l"(raw[0] ^ raw[1] ^ raw[2]));  // stamp after the loads arrived
            tr[kTrPanelLoaded * kTraceMaxPanels + j] = trace_clock();
        })
        FastCols st;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            st.A[u] = transpose32((uint32_t)raw[u], lane);
            st.B[u] = transpose32((uint32_t)(raw[u] >> 32), lane);
            st.ID[u] = slot_index_bits(u, lane);
            sh.fraw[32 * u + lane] = raw[u];
            sh.fsrow[32 * u + lane] = srw[u];
        }
        st.EA = 0;
        st.EB = 0;
        st.k = 0;
        st.s = 0;
        const int smax = min(64, nrows);
        const bool more_rows = fend < n;
        bool leave = fast_phase<0>(st, nbits, smax, more_rows);
        if (!leave) leave = fast_phase<1>(st, nbits, smax, more_rows);
        __syncwarp();
        s = st.s;
        k = st.k;
        EA = st.EA;
        EB = st.EB;
        // the row now at each position: its original slot from the
        // identity bits, then its storage row and raw word
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            int q = 0;
#pragma unroll
            for (int b = 0; b < 7; ++b) q |= (int)((__shfl_sync(kFull, st.ID[u], b) >> lane) & 1) << b;
            const int p = 32 * u + lane;
            if (p < nrows) {
                const int srow = sh.fsrow[q];
                if (q != p) c.perm[R + p] = srow;
                if (p < s) {
                    sh.B[p] = sh.fraw[q];
                    sh.prow[p] = srow;
                    c.pivpanel[srow] = j;
                }
            }
        }
        // the bit of pivot t is the lowest set bit of E_t: E_t is zero at the
        // earlier pivot bits and at the bits that got no pivot before it
        {
            uint64_t e2[2] = {EA, EB};
            transpose64(e2, lane);  // e2[h] = E_{lane + 32h}
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int t = lane + 32 * hh;
                if (t < s) {
                    const int kt = __ffsll((long long)e2[hh]) - 1;
                    sh.pb[t] = kt;
                    sh.sidx[kt] = t;
                }
            }
        }
        __syncwarp();
        s_done = s;
        ib = R + s;
        fill = ib;  // the general loop starts from an empty window
        if (!leave) fast_complete = true;
    }

    if (!fast_complete) refill();
    // red(e_lane), red(e_lane+32) (the reduced unit rows) in registers: from
    // the pivots so far at the panel's first scan, then updated with every
    // pivot added (a new pivot reduces last, so red(e_p) takes its row when
    // it has the pivot's bit)
    uint64_t P0 = 0, P1 = 0;
    bool pred_ok = false;
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
                if (!pred_ok) {
                    publish_reduced_units();
                    P0 = sh.pred[lane];
                    P1 = sh.pred[lane + 32];
                    pred_ok = true;
                } else {
                    sh.pred[lane] = P0;
                    sh.pred[lane + 32] = P1;
                    __syncwarp();
                }
                // bit p: entry k of red(e_p)
                const uint64_t ck = (uint64_t)__ballot_sync(kFull, (P0 >> k) & 1) |
                                    ((uint64_t)__ballot_sync(kFull, (P1 >> k) & 1) << 32);
                // (the OR of the window's reduced rows seeds the scan's OR)
                const uint64_t wor = (uint64_t)__ballot_sync(kFull, (A & valid) != 0) |
                                     ((uint64_t)__ballot_sync(kFull, (B & valid) != 0) << 32);
                request(kReqFind, fill, ck, wor);
                const int q = sh.found;
                if (q != INT_MAX) {
                    // pivot outside the window; the row in the pivot slot
                    // moves there and leaves the window
                    const int psrow = c.perm[q];
                    const uint64_t v = c.zpos ? sh.found_raw : panel_word(Wj, pv, sh, psrow);
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
                    if ((P0 >> k) & 1) P0 ^= red;  // the new pivot's row E_s = red
                    if ((P1 >> k) & 1) P1 ^= red;
                    if (lane == 0) {
                        c.perm[ib] = psrow;
                        c.perm[q] = sh.slot_srow[hs];
                        if (c.zpos)  // the list entry of position q
                            list_put(c, L, sh.found_idx, q, sh.slot_raw[hs]);
                        c.pivpanel[psrow] = j;
                        sh.B[s] = v;
                        sh.prow[s] = psrow;
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
                // lowest bit above k set in some reduced remaining row: the
                // find scan went over every row behind the window and left
                // their OR (with the window's) in sh.orv.
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
        if (pred_ok) {  // (only after a scan in this panel)
            const uint64_t Es = (uint64_t)__ballot_sync(kFull, eA) | ((uint64_t)__ballot_sync(kFull, eB) << 32);
            if ((P0 >> k) & 1) P0 ^= Es;
            if ((P1 >> k) & 1) P1 ^= Es;
        }
        const uint32_t rec = (uint32_t)k | ((uint32_t)f << 8);
        recA = (lane == s) ? rec : recA;
        recB = (lane + 32 == s) ? rec : recB;
        ++ib;
        ++s;
        ++k;
    }
    replay();
    // E (rows) and U (columns: U = E at the pivot columns, unit upper
    // triangular; zero past s) into shared memory for the end phase
    {
        uint64_t e2[2] = {EA, EB};
        transpose64(e2, lane);
        sh.E[lane] = e2[0];
        sh.E[lane + 32] = e2[1];
        sh.Ucol[lane] = 0;
        sh.Ucol[lane + 32] = 0;
        __syncwarp();
        // column s' of U = column pb[s'] of E
        const int sa = sh.sidx[lane], sb = sh.sidx[lane + 32];
        if (sa >= 0) sh.Ucol[sa] = EA;
        if (sb >= 0) sh.Ucol[sb] = EB;
        if (lane == 0) sh.ns = s;
    }
    // release the helpers (they join the end phase)
    if (lane == 0) sh.req = kReqDone;
    __syncwarp();
    bar_sync(1, kPanelThreads);
    GF2_TR(if (tr && lane == 0) tr[kTrPanelLoop * kTraceMaxPanels + j] = trace_clock();)
    }  // warp 0

    panel_end_phase(c, j, R, pi, sh, tr);
}

}  // namespace
}  // namespace gf2
