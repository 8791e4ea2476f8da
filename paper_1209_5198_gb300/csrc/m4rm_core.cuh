// Four Russians (M4RM, Section 6 of the paper) building blocks over one
// column tile of kTileWords words: tables of the 64 pivot rows C of a panel
// in shared memory, lookups, the pivot rows' loads and echelon words.  Shared
// by the decomposition's update kernels and the batched decomposition; every
// definition is internal to the translation unit that includes this file.
//
// Shared-memory layout of the tables: [table quad][x][quarter][kTileWords
// words]; the four rows of a quarter-warp (one 128-bit shared-memory phase)
// read tables g, g^1, g^2, g^3, which live in the four 32-byte quarters of the
// bank space, so lookups are conflict-free for any multiplier.
#pragma once
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

template <int C>
struct Tabs {
    static constexpr int K = 64 / C;                 // tables
    static constexpr int X = 1 << C;                 // entries per table
    static constexpr int Words = K * X * kTileWords; // shared-memory words
};

// index (in tile-word entries) of entry x of table g
template <int C>
__device__ __forceinline__ int tab_entry(int g, int x)
{
    return ((((g >> 2) << C) + x) << 2) | (g & 3);
}

// tables in use for r pivot rows: a multiple of 4 (whole quads; unused ones are zero)
template <int C>
__device__ __forceinline__ int tables_used(int r)
{
    return ((r + C - 1) / C + 3) & ~3;
}

// Tables g0.. of the 64 tile rows in crow (rows beyond r are zero): row t,
// word w at crow[t * kTileWords + w + PAD * (t / C)] (PAD = 4 skews the C-row
// groups across the banks, so that a warp's reads of one row of each group
// do not collide).
// Thread -> (word w, table g, sub-range of x); each sub-range walks its low
// bits in Gray order, one XOR per entry.
template <int C, int T, int PAD = 0>
__device__ __forceinline__ void build_tables(uint64_t *tab, const uint64_t *crow, int g0 = 0)
{
    constexpr int K = Tabs<C>::K, X = Tabs<C>::X;
    constexpr int PAIRS = K * kTileWords;
    static_assert(T % PAIRS == 0, "thread count must cover every (table, word)");
    constexpr int SUBS = T / PAIRS;
    static_assert(SUBS <= X, "too many threads for this table size");
    constexpr int Q = X / SUBS;
    constexpr int LQ = (Q >= 256) ? 8 : (Q >= 128) ? 7 : (Q >= 64) ? 6 : (Q >= 32) ? 5 : (Q >= 16) ? 4 : (Q >= 8) ? 3 : (Q >= 4) ? 2 : (Q >= 2) ? 1 : 0;
    const int tid = threadIdx.x;
    const int w = tid % kTileWords, g = (tid / kTileWords) % K, sub = tid / (kTileWords * K);
    uint64_t cb[C];
#pragma unroll
    for (int b = 0; b < C; ++b) cb[b] = crow[(C * g + b) * kTileWords + w + PAD * g];
    const int x0 = sub * Q;
    uint64_t v = 0;
#pragma unroll
    for (int b = LQ; b < C; ++b)
        if ((x0 >> b) & 1) v ^= cb[b];
    tab[tab_entry<C>(g0 + g, x0) * kTileWords + w] = v;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : (i & 16) ? 4 : (i & 32) ? 5 : (i & 64) ? 6 : 7;
        v ^= cb[b];
        tab[tab_entry<C>(g0 + g, x0 + (i ^ (i >> 1))) * kTileWords + w] = v;
    }
}

// a ^= y * C for this lane's word pair (tables of C in tab2).
template <int C>
__device__ __forceinline__ void lookup(const ulonglong2 *tab2, uint64_t y, int wp, int swp, int ng, ulonglong2 &a)
{
    constexpr int X = Tabs<C>::X;
    for (int g = 0; g < ng; ++g) {
        const int gg = g ^ swp;
        const int x = (int)((y >> (C * gg)) & (X - 1));
        const ulonglong2 t = tab2[tab_entry<C>(gg, x) * (kTileWords / 2) + wp];
        a.x ^= t.x;
        a.y ^= t.y;
    }
}

#ifdef GF2_COUNT_OPS
// adds a thread's tally to a counter of the op-counting build
__device__ __forceinline__ void add_ops(unsigned long long *ops, int kind, unsigned long long v)
{
    if (v) atomicAdd(ops + kind, v);
}

// words of the tile at word q0 before the last column block's end (mu words)
__device__ __forceinline__ int live_words(int q0, int mu)
{
    return max(0, min(kTileWords, mu - q0));
}
#endif

// Words of a staged block of 64 tile rows with the bank skew of build_tables
// (PAD words after every C rows).
template <int C, int PAD>
constexpr int crow_words()
{
    return 64 * kTileWords + PAD * (64 / C);
}

// Loads the C rows of panel j (the pivot rows, by their storage rows prow)
// for the tile starting at word q0 (zero beyond r), in build_tables' layout.
template <int T, int C = 8, int PAD = 0>
__device__ __forceinline__ void load_pivot_rows(const DecompCtx &c, const int32_t *prow, int r, int q0, uint64_t *crow)
{
    for (int idx = threadIdx.x; idx < 64 * kTileWords; idx += T) {
        const int t = idx / kTileWords, w = idx % kTileWords;
        uint64_t v = 0;
        if (t < r) v = c.W[widx(c, prow[t], q0 + w)];
        crow[idx + PAD * (t / C)] = v;
    }
}

// Echelon rows of the panel's pivots on one tile: E_s = Tinv[s] * C (the
// panel's tables are g0..g0+ng-1).
template <int C, int T>
__device__ __forceinline__ void echelon_rows(const DecompCtx &c, const PanelInfo *pi, int R, int r, int q0,
                                             int live_from, int ng, const uint64_t *tab, int g0 = 0)
{
    for (int idx = threadIdx.x; idx < r * kTileWords; idx += T) {
        const int t = idx / kTileWords, w = idx % kTileWords;
        const int q = q0 + w;
        if (q < live_from || q >= c.mu) continue;
        const uint64_t ym = pi->Tinv[t];
        uint64_t acc = 0;
        for (int g = 0; g < ng; ++g)
            acc ^= tab[tab_entry<C>(g0 + g, (int)((ym >> (C * g)) & (Tabs<C>::X - 1))) * kTileWords + w];
        c.Eint[(int64_t)(R + t) * c.lde + q] = acc;
    }
}

}  // namespace
}  // namespace gf2
