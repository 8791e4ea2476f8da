// Device code of the decomposition's look-ahead and wide trailing updates
// (eq. (Aj) of the paper by the Method of Four Russians, Section 6), shared
// by the separate-launch kernels (csrc/k_update.cu) and the persistent
// decomposition kernel (csrc/k_factor.cu).  Every definition is internal to
// the translation unit that includes this file.  The counters of the
// op-counting build go to the including unit's g_update_ops.
//
// None of the data read here is read through the read-only (non-coherent)
// path: in the persistent kernel the look-ahead writes Y, the active lists
// and W while other CTAs of the same launch run, and they read those after
// an acquire on the launch's progress counters.
#pragma once
#include "m4rm_core.cuh"

namespace gf2 {
namespace {

// -------------------------------------------------------------------- look-ahead
// Look-ahead of panel j over the rows still active before it (ROWS per chunk):
//   d      = the row's word j with every panel < j applied (F[j%2]; W for j = 0)
//   y      = d Zp (the paper's Y = D Z; 0 for the pivot rows of panels <= j) -> Y[j % kRing]
//   lambda = d Comp -> the row's L multipliers of panel j
//   F[(j+1)%2] = word j+1 with panel j applied (W keeps word j+1 without it:
//            panel j+1 may be reading it meanwhile and adds the update itself)
//   W ^= y C on the words >= j+2 of the tile holding word j+2 and, when
//            panel j opens a pair of panels (whose wide update starts after
//            the tile holding word j+3), of that tile too
//   the compacted list of the rows that stay active (act[j % kRing]: a ring
//            of lists, so that no list is rewritten while an update that
//            reads it may run)
// and, in chunk 0, the pivot rows' L rows (T) and their echelon words on
// the same columns.  (The second panel of a pair gets the first panel's
// update on the tiles of the wide update inside that update, where its
// pivot rows are table rows.)
constexpr int kNextC = 4;
constexpr int kNextTiles = 2;   // tiles of W the look-ahead updates (at most)
constexpr int kNextSmemWords = kNextTiles * (Tabs<kNextC>::Words + 64 * kTileWords) + 16 * 16 * 2 + 16 * 16;

#ifdef GF2_COUNT_OPS
__device__ unsigned long long g_update_ops[kNumOps];  // the op-counting build's counters (per unit)
#endif

// One chunk of ROUNDS x ROWS list entries: the tables once, then ROUNDS
// rounds of ROWS entries (one per thread).
// smem: kNextSmemWords words; keep_row: ROWS ints; keep_warp: THREADS / 32 + 1 ints.
template <int THREADS, int ROWS, int ROUNDS = 1>
__device__ __forceinline__ void next_body(const DecompCtx &c, int j, int chunk, uint64_t *smem, int *keep_row,
                                          int *keep_warp)
{
    static_assert(THREADS == ROWS && THREADS >= 256, "one list entry per thread; 256 threads build the y tables");
    uint64_t *tab = smem;                                      // [tile][Tabs<4>::Words]
    uint64_t *crow = tab + kNextTiles * Tabs<kNextC>::Words;   // [tile][64 x kTileWords]
    uint64_t *zc = crow + kNextTiles * 64 * kTileWords;        // [g][x][y, lambda], 16 tables of 16 entries
    uint64_t *c1 = zc + 16 * 16 * 2;                           // [g][x]: y * (word j+1 of the pivot rows)
    const PanelInfo *pi = c.info + j;
    const int R = pi->R, r = pi->r;
    const int tid = threadIdx.x;
    const bool has_f = j + 1 < c.mu;
    const bool pair_first = c.pair && !(j & 1) && j + 1 < c.mu;
    const int ntiles_w = (c.mu + kTileWords - 1) / kTileWords;
    const int t0 = (j + 2) / kTileWords;  // first tile of the range
    const int nt = j + 2 >= c.mu ? 0 : min((j + 2 + (pair_first ? 1 : 0)) / kTileWords, ntiles_w - 1) - t0 + 1;
    const int q0 = t0 * kTileWords;
    const int lane = tid & 31, warp = tid >> 5;
    const int rs = lane / kLanesPerRow, wp = lane % kLanesPerRow, swp = rs & 3;
    const int col = q0 + 2 * wp;
    const bool live_hi = nt > 0 && r > 0 && col + 1 >= j + 2;  // word col+1 takes the update
    const bool live_lo = live_hi && col >= j + 2;                // and word col too
    const int wq = R >> 6, sh = R & 63;
    const bool two = sh + r > 64;
    // this CTA's rows: entries [rb, re) of the rows still active before
    // panel j (every storage row for j = 0)
    const int cnt = j == 0 ? c.n : c.nact[j - 1];
    const int32_t *lst = j == 0 ? nullptr : c.act + (int64_t)((j - 1) % kRing) * c.n;
    const int cbase = chunk * ROUNDS * ROWS;
    if (cbase >= cnt && chunk != 0) return;
    const uint64_t *Fj = c.F + (int64_t)(j & 1) * c.n;
    uint64_t *Fn = c.F + (int64_t)((j + 1) & 1) * c.n;
    constexpr int U = ROWS / (kRowsPerWarp * (THREADS / 32));  // row groups per warp
    const int ng = tables_used<kNextC>(r);
    GF2_OPS(unsigned long long n_upd = 0, n_y = 0, n_lk = 0, n_tab = 0;)
    for (int round = 0; round < ROUNDS; ++round) {
    const int rb = cbase + round * ROWS, re = min(cnt, rb + ROWS);
    if (round > 0 && rb >= re) break;

    // 1. every load of this thread's rows, issued before anything waits
    int rows[U];
    uint32_t active = 0;  // bit u: row u is not a pivot of panels <= j (and r > 0)
    uint32_t keepm = 0;   // bit u: row u is not a pivot of panels <= j
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int k = rb + (warp * U + u) * kRowsPerWarp + rs;
        rows[u] = k < re ? (lst ? lst[k] : k) : -1;
    }
    uint64_t d[U], w1[U];
    ulonglong2 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int row = rows[u];
        const bool in = row >= 0;
        const int64_t rr = in ? row : 0;
        const bool keep = in && c.pivpanel[row] > j;
        if (keep) keepm |= 1u << u;
        if (keep && r > 0) active |= 1u << u;
        if (wp == 0) keep_row[(warp * U + u) * kRowsPerWarp + rs] = keep ? row : -1;
        d[u] = !in ? 0 : (j == 0 ? c.W[widx(c, rr, 0)] : Fj[rr]);
        w1[u] = (in && has_f && wp == 0) ? c.W[widx(c, rr, j + 1)] : 0;
        a[u] = (in && live_hi) ? *reinterpret_cast<const ulonglong2 *>(c.W + widx(c, rr, col)) : make_ulonglong2(0, 0);
    }
    // 2. (once) tables of (Zp, Comp) for y and lambda, of word j+1 of the
    // pivot rows, and of C for the tiles
    if (round == 0) {
    if (r > 0) {
        if (tid < 256) {  // 16 tables of 16 entries
        const int g = tid >> 4, x = tid & 15;
        uint64_t y = 0, l = 0, v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((x >> b) & 1) {
                const int s2 = 4 * g + b;
                y ^= pi->Zp[s2];
                l ^= pi->Comp[s2];
                if (has_f && s2 < r) v ^= c.W[widx(c, pi->prow[s2], j + 1)];
            }
        zc[2 * tid] = y;
        zc[2 * tid + 1] = l;
        c1[tid] = v;
        }
        for (int tt = 0; tt < nt; ++tt)
            load_pivot_rows<THREADS>(c, pi->prow, r, q0 + tt * kTileWords, crow + tt * 64 * kTileWords);
    }
    __syncthreads();
    if (r > 0)
        for (int tt = 0; tt < nt; ++tt)
            build_tables<kNextC, THREADS>(tab + tt * Tabs<kNextC>::Words, crow + tt * 64 * kTileWords);
    GF2_OPS(if (tid == 0 && r > 0) {
                constexpr int E4 = Tabs<kNextC>::X - 1;
                n_tab += has_f ? 16 * E4 : 0;  // the tables of word j+1 (c1)
                for (int tt = 0; tt < nt; ++tt)
                    n_tab += (unsigned long long)Tabs<kNextC>::K * E4 * live_words(q0 + tt * kTileWords, c.mu);
            })
    } else {
        __syncthreads();  // this round's keep_row entries are written
    }
    // the rows that stay active, appended to the list of panel j in list order
    const int kept_row = keep_row[tid];
    const unsigned kept_mask = __ballot_sync(0xffffffffu, kept_row >= 0);
    if (lane == 0) keep_warp[warp] = __popc(kept_mask);
    __syncthreads();
    if (tid == 0) {
        int total = 0;
        for (int w = 0; w < THREADS / 32; ++w) {
            const int t = keep_warp[w];
            keep_warp[w] = total;
            total += t;
        }
        keep_warp[THREADS / 32] = total ? atomicAdd(c.nact + j, total) : 0;
    }
    __syncthreads();
    if (kept_row >= 0) {
        const int pos = keep_warp[THREADS / 32] + keep_warp[warp] + __popc(kept_mask & ((1u << lane) - 1));
        c.act[(int64_t)(j % kRing) * c.n + pos] = kept_row;
    }

    // 3. compute and store
    const ulonglong2 *zc2 = reinterpret_cast<const ulonglong2 *>(zc);
    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(tab);
    uint64_t *Ynext = c.Y + (int64_t)(j % kRing) * c.n;
    uint64_t yv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int row = rows[u];
        yv[u] = 0;
        if (row < 0) continue;
        uint64_t y = 0, l = 0;
        if ((active >> u) & 1) {
#pragma unroll
            for (int g = 0; g < 16; ++g) {
                const ulonglong2 t = zc2[g * 16 + (int)((d[u] >> (4 * g)) & 15)];
                y ^= t.x;
                l ^= t.y;
            }
        }
        yv[u] = y;
        GF2_OPS(if (wp == 0 && ((active >> u) & 1)) n_y += 1;)
        if (wp == 0) {
            Ynext[row] = y;
            if (c.Lint && l) {  // this panel's bits of the L row: disjoint from every other panel's
                unsigned long long *Lr = reinterpret_cast<unsigned long long *>(c.Lint + (int64_t)row * c.ldl);
                atomicOr(Lr + wq, (unsigned long long)(l << sh));
                if (two) atomicOr(Lr + wq + 1, (unsigned long long)(l >> (64 - sh)));
            }
            if (has_f) {
                uint64_t f = w1[u];
                if (y) {
#pragma unroll
                    for (int g = 0; g < 16; ++g) f ^= c1[g * 16 + (int)((y >> (4 * g)) & 15)];
                    GF2_OPS(n_upd += 1; n_lk += 16;)
                }
                Fn[row] = f;
            }
        }
        if (live_hi && y) {
            lookup<kNextC>(tab2, y, wp, swp, ng, a[u]);
            GF2_OPS(const int lw = (live_lo && col < c.mu) + (col + 1 < c.mu); n_upd += lw;
                    n_lk += (unsigned long long)ng * lw;)
            uint64_t *dst = c.W + widx(c, row, col);
            if (live_lo) *reinterpret_cast<ulonglong2 *>(dst) = a[u];
            else dst[1] = a[u].y;
        }
    }
    // After a rank-deficient panel (the rank may be used up): whether any row
    // that stays active has a nonzero word j+2 now (every panel <= j
    // applied).  orw[j+2] bit 1: computed (by the first chunk), bit 0: some
    // nonzero word seen.  With no pivot in panel j+1 either, "computed and
    // none" tells panel j+2 that its block has no pivot.
    if (c.orw && j + 2 < c.mu && r < 64) {
        uint64_t o = 0;
        if (wp == ((j + 2) & 3) >> 1)  // this lane's word pair holds word j+2
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!((keepm >> u) & 1)) continue;
                o |= live_hi ? (((j + 2) & 1) ? a[u].y : a[u].x) : c.W[widx(c, rows[u], j + 2)];
            }
        const int any = __syncthreads_or(o != 0);
        if (tid == 0) {  // one atomic per CTA at most
            const int v = (any ? 1 : 0) | ((chunk == 0 && round == 0) ? 2 : 0);
            if (v && (*reinterpret_cast<volatile int32_t *>(c.orw + j + 2) & v) != v) atomicOr(c.orw + j + 2, v);
        }
    }
    // the second tile of a pair's range: every word of it
    if (nt > 1 && r > 0) {
        const int col2 = q0 + kTileWords + 2 * wp;
        const ulonglong2 *tab2b = reinterpret_cast<const ulonglong2 *>(tab + Tabs<kNextC>::Words);
        ulonglong2 b2[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            b2[u] = (rows[u] >= 0 && yv[u]) ? *reinterpret_cast<const ulonglong2 *>(c.W + widx(c, rows[u], col2))
                                            : make_ulonglong2(0, 0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (rows[u] < 0 || !yv[u]) continue;
            lookup<kNextC>(tab2b, yv[u], wp, swp, ng, b2[u]);
            *reinterpret_cast<ulonglong2 *>(c.W + widx(c, rows[u], col2)) = b2[u];
            GF2_OPS(const int lw = (col2 < c.mu) + (col2 + 1 < c.mu); n_upd += lw;
                    n_lk += (unsigned long long)ng * lw;)
        }
    }
    }  // rounds
    GF2_OPS(add_ops(g_update_ops, kOpUpdates, n_upd); add_ops(g_update_ops, kOpYRows, n_y);
            add_ops(g_update_ops, kOpLookups4, n_lk); add_ops(g_update_ops, kOpTable4, n_tab);)

    if (chunk == 0 && r > 0) {
        // the pivot rows: their L rows (T) and echelon words j and j+1
        for (int t = tid; t < r; t += THREADS) {
            const int srow = pi->prow[t];
            if (c.Lint) {
                const uint64_t l = pi->T[t];
                unsigned long long *Lr = reinterpret_cast<unsigned long long *>(c.Lint + (int64_t)srow * c.ldl);
                atomicOr(Lr + wq, (unsigned long long)(l << sh));
                if (two) atomicOr(Lr + wq + 1, (unsigned long long)(l >> (64 - sh)));
            }
            if (c.Eint) {
                uint64_t *Er = c.Eint + (int64_t)(R + t) * c.lde;
                Er[j] = pi->Erow[t];
                if (has_f) {
                    const uint64_t ti = pi->Tinv[t];
                    uint64_t e = 0;
#pragma unroll
                    for (int g = 0; g < 16; ++g) e ^= c1[g * 16 + (int)((ti >> (4 * g)) & 15)];
                    Er[j + 1] = e;
                }
            }
        }
        if (c.Eint)
            for (int tt = 0; tt < nt; ++tt)
                echelon_rows<kNextC, THREADS>(c, pi, R, r, q0 + tt * kTileWords, j + 2, ng,
                                                   tab + tt * Tabs<kNextC>::Words);
    }
}

// -------------------------------------------------------------------- wide update
// The wide update of panel j (NP = 1), or of the pair of panels j, j+1 at
// once (NP = 2, the wide-panel form of Section 5: w = 128 columns, one read
// and one write of every trailing word per pair): W ^= y_j C_j (+ y_j+1 C_j+1)
// on the tiles after the look-ahead range, over the rows that are not pivots
// of panels <= j + NP - 1.  For a pair the tables of C_j+1 are built from the
// second panel's pivot rows AFTER the first panel's update (the look-ahead
// kernel of panel j+1 applied it), so the two products simply add.
// A unit of work is a column tile and a range of entries of the active list;
// rest_prepare builds the tile's tables (once per tile and CTA), rest_pass
// updates the rows of one range.
constexpr int kRestChunk = 256;  // list entries per work item
constexpr int kRestPad = 4;      // bank skew of the staged pivot rows (build_tables)

template <int C, int NP>
constexpr int rest_smem_bytes()
{
    return (NP * Tabs<C>::Words + NP * crow_words<C, kRestPad>()) * 8;
}

struct UpdOps {  // the op-counting build's tallies of one thread
    unsigned long long upd = 0, lk = 0, tab = 0;
};

// The pivot rows of panel j (and j+1) on `tile`, their tables in smem, and
// for a pair panel j's update of panel j+1's pivot rows: they are not on the
// active list, so they take it here (with panel j's tables) before panel
// j+1's tables are built from them (their words in W are not read again: the
// echelon rows come from these tables).  first: the CTA that takes the
// tile's first chunk also writes the pivot rows' echelon words of the tile.
// rest_prepare's loads that do not read W, the same for every tile (entry e
// as below; row -1 past the panel's pivots): the head launches make them
// before their grid-dependency wait.
template <int NP, int THREADS>
struct RestPre {
    static constexpr int NE = NP * 64 * kTileWords;
    static constexpr int RPT = (NE + THREADS - 1) / THREADS;
    int row[RPT];
    uint64_t yv[RPT];
};

template <int NP, int THREADS>
__device__ __forceinline__ void rest_preload(const DecompCtx &c, int j, int r0, int r1, RestPre<NP, THREADS> &p)
{
    const PanelInfo *pi0 = c.info + j;
    const PanelInfo *pi1 = c.info + j + NP - 1;
    const uint64_t *Y0 = c.Y + (int64_t)(j % kRing) * c.n;
#pragma unroll
    for (int k = 0; k < RestPre<NP, THREADS>::RPT; ++k) {
        const int e = threadIdx.x + k * THREADS, t = (e & 255) / kTileWords;
        const bool p1 = e >= 64 * kTileWords;
        p.row[k] = -1;
        p.yv[k] = 0;
        if (e < RestPre<NP, THREADS>::NE && t < (p1 ? r1 : r0)) {
            p.row[k] = (p1 ? pi1 : pi0)->prow[t];
            if (p1) p.yv[k] = Y0[p.row[k]];
        }
    }
}

// PRE: the loads of rest_preload are in pre.
template <int C, int NP, int THREADS, bool PRE = false>
__device__ __forceinline__ void rest_prepare(const DecompCtx &c, int j, int tile, bool first, uint64_t *smem,
                                             UpdOps &ops, const RestPre<NP, THREADS> &pre = RestPre<NP, THREADS>{})
{
    constexpr int K = Tabs<C>::K;
    uint64_t *tab = smem;                          // [NP * K tables][X][kTileWords]
    uint64_t *crow = smem + NP * Tabs<C>::Words;   // [NP][crow_words]: 64 x kTileWords, skewed
    uint64_t *crow1 = crow + crow_words<C, kRestPad>();
    const PanelInfo *pi0 = c.info + j;
    const PanelInfo *pi1 = c.info + j + NP - 1;
    const int r0 = pi0->r, r1 = NP == 2 ? pi1->r : 0;
    const int ng0 = tables_used<C>(r0), ng1 = NP == 2 ? tables_used<C>(r1) : 0;
    const int tid = threadIdx.x;
    const int q0 = tile * kTileWords;
    const uint64_t *Y0 = c.Y + (int64_t)(j % kRing) * c.n;
    (void)ops;
    if constexpr (PRE) {
        // one round of loads, from rest_preload's storage rows: the pivot
        // rows' tile words of both panels (entry e: panel e / 256, row
        // (e % 256) / kTileWords, word e % kTileWords)
        constexpr int NE = RestPre<NP, THREADS>::NE, RPT = RestPre<NP, THREADS>::RPT;
        uint64_t v[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            v[k] = pre.row[k] >= 0 ? c.W[widx(c, pre.row[k], q0 + (tid + k * THREADS) % kTileWords)] : 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int e = tid + k * THREADS, idx = e & 255, t = idx / kTileWords;
            if (e < NE) (e >= 64 * kTileWords ? crow1 : crow)[idx + kRestPad * (t / C)] = v[k];
        }
        __syncthreads();
        build_tables<C, THREADS, kRestPad>(tab, crow);
        GF2_OPS(if (tid == 0) ops.tab += (unsigned long long)NP * K * (Tabs<C>::X - 1) * live_words(q0, c.mu);)
        if (NP == 2) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int e = tid + k * THREADS, idx = e & 255;
                if (e < 64 * kTileWords || e >= NE || !pre.yv[k]) continue;
                const uint64_t y = pre.yv[k];
                uint64_t acc = 0;
                for (int g = 0; g < ng0; ++g)
                    acc ^= tab[tab_entry<C>(g, (int)((y >> (C * g)) & (Tabs<C>::X - 1))) * kTileWords + idx % kTileWords];
                crow1[idx + kRestPad * (idx / kTileWords / C)] ^= acc;
                GF2_OPS(if (first && q0 + idx % kTileWords < c.mu) { ops.upd += 1; ops.lk += ng0; })
            }
            __syncthreads();
            build_tables<C, THREADS, kRestPad>(tab, crow1, K);
        }
    } else {
        __syncthreads();
        load_pivot_rows<THREADS, C, kRestPad>(c, pi0->prow, r0, q0, crow);
        if (NP == 2) load_pivot_rows<THREADS, C, kRestPad>(c, pi1->prow, r1, q0, crow1);
        __syncthreads();
        build_tables<C, THREADS, kRestPad>(tab, crow);
        GF2_OPS(if (tid == 0) ops.tab += (unsigned long long)NP * K * (Tabs<C>::X - 1) * live_words(q0, c.mu);)
        if (NP == 2) {
            __syncthreads();
            for (int idx = tid; idx < r1 * kTileWords; idx += THREADS) {
                const uint64_t y = Y0[pi1->prow[idx / kTileWords]];
                if (!y) continue;
                uint64_t acc = 0;
                for (int g = 0; g < ng0; ++g)
                    acc ^= tab[tab_entry<C>(g, (int)((y >> (C * g)) & (Tabs<C>::X - 1))) * kTileWords + idx % kTileWords];
                crow1[idx + kRestPad * (idx / kTileWords / C)] ^= acc;
                // (every CTA that shares the tile redoes this; counted once, by the one with chunk 0)
                GF2_OPS(if (first && q0 + idx % kTileWords < c.mu) { ops.upd += 1; ops.lk += ng0; })
            }
            __syncthreads();
            build_tables<C, THREADS, kRestPad>(tab, crow1, K);
        }
    }
    __syncthreads();
    if (c.Eint && first) {
        echelon_rows<C, THREADS>(c, pi0, pi0->R, r0, q0, 0, ng0, tab);
        if (NP == 2) echelon_rows<C, THREADS>(c, pi1, pi1->R, r1, q0, 0, ng1, tab, K);
    }
}

// -------------------------------------------------------------------- lookups
// The 8-bit table lookups of the wide update with their addresses reduced
// to two integer operations.  At step g a lane reads table g ^ swp (swp = its
// row slot & 3: the four rows of a quarter-warp read the four 32-byte
// quarters of the bank space), entry x = byte g ^ swp of its multiplier y.
// Entry (t, x) of the [quad][x][quarter][kTileWords] layout is at byte
// ((t >> 2) * 256 + x) * 128 + (t & 3) * 32 of the tables, the lane's word
// pair 16 bytes further for wp = 1.  So with q = g & 3:
//   x    = the low byte of __byte_perm(half g >> 2 of y, 0, sel[q]),
//          sel[q] = 0x4440 | (q ^ swp)
//   addr = base[q] + 128 x + (g >> 2) * 32768
//          base[q] = tables + (q ^ swp) * 32 + wp * 16.
struct Lk8 {
    uint32_t base[4];  // shared-window byte addresses
    uint32_t sel[4];
};

__device__ __forceinline__ Lk8 lk8_lane(const uint64_t *tab, int swp, int wp)
{
    Lk8 l;
    const uint32_t t = (uint32_t)__cvta_generic_to_shared(tab);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        l.base[q] = t + (uint32_t)(((q ^ swp) << 5) + (wp << 4));
        l.sel[q] = 0x4440u | (uint32_t)(q ^ swp);
    }
    return l;
}

// acc[u] ^= y[u] * C for the NG tables from table G0 (compile time; G0 a
// multiple of 8: tables G0.. belong to one panel and take bytes 0.. of y).
template <int G0, int NG, int U>
__device__ __forceinline__ void lk8_rows(const Lk8 &l, const uint64_t (&y)[U], ulonglong2 (&acc)[U])
{
    static_assert(G0 % 8 == 0 && (NG == 4 || NG == 8), "whole quads of one panel's tables");
#pragma unroll
    for (int g = 0; g < NG; ++g) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t h = g < 4 ? (uint32_t)y[u] : (uint32_t)(y[u] >> 32);
            const uint32_t x = __byte_perm(h, 0u, l.sel[g & 3]);
            const uint32_t addr = l.base[g & 3] + (x << 7) + (uint32_t)(((G0 + g) >> 2) * 256 * 128);
            uint64_t tx, ty;
            asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(tx), "=l"(ty) : "r"(addr));
            acc[u].x ^= tx;
            acc[u].y ^= ty;
        }
    }
}

// One iteration of the wide update for U row groups: W ^= y0 C_j (+ y1
// C_j+1) on this lane's word pair of the rows row[u] (-1: none; a row with
// y0 = y1 = 0 is neither read nor written).  The row words, like the
// multipliers and the list entries, are cached in L2 only (.cg): nothing
// re-reads them from L1, and an L1 fill would take cycles of the data
// pipe that the table lookups are bound by.
template <int C, int U, int NP>
__device__ __forceinline__ void rest_rows(const Lk8 &lk, const ulonglong2 *tab2, int swp, int wp, int ng0, int ng1,
                                          const uint64_t (&y0)[U], const uint64_t (&y1)[U], const int (&row)[U],
                                          uint64_t *Wt)
{
    constexpr int K = Tabs<C>::K;
    ulonglong2 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        a[u] = make_ulonglong2(0, 0);
        if (y0[u] | y1[u]) a[u] = __ldcg(reinterpret_cast<const ulonglong2 *>(Wt + (int64_t)row[u] * kTileWords));
    }
    if (C == 8) {
        if (ng0 == 8) lk8_rows<0, 8, U>(lk, y0, a);
        else if (ng0 == 4) lk8_rows<0, 4, U>(lk, y0, a);
        if (NP == 2) {
            if (ng1 == 8) lk8_rows<8, 8, U>(lk, y1, a);
            else if (ng1 == 4) lk8_rows<8, 4, U>(lk, y1, a);
        }
    } else {
        for (int g = 0; g < ng0; ++g) {
            const int gg = g ^ swp;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = (int)((y0[u] >> (C * gg)) & (Tabs<C>::X - 1));
                const ulonglong2 t = tab2[tab_entry<C>(gg, x) * (kTileWords / 2) + wp];
                a[u].x ^= t.x;
                a[u].y ^= t.y;
            }
        }
        if (NP == 2) {
            for (int g = 0; g < ng1; ++g) {
                const int gg = g ^ swp;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int x = (int)((y1[u] >> (C * gg)) & (Tabs<C>::X - 1));
                    const ulonglong2 t = tab2[tab_entry<C>(K + gg, x) * (kTileWords / 2) + wp];
                    a[u].x ^= t.x;
                    a[u].y ^= t.y;
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (y0[u] | y1[u]) __stcg(reinterpret_cast<ulonglong2 *>(Wt + (int64_t)row[u] * kTileWords), a[u]);
}

// W ^= y_j C_j (+ y_j+1 C_j+1) on `tile` for the list entries [rb, re), with
// the tables rest_prepare built; U row groups of 16 rows per warp and
// iteration, y and the next rows' indices prefetched one iteration ahead.
// The loads of rest_pass's first iteration (list entries, then
// multipliers; no W) for the warp whose rows start at base: row -1 past re.
template <int U>
struct RestIter {
    int row[U];
    uint64_t y0[U], y1[U];
};

template <int U, int NP>
__device__ __forceinline__ void rest_iter_load(const DecompCtx &c, int j, int base, int re, RestIter<U> &it)
{
    const int32_t *act = c.act + (int64_t)((j + NP - 1) % kRing) * c.n;
    const uint64_t *Y0 = c.Y + (int64_t)(j % kRing) * c.n;
    const uint64_t *Y1 = c.Y + (int64_t)((j + 1) % kRing) * c.n;
    const int rs = (threadIdx.x & 31) / kLanesPerRow;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int k = base + u * kRowsPerWarp + rs;
        it.row[u] = k < re ? __ldcg(act + k) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        it.y0[u] = it.row[u] >= 0 ? __ldcg(Y0 + it.row[u]) : 0;
        it.y1[u] = (NP == 2 && it.row[u] >= 0) ? __ldcg(Y1 + it.row[u]) : 0;
    }
}

// PRE: the first iteration's loads are in first (rest_iter_load with base =
// rb + warp * kRowsPerWarp * U).
template <int C, int U, int NP, int THREADS, bool PRE = false>
__device__ __forceinline__ void rest_pass(const DecompCtx &c, int j, int tile, int rb, int re, const uint64_t *smem,
                                          UpdOps &ops, const RestIter<U> &first = RestIter<U>{})
{
    constexpr int K = Tabs<C>::K;
    const PanelInfo *pi0 = c.info + j;
    const PanelInfo *pi1 = c.info + j + NP - 1;
    const int r0 = pi0->r, r1 = NP == 2 ? pi1->r : 0;
    const int ng0 = tables_used<C>(r0), ng1 = NP == 2 ? tables_used<C>(r1) : 0;
    const int jl = j + NP - 1;
    const int32_t *act = c.act + (int64_t)(jl % kRing) * c.n;
    const uint64_t *Y0 = c.Y + (int64_t)(j % kRing) * c.n;
    const uint64_t *Y1 = c.Y + (int64_t)((j + 1) % kRing) * c.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = lane / kLanesPerRow, wp = lane % kLanesPerRow, swp = rs & 3;
    constexpr int NW = THREADS / 32;
    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(smem);
    const Lk8 lk = lk8_lane(smem, swp, wp);
    const int q0 = tile * kTileWords;
    (void)ops;
    (void)q0;
    (void)K;
    uint64_t *Wt = c.W + (int64_t)tile * c.tstride + 2 * wp;  // this lane's word pair of the tile
    constexpr int STEP = kRowsPerWarp * U * NW;
    uint64_t yn0[U], yn1[U];
    int rown[U];
    if constexpr (PRE) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            rown[u] = first.row[u];
            yn0[u] = first.y0[u];
            yn1[u] = first.y1[u];
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = rb + warp * kRowsPerWarp * U + u * kRowsPerWarp + rs;
            rown[u] = k < re ? __ldcg(act + k) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            yn0[u] = rown[u] >= 0 ? __ldcg(Y0 + rown[u]) : 0;
            yn1[u] = (NP == 2 && rown[u] >= 0) ? __ldcg(Y1 + rown[u]) : 0;
        }
    }
    for (int base = rb + warp * kRowsPerWarp * U; base < re; base += STEP) {
        uint64_t y0[U], y1[U];
        int row[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            y0[u] = yn0[u];
            y1[u] = yn1[u];
            row[u] = rown[u];
            const int k = base + STEP + u * kRowsPerWarp + rs;
            rown[u] = k < re ? __ldcg(act + k) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            yn0[u] = rown[u] >= 0 ? __ldcg(Y0 + rown[u]) : 0;
            yn1[u] = (NP == 2 && rown[u] >= 0) ? __ldcg(Y1 + rown[u]) : 0;
        }
        rest_rows<C, U, NP>(lk, tab2, swp, wp, ng0, ng1, y0, y1, row, Wt);
        GF2_OPS(const int lw = (q0 + 2 * wp < c.mu) + (q0 + 2 * wp + 1 < c.mu);
                for (int u = 0; u < U; ++u) {
                    if (y0[u]) { ops.upd += lw; ops.lk += (unsigned long long)ng0 * lw; }
                    if (NP == 2 && y1[u]) { ops.upd += lw; ops.lk += (unsigned long long)ng1 * lw; }
                })
    }
}

// rest_pass that can stop between iterations and resume: warp w starts at
// its iteration kw[w] (iterations of STEP list entries from rb) and, before
// each iteration, leaves if *stop is set.  Thread 0 sets *stop itself once
// the word it polls here reaches poll_val (poll: the condition its caller
// waits for; null: never).  On return kw[w] = the first iteration warp w
// has not done; the result is 1 when every warp has finished [rb, re).
template <int C, int U, int NP, int THREADS>
__device__ __forceinline__ int rest_pass_from(const DecompCtx &c, int j, int tile, int rb, int re,
                                              const uint64_t *smem, UpdOps &ops, int *kw, volatile int *stop,
                                              const int32_t *poll, int poll_val)
{
    constexpr int K = Tabs<C>::K;
    const PanelInfo *pi0 = c.info + j;
    const PanelInfo *pi1 = c.info + j + NP - 1;
    const int r0 = pi0->r, r1 = NP == 2 ? pi1->r : 0;
    const int ng0 = tables_used<C>(r0), ng1 = NP == 2 ? tables_used<C>(r1) : 0;
    const int jl = j + NP - 1;
    const int32_t *act = c.act + (int64_t)(jl % kRing) * c.n;
    const uint64_t *Y0 = c.Y + (int64_t)(j % kRing) * c.n;
    const uint64_t *Y1 = c.Y + (int64_t)((j + 1) % kRing) * c.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = lane / kLanesPerRow, wp = lane % kLanesPerRow, swp = rs & 3;
    constexpr int NW = THREADS / 32;
    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(smem);
    const Lk8 lk = lk8_lane(smem, swp, wp);
    const int q0 = tile * kTileWords;
    (void)ops;
    (void)q0;
    (void)K;
    uint64_t *Wt = c.W + (int64_t)tile * c.tstride + 2 * wp;
    constexpr int STEP = kRowsPerWarp * U * NW;
    int k = kw[warp];
    int base = rb + warp * kRowsPerWarp * U + k * STEP;
    uint64_t yn0[U], yn1[U];
    int rown[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int e = base + u * kRowsPerWarp + rs;
        rown[u] = e < re ? __ldcg(act + e) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        yn0[u] = rown[u] >= 0 ? __ldcg(Y0 + rown[u]) : 0;
        yn1[u] = (NP == 2 && rown[u] >= 0) ? __ldcg(Y1 + rown[u]) : 0;
    }
    int polled = -1;  // thread 0: the polled word, read one iteration ahead
    for (; base < re; base += STEP, ++k) {
        if (tid == 0 && poll) {
            if (polled >= poll_val) *stop = 1;
            int v;
            asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(poll) : "memory");
            polled = v;
        }
        if (__shfl_sync(0xffffffffu, lane == 0 ? *stop : 0, 0)) break;
        uint64_t y0[U], y1[U];
        int row[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            y0[u] = yn0[u];
            y1[u] = yn1[u];
            row[u] = rown[u];
            const int e = base + STEP + u * kRowsPerWarp + rs;
            rown[u] = e < re ? __ldcg(act + e) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            yn0[u] = rown[u] >= 0 ? __ldcg(Y0 + rown[u]) : 0;
            yn1[u] = (NP == 2 && rown[u] >= 0) ? __ldcg(Y1 + rown[u]) : 0;
        }
        rest_rows<C, U, NP>(lk, tab2, swp, wp, ng0, ng1, y0, y1, row, Wt);
        GF2_OPS(const int lw = (q0 + 2 * wp < c.mu) + (q0 + 2 * wp + 1 < c.mu);
                for (int u = 0; u < U; ++u) {
                    if (y0[u]) { ops.upd += lw; ops.lk += (unsigned long long)ng0 * lw; }
                    if (NP == 2 && y1[u]) { ops.upd += lw; ops.lk += (unsigned long long)ng1 * lw; }
                })
    }
    if (lane == 0) kw[warp] = k;
    return __syncthreads_and(base >= re);
}

}  // namespace
}  // namespace gf2
