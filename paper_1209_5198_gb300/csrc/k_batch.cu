// Batched decomposition: many independent matrices (the batched workload of
// the paper's use cases: thousands of small and medium systems), P*A = L*E for
// each, in ONE persistent launch.  One CTA of four warps factors one matrix at
// a time and takes the next from a shared counter (matrices in decreasing
// order of work), so large and small matrices balance across the SMs.
//
// Per matrix the CTA runs the decomposition of Lemma 4.1 block by block with
// no look-ahead (nothing else touches its working copy): the panel step of
// block j (panel_core.cuh, the same code as the panel kernel), then, with all
// four warps, y = d Zp and lambda = d Comp for every row, the L multipliers,
// and the update W ^= y C of every word after column block j by Four Russians
// tables of c bits of the pivot rows, tile by tile.  The working copy lives in
// a per-CTA slice of the workspace (tiled as in the plain decomposition); the
// factors are written to the caller's column blocks at the end.
//
// Two table sizes: c = 4 (8 KB of tables, up to four CTAs per SM: the small
// matrices, whose panel steps are latency-bound, overlap best) and c = 8
// (64 KB of tables sharing shared memory with the panel step's state, three
// CTAs per SM, half the lookups: the larger matrices, whose updates dominate).
// The host routes each matrix by its size (gf2_batched_autotune measures the
// crossover on the device) and runs the two kernels side by side.
#include "m4rm_core.cuh"
#include <mutex>

#include "panel_core.cuh"

namespace gf2 {
namespace {

constexpr int kBatchU = 2;  // row groups of 16 rows per warp and pass

// the update's tables and rows (used between panel steps only)
constexpr int kBatchPad = 4;  // bank skew of the staged pivot rows (build_tables)

template <int C>
struct BatchUpdateShared {
    __align__(16) uint64_t tab[Tabs<C>::Words];
    uint64_t crow[crow_words<C, kBatchPad>()];
    uint64_t zc[16 * 16 * 2];  // [g][x][y, lambda]
};

template <int C>
struct BatchShared {
    union {
        PanelShared panel;
        BatchUpdateShared<C> upd;
    };
    int item;
    int32_t rank;
};

__device__ __forceinline__ uint64_t *scratch_of(const BatchCtx &b, int cta) { return b.scratch + (int64_t)cta * b.scratch_words; }

// 1. the working copy from the caller's column blocks (padding checked),
// the identity permutation, no pivots yet, L multipliers zero
__device__ void batch_ingest(const BatchItem &it, const DecompCtx &c, uint32_t *err, int check)
{
    const int n = c.n, mu = c.mu, tid = threadIdx.x;
    const int nt = (mu + kTileWords - 1) / kTileWords;
    const uint64_t last = (c.m % 64) ? ((1ull << (c.m % 64)) - 1) : ~0ull;
    bool bad = false;
    for (int64_t e = tid; e < (int64_t)nt * kTileWords * n; e += kPanelThreads) {
        const int q = (int)(e / n), i = (int)(e % n);  // consecutive threads: consecutive rows
        uint64_t v = q < mu ? it.A[(int64_t)q * it.lda + i] : 0;
        if (q == mu - 1 && (v & ~last)) {
            bad = true;
            v &= last;
        }
        c.W[widx(c, i, q)] = v;
    }
    if (bad && check) atomicOr(err, 1u);
    for (int i = tid; i < n; i += kPanelThreads) {
        c.perm[i] = i;
        c.pivpanel[i] = 0x7fffffff;
    }
    if (c.Lint)
        for (int64_t e = tid; e < (int64_t)n * c.ldl; e += kPanelThreads) c.Lint[e] = 0;
}

// 2b. the update of panel j by the whole CTA
template <int C>
__device__ void batch_update(const DecompCtx &c, int j, BatchUpdateShared<C> &bs)
{
    const PanelInfo *pi = panel_info(c, j);
    const int R = pi->R, r = pi->r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = c.n;
    if (r == 0) return;
    const int wq = R >> 6, sh = R & 63;
    const bool two = sh + r > 64;
    // tables of (Zp, Comp) for y and lambda
    for (int e = tid; e < 256; e += kPanelThreads) {
        const int g = e >> 4, x = e & 15;
        uint64_t y = 0, l = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((x >> b) & 1) {
                y ^= pi->Zp[4 * g + b];
                l ^= pi->Comp[4 * g + b];
            }
        bs.zc[2 * e] = y;
        bs.zc[2 * e + 1] = l;
    }
    __syncthreads();
    // y and the L multipliers of every row that is not a pivot yet
    const ulonglong2 *zc2 = reinterpret_cast<const ulonglong2 *>(bs.zc);
    for (int i = tid; i < n; i += kPanelThreads) {
        uint64_t y = 0;
        if (c.pivpanel[i] > j) {
            const uint64_t d = c.W[widx(c, i, j)];
            uint64_t l = 0;
#pragma unroll
            for (int g = 0; g < 16; ++g) {
                const ulonglong2 t = zc2[g * 16 + (int)((d >> (4 * g)) & 15)];
                y ^= t.x;
                l ^= t.y;
            }
            if (c.Lint && l) {
                uint64_t *Lr = c.Lint + (int64_t)i * c.ldl;
                Lr[wq] |= l << sh;
                if (two) Lr[wq + 1] |= l >> (64 - sh);
            }
        }
        c.Y[i] = y;
    }
    // the pivot rows: their L rows (T) and echelon words of this block
    for (int t = tid; t < r; t += kPanelThreads) {
        if (c.Lint) {
            uint64_t *Lr = c.Lint + (int64_t)pi->prow[t] * c.ldl;
            Lr[wq] |= pi->T[t] << sh;
            if (two) Lr[wq + 1] |= pi->T[t] >> (64 - sh);
        }
        if (c.Eint) c.Eint[(int64_t)(R + t) * c.lde + j] = pi->Erow[t];
    }
    // W ^= y C on every word after column j, tile by tile
    const int rs = lane / kLanesPerRow, wp = lane % kLanesPerRow, swp = rs & 3;
    const int ng = tables_used<C>(r);
    const int ntiles = (c.mu + kTileWords - 1) / kTileWords;
    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(bs.tab);
    for (int tile = (j + 1) / kTileWords; tile < ntiles; ++tile) {
        const int q0 = tile * kTileWords, col = q0 + 2 * wp;
        const bool live_hi = col + 1 >= j + 1, live_lo = col >= j + 1;
        __syncthreads();
        load_pivot_rows<kPanelThreads, C, kBatchPad>(c, pi->prow, r, q0, bs.crow);
        __syncthreads();
        build_tables<C, kPanelThreads, kBatchPad>(bs.tab, bs.crow);
        __syncthreads();
        if (c.Eint) echelon_rows<C, kPanelThreads>(c, pi, R, r, q0, j + 1, ng, bs.tab);
        // (every lane runs the loop; a lane whose words precede column j+1 skips its loads and stores)
        constexpr int STEP = kRowsPerWarp * kBatchU * (kPanelThreads / 32);
        for (int base = warp * kRowsPerWarp * kBatchU; base < n; base += STEP) {
            uint64_t y[kBatchU];
            ulonglong2 a[kBatchU];
#pragma unroll
            for (int u = 0; u < kBatchU; ++u) {
                const int i = base + u * kRowsPerWarp + rs;
                y[u] = (i < n && live_hi) ? c.Y[i] : 0;
                a[u] = y[u] ? *reinterpret_cast<const ulonglong2 *>(c.W + widx(c, i, col)) : make_ulonglong2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < kBatchU; ++u) {
                if (!y[u]) continue;
                lookup<C>(tab2, y[u], wp, swp, ng, a[u]);
                uint64_t *dst = c.W + widx(c, base + u * kRowsPerWarp + rs, col);
                if (live_lo) *reinterpret_cast<ulonglong2 *>(dst) = a[u];
                else dst[1] = a[u].y;
            }
        }
    }
    __syncthreads();
}

// 3. rank, pivot columns, E and L into the caller's buffers
__device__ void batch_finish(const BatchItem &it, const DecompCtx &c, int rank)
{
    const int tid = threadIdx.x, n = c.n, kmax = c.kmax, mu = c.mu;
    if (tid == 0) *it.rank = rank;
    for (int t = rank + tid; t < kmax; t += kPanelThreads) c.pivcols[t] = -1;
    if (it.E)
        for (int64_t e = tid; e < (int64_t)mu * kmax; e += kPanelThreads) {
            const int q = (int)(e / kmax), t = (int)(e % kmax);
            uint64_t v = 0;
            if (t < rank && q >= (c.pivcols[t] >> 6)) v = c.Eint[(int64_t)t * c.lde + q];
            it.E[(int64_t)q * it.lde + t] = v;
        }
    if (it.L) {
        const int lw = (kmax + 63) / 64;
        for (int64_t e = tid; e < (int64_t)lw * n; e += kPanelThreads) {
            const int q = (int)(e / n), t = (int)(e % n);
            it.L[(int64_t)q * it.ldl + t] = c.Lint[(int64_t)c.perm[t] * c.ldl + q];
        }
    }
}

template <int C>
__global__ void __launch_bounds__(kPanelThreads, 4) k_batch(BatchCtx b)
{
    extern __shared__ __align__(16) uint8_t batch_smem[];
    BatchShared<C> &bs = *reinterpret_cast<BatchShared<C> *>(batch_smem);
    const int tid = threadIdx.x;
    uint64_t *base = scratch_of(b, blockIdx.x);
    for (;;) {
        if (tid == 0) {
            const int k = atomicAdd(b.next_item, 1);
            bs.item = k < b.count ? b.order[k] : -1;
        }
        __syncthreads();
        const int idx = bs.item;
        __syncthreads();
        if (idx < 0) return;
        const BatchItem it = b.items[idx];
        DecompCtx c{};
        c.n = it.n;
        c.m = it.m;
        c.mu = (it.m + 63) / 64;
        c.kmax = it.n < it.m ? it.n : it.m;
        c.tstride = (int64_t)it.n * kTileWords;
        c.lde = (c.mu + kTileWords - 1) / kTileWords * kTileWords;
        c.ldl = (c.kmax + 63) / 64 > 0 ? (c.kmax + 63) / 64 : 1;
        c.perm = it.perm;
        c.pivcols = it.pivcols;
        c.W = base;
        c.Y = base + b.off_y;
        c.info = reinterpret_cast<PanelInfo *>(base + b.off_info);
        c.info_ring = 1;
        c.pivpanel = reinterpret_cast<int32_t *>(base + b.off_pivpanel);
        c.Lint = b.factors ? base + b.off_lint : nullptr;
        c.Eint = b.factors ? base + b.off_eint : nullptr;
        c.F = nullptr;  // W holds every finished word: no look-ahead here
        if (c.n == 0 || c.m == 0) {
            if (tid == 0) *it.rank = 0;
            for (int i = tid; i < c.n; i += kPanelThreads) it.perm[i] = i;
            if (it.L)
                for (int64_t e = tid; e < (int64_t)it.ldl * ((c.kmax + 63) / 64); e += kPanelThreads) it.L[e] = 0;
            continue;
        }
        batch_ingest(it, c, b.err, b.check);
        __syncthreads();
        int rank = 0;
        for (int j = 0; j < c.mu; ++j) {
            panel_block(c, j, bs.panel);
            __syncthreads();
            rank += panel_info(c, j)->r;
            batch_update<C>(c, j, bs.upd);  // (reuses the panel step's shared memory)
            __syncthreads();
        }
        batch_finish(it, c, rank);
        __syncthreads();
    }
}

template <int C>
cudaError_t prepare_batch()
{
    // (several host threads may launch batches at once: the serving engine's
    // lanes and callers on other streams)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchShared<C>));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <int C>
int ctas_per_sm()
{
    if (prepare_batch<C>() != cudaSuccess) return 1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<C>, kPanelThreads, sizeof(BatchShared<C>)) !=
        cudaSuccess)
        return 1;
    return per_sm > 0 ? per_sm : 1;
}

}  // namespace

int batch_ctas_per_sm(int c) { return c == 8 ? ctas_per_sm<8>() : ctas_per_sm<4>(); }

cudaError_t launch_batch(const BatchCtx &b, int grid, int c, cudaStream_t s)
{
    if (c == 8) {
        const cudaError_t e = prepare_batch<8>();
        if (e != cudaSuccess) return e;
        k_batch<8><<<grid, kPanelThreads, sizeof(BatchShared<8>), s>>>(b);
    } else {
        const cudaError_t e = prepare_batch<4>();
        if (e != cudaSuccess) return e;
        k_batch<4><<<grid, kPanelThreads, sizeof(BatchShared<4>), s>>>(b);
    }
    return cudaGetLastError();
}

}  // namespace gf2
