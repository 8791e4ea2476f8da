// The product C (+)= A B over F2 by the Four Russians method (Section 6 of
// the paper: tables of 2^8 combinations of 8 rows of B, one lookup per 8
// bits of a row of A), on the boundary layout itself (column blocks: no
// conversion in or out).
//
// One CTA owns a block of C: 256 U rows by one 4-word column tile, and keeps
// it in registers over the whole inner dimension (or over its share of it).
// Per 64 rows of B it builds the 8 tables of that slice of the tile in shared
// memory (64 KB, the conflict-free quad layout of m4rm_core.cuh) and every
// row of the block takes 8 lookups.  So A is read once per tile, B once per
// row block and C written once: the shared-memory lookups (32 B per row and
// 64 rows of B) are the bound, as in the decomposition's update.  CTAs are
// numbered tile-fastest, so the CTAs that run together share the same rows
// of A in L2.  When there are too few blocks to fill the GPU the inner
// dimension is split over CTAs that combine their parts with atomic XORs.
#include <cstdlib>
#include <cstring>

#include "m4rm_core.cuh"

namespace gf2 {
namespace {

constexpr int kPThreads = 512;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPC = 8;  // bits per lookup

#ifdef GF2_COUNT_OPS
__device__ unsigned long long g_mmm_ops[kNumOps];  // the op-counting build's counters
#endif

constexpr int kPPad = 4;  // words between the 8-row groups of the staged slice of B
constexpr int kPSmemBytes = (Tabs<kPC>::Words + 64 * kTileWords + kPPad * (64 / kPC)) * 8;

template <int U, int MINB>
__global__ void __launch_bounds__(kPThreads, MINB) k_mmm(MmmCtx c, int kb_per_split)
{
    constexpr int kStride = kRowsPerWarp * kPWarps;  // rows per row group
    extern __shared__ __align__(16) uint64_t smem[];
    uint64_t *tab = smem;
    uint64_t *crow = smem + Tabs<kPC>::Words;
    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(tab);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = lane / kLanesPerRow, wp = lane % kLanesPerRow, swp = rs & 3;
    const int q0 = blockIdx.x * kTileWords, col = q0 + 2 * wp;
    const int kw = (c.k + 63) / 64;
    const int kb0 = blockIdx.z * kb_per_split, kb1 = min(kw, kb0 + kb_per_split);
    // rows of this thread: base + kStride u (u < U); n < 2^31
    const int base = blockIdx.y * (kStride * U) + warp * kRowsPerWarp + rs;
    ulonglong2 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = make_ulonglong2(0, 0);
    GF2_OPS(unsigned long long n_lk = 0, n_tab = 0; const int lw = (col < c.mw) + (col + 1 < c.mw);)
    for (int kb = kb0; kb < kb1; ++kb) {
        // rows 64 kb .. of B on this tile (zero beyond k and beyond the last word)
        if (tid < 64 * kTileWords) {
            const int t = tid / kTileWords, w = tid % kTileWords;
            const int64_t r = 64 * (int64_t)kb + t;
            crow[tid + kPPad * (t / kPC)] = (r < c.k && q0 + w < c.mw) ? c.B[(int64_t)(q0 + w) * c.ldb + r] : 0;
        }
        // this slice's word of A for every row (consumed after the table build)
        uint64_t y[U];
        const uint64_t *Ak = c.A + (int64_t)kb * c.lda;
#pragma unroll
        for (int u = 0; u < U; ++u) y[u] = base + u * kStride < c.n ? Ak[base + u * kStride] : 0;
        __syncthreads();  // the previous slice's lookups are done; crow is complete
        build_tables<kPC, kPThreads, kPPad>(tab, crow);
        GF2_OPS(if (tid == 0) n_tab += (unsigned long long)Tabs<kPC>::K * (Tabs<kPC>::X - 1) * live_words(q0, c.mw);)
        __syncthreads();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!y[u]) continue;
            GF2_OPS(n_lk += (unsigned long long)Tabs<kPC>::K * lw;)
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int gg = g ^ swp;
                const int x = (int)((y[u] >> (kPC * gg)) & 255);
                const ulonglong2 t = tab2[tab_entry<kPC>(gg, x) * (kTileWords / 2) + wp];
                acc[u].x ^= t.x;
                acc[u].y ^= t.y;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int row = base + u * kStride;
        if (row >= c.n) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = col + h;
            if (q >= c.mw) continue;
            const uint64_t v = h ? acc[u].y : acc[u].x;
            uint64_t *dst = c.C + (int64_t)q * c.ldc + row;
            if (c.mode == kMmmStore) *dst = v;
            else if (c.mode == kMmmXor) *dst ^= v;
            else if (v) atomicXor(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)v);
        }
    }
    GF2_OPS(add_ops(g_mmm_ops, kOpMmmLookups, n_lk); add_ops(g_mmm_ops, kOpMmmTable, n_tab);)
}

// D = X ^ Y: threads along the rows of a column block, column blocks over
// the grid's y dimension
__global__ void k_xor(uint64_t *__restrict__ D, int64_t ldd, const uint64_t *X, int64_t ldx, const uint64_t *Y,
                      int64_t ldy, int64_t rows, int64_t words)
{
    GF2_OPS(unsigned long long n_add = 0;)
    for (int64_t q = blockIdx.y; q < words; q += gridDim.y) {
        uint64_t *d = D + q * ldd;
        const uint64_t *x = X + q * ldx, *y = Y + q * ldy;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
            d[i] = x[i] ^ y[i];
            GF2_OPS(++n_add;)
        }
    }
    GF2_OPS(add_ops(g_mmm_ops, kOpMmmAdds, n_add);)
}

int g_sms = 0;

int sm_count()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

template <int U, int MINB>
cudaError_t launch_u(MmmCtx c, int splits, cudaStream_t s)
{
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        e = cudaFuncSetAttribute(k_mmm<U, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    const int rows_per_cta = kRowsPerWarp * kPWarps * U;
    const int kw = (c.k + 63) / 64;
    const int64_t tiles = (c.mw + kTileWords - 1) / kTileWords, blocks = (c.n + rows_per_cta - 1) / rows_per_cta;
    const int per = (kw + splits - 1) / splits;
    splits = (kw + per - 1) / per;
    if (splits > 1) {
        if (c.mode == kMmmStore) {
            e = cudaMemset2DAsync(c.C, (size_t)c.ldc * 8, 0, (size_t)c.n * 8, (size_t)c.mw, s);
            if (e != cudaSuccess) return e;
        }
        c.mode = kMmmAtomicXor;
    }
    dim3 grid((unsigned)tiles, (unsigned)blocks, (unsigned)splits);
    k_mmm<U, MINB><<<grid, kPThreads, kPSmemBytes, s>>>(c, per);
    return cudaGetLastError();
}

// The launch shapes: (row groups U, resident CTAs per SM).  U = 6 is the
// most that stays within 64 registers (two CTAs per SM); U = 12 runs one CTA
// per SM with up to 128 registers and amortises each slice's table build
// over twice the rows (measured fastest from n = 8192 up).
struct Shape {
    int u, minb;
};
constexpr Shape kShapes[] = {{2, 2}, {4, 2}, {6, 2}, {12, 1}};
int g_split_override = 0;
const int g_shape_override = [] {
    const char *e = getenv("GF2_MMM_SHAPE");
    if (!e) return -1;
    const int i = atoi(e);
    const char *c = strchr(e, ':');
    if (c) g_split_override = atoi(c + 1);
    return (i >= 0 && i < 4) ? i : -1;
}();

}  // namespace

cudaError_t launch_mmm(MmmCtx c, cudaStream_t s)
{
    if (c.n <= 0 || c.mw <= 0) return cudaSuccess;
    if (c.k <= 0) {
        if (c.mode != kMmmStore) return cudaSuccess;
        return cudaMemset2DAsync(c.C, (size_t)c.ldc * 8, 0, (size_t)c.n * 8, (size_t)c.mw, s);
    }
    // Cost model: whole waves of CTAs, each CTA's time proportional to its
    // slices of B times (its row groups + the per-slice overhead of table
    // build, barriers and loads: about four row groups); two resident CTAs
    // share an SM, each at half rate.  Splitting the inner dimension evens
    // out the last wave (it zeroes C first and combines the parts by atomics
    // in L2: more DRAM traffic, but the kernel is bound by shared memory); a
    // split keeps at least min(32, max(8, kw/8)) slices per CTA.  Fitted to
    // measured times of every shape and of 1..32 splits at n = 8192..32768.
    const int kw = (c.k + 63) / 64;
    const int64_t tiles = (c.mw + kTileWords - 1) / kTileWords;
    const int minper = kw / 8 < 8 ? 8 : (kw / 8 > 32 ? 32 : kw / 8);
    double best = 1e300;
    int bi = 0, bsplit = 1;
    for (int i = 0; i < (int)(sizeof(kShapes) / sizeof(kShapes[0])); ++i) {
        const int64_t rows_per_cta = (int64_t)kRowsPerWarp * kPWarps * kShapes[i].u;
        const int64_t blocks = (c.n + rows_per_cta - 1) / rows_per_cta;
        const int64_t slots = (int64_t)kShapes[i].minb * sm_count();
        for (int splits = 1; splits <= 64 && (splits == 1 || kw / splits >= minper); ++splits) {
            const int per = (kw + splits - 1) / splits;
            const int64_t ctas = tiles * blocks * ((kw + per - 1) / per);
            const int64_t waves = (ctas + slots - 1) / slots;
            const double share = kShapes[i].minb == 2 ? 2.0 : 1.0;
            const double cost = (double)waves * per * (kShapes[i].u + 4.0) * share * (splits > 1 ? 1.02 : 1.0);
            if (cost < best) {
                best = cost;
                bi = i;
                bsplit = splits;
            }
        }
    }
    if (g_shape_override >= 0) {  // GF2_MMM_SHAPE=index[:splits], for calibrating the model
        bi = g_shape_override;
        if (g_split_override > 0) bsplit = g_split_override;
    }
    switch (bi) {
    case 0: return launch_u<2, 2>(c, bsplit, s);
    case 1: return launch_u<4, 2>(c, bsplit, s);
    case 2: return launch_u<6, 2>(c, bsplit, s);
    default: return launch_u<12, 1>(c, bsplit, s);
    }
}

#ifdef GF2_COUNT_OPS
cudaError_t read_mmm_ops(unsigned long long *acc, bool reset)
{
    unsigned long long h[kNumOps];
    cudaError_t e = cudaMemcpyFromSymbol(h, g_mmm_ops, sizeof(h));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < kNumOps; ++i) acc[i] += h[i];
    if (reset) {
        const unsigned long long z[kNumOps] = {};
        e = cudaMemcpyToSymbol(g_mmm_ops, z, sizeof(z));
    }
    return e;
}
#endif

cudaError_t launch_xor(uint64_t *D, int64_t ldd, const uint64_t *X, int64_t ldx, const uint64_t *Y, int64_t ldy,
                       int64_t rows, int64_t words, cudaStream_t s)
{
    if (rows <= 0 || words <= 0) return cudaSuccess;
    const int64_t bx = (rows + 255) / 256, by = words < 65535 ? words : 65535;
    const int64_t cap = 16 * (int64_t)sm_count();
    const int64_t gx = bx * by > cap ? (cap / by > 0 ? cap / by : 1) : bx;
    k_xor<<<dim3((unsigned)gx, (unsigned)by), 256, 0, s>>>(D, ldd, X, ldx, Y, ldy, rows, words);
    return cudaGetLastError();
}

}  // namespace gf2
