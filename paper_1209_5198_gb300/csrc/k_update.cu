// Trailing update A(j+1) = E xor Y C (eq. (Aj) of the paper) by the Method
// of Four Russians (M4RM, Section 6): the r <= 64 pivot rows C of the panel
// are combined into 8 tables of 2^8 entries per 8-word column tile (one XOR
// per entry), and every row of E then takes 8 table lookups and XORs per
// word, indexed by the 8 bytes of its multiplier y.
//
// GB300 layout choices:
//   * rows are row-major inside the library, so one row's 8-word tile is 64
//     contiguous bytes; a warp covers 8 rows x 8 words with 128-bit accesses
//     (lane = row slot (lane/4) x word pair (lane%4)) -- full sectors, no
//     re-reads;
//   * the tables sit in shared memory as [table pair][x][half][8 words]: the
//     two rows of a quarter-warp (one LDS.128 phase) read tables g and g^1,
//     which live in opposite 64-byte halves of the bank space, so every
//     lookup is conflict-free whatever the bytes of y are;
//   * a CTA owns one column tile and a contiguous chunk of rows, so each
//     table build (2048 x 8 XORs) is amortised over thousands of rows.
// The same kernel serves the standalone product C ^= A B (one launch per
// 64-row slice of B).
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr int kTabWords = kNumTables * 256 * kTileWords;          // 16384 words = 128 KB
constexpr int kSmemBytes = (kTabWords + 64 * kTileWords) * 8;      // + C rows

// index (in 8-word entries) of entry x of table g
__device__ __forceinline__ int tab_entry(int g, int x) { return (((g >> 1) * 256 + x) << 1) | (g & 1); }

__device__ __forceinline__ void build_tables(uint64_t *tab, const uint64_t *crow)
{
    // warp g builds table g; lane = word w (lane & 7) x quarter qq (lane >> 3);
    // each quarter fixes the top 2 bits of x and walks the low 6 in Gray order.
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int w = lane & 7, qq = lane >> 3;
    uint64_t cb[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cb[b] = crow[(8 * g + b) * kTileWords + w];
    uint64_t v = ((qq & 1) ? cb[6] : 0) ^ ((qq & 2) ? cb[7] : 0);
    tab[tab_entry(g, qq * 64) * kTileWords + w] = v;
#pragma unroll
    for (int i = 1; i < 64; ++i) {
        const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : (i & 16) ? 4 : 5;
        v ^= cb[b];
        tab[tab_entry(g, qq * 64 + (i ^ (i >> 1))) * kTileWords + w] = v;
    }
}

template <bool kDecomp>
__global__ void __launch_bounds__(kUpdateThreads, 1)
k_update(DecompCtx dc, MmmCtx mc, int j, int tile0, int m_words)
{
    extern __shared__ __align__(16) uint64_t smem[];
    uint64_t *tab = smem;
    uint64_t *crow = smem + kTabWords;
    const int tid = threadIdx.x;
    const int q0 = (tile0 + blockIdx.x) * kTileWords;

    int r, R = 0, row_begin, row_end, live_from;
    if (kDecomp) {
        R = dc.info[j].R;
        r = dc.info[j].r;
        if (r == 0) return;
        row_begin = R + r;
        row_end = dc.n;
        live_from = j + 1;
    } else {
        r = min(64, mc.k - 64 * j);
        row_begin = 0;
        row_end = mc.n;
        live_from = 0;
    }

    // C rows of this column tile (zero beyond r)
    for (int idx = tid; idx < 64 * kTileWords; idx += kUpdateThreads) {
        const int t = idx / kTileWords, w = idx % kTileWords;
        uint64_t v = 0;
        if (t < r) {
            if (kDecomp) {
                const int64_t srow = dc.perm[R + t];
                v = dc.W[srow * dc.ldw + q0 + w];
            } else if (q0 + w < m_words) {
                v = mc.B[(int64_t)(64 * j + t) * mc.ldb + q0 + w];
            }
        }
        crow[idx] = v;
    }
    __syncthreads();
    build_tables(tab, crow);
    __syncthreads();

    const ulonglong2 *tab2 = reinterpret_cast<const ulonglong2 *>(tab);
    const int ng2 = ((r + 7) / 8 + 1) & ~1;  // tables in use, rounded to pairs
    const int lane = tid & 31, warp = tid >> 5;
    const int rs = lane >> 2, wp = lane & 3, swp = rs & 1;
    const int col = q0 + 2 * wp;
    const bool live = (col + 1 >= live_from) && (kDecomp || col < m_words);

    uint64_t *T;
    int64_t ldt;
    if (kDecomp) { T = dc.W; ldt = dc.ldw; }
    else { T = mc.C; ldt = mc.ldc; }

    const int rows = row_end - row_begin;
    const int chunk = (rows + gridDim.y - 1) / gridDim.y;
    const int rb = row_begin + blockIdx.y * chunk;
    const int re = min(row_end, rb + chunk);

    constexpr int U = 4;
    for (int base = rb + warp * 8 * U; base < re; base += 8 * U * (kUpdateThreads / 32)) {
        int64_t off[U];
        uint64_t y[U];
        ulonglong2 a[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * 8 + rs;
            ok[u] = i < re;
            y[u] = 0;
            off[u] = 0;
            if (ok[u]) {
                if (kDecomp) {
                    off[u] = (int64_t)dc.perm[i] * ldt + col;
                    y[u] = dc.Y[i];
                } else {
                    off[u] = (int64_t)i * ldt + col;
                    y[u] = mc.A[(int64_t)i * mc.lda + j];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = make_ulonglong2(0, 0);
            if (ok[u] && live) a[u] = *reinterpret_cast<const ulonglong2 *>(T + off[u]);
        }
        for (int g = 0; g < ng2; ++g) {
            const int gg = g ^ swp;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = (int)((y[u] >> (8 * gg)) & 255);
                const ulonglong2 t = tab2[tab_entry(gg, x) * (kTileWords / 2) + wp];
                a[u].x ^= t.x;
                a[u].y ^= t.y;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (ok[u] && live) *reinterpret_cast<ulonglong2 *>(T + off[u]) = a[u];
    }

    // Echelon rows of the panel's pivots: E_s = T^-1[s] * C on this tile.
    if (kDecomp && dc.Eint && blockIdx.y == 0) {
        const PanelInfo *pi = dc.info + j;
        for (int idx = tid; idx < r * kTileWords; idx += kUpdateThreads) {
            const int t = idx / kTileWords, w = idx % kTileWords;
            const int q = q0 + w;
            if (q < live_from || q >= dc.mu) continue;
            const uint64_t ym = pi->Tinv[t];
            uint64_t acc = 0;
            for (int g = 0; g < ng2; ++g) acc ^= tab[tab_entry(g, (int)((ym >> (8 * g)) & 255)) * kTileWords + w];
            dc.Eint[(int64_t)(R + t) * dc.ldw + q] = acc;
        }
    }
}

// Y (per position) and the L multipliers (per storage row) of panel j.
__global__ void __launch_bounds__(256) k_ly(DecompCtx c, int j)
{
    const PanelInfo *pi = c.info + j;
    const int R = pi->R, r = pi->r;
    if (r == 0) return;
    __shared__ uint64_t zp[64], cp[64];
    if (threadIdx.x < 64) {
        zp[threadIdx.x] = pi->Zp[threadIdx.x];
        cp[threadIdx.x] = pi->Comp[threadIdx.x];
    }
    __syncthreads();
    const int wq = R >> 6, sh = R & 63;
    const bool two = sh + r > 64;
    const int stride = gridDim.x * blockDim.x;
    for (int i = R + r + blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += stride) {
        const int srow = c.perm[i];
        const uint64_t d = c.W[(int64_t)srow * c.ldw + j];
        uint64_t y = 0, l = 0;
        for (uint64_t x = d; x; x &= x - 1) {
            const int p = __ffsll((long long)x) - 1;
            y ^= zp[p];
            l ^= cp[p];
        }
        c.Y[i] = y;
        if (c.Lint) {
            uint64_t *Lr = c.Lint + (int64_t)srow * c.ldl;
            Lr[wq] |= l << sh;
            if (two) Lr[wq + 1] |= l >> (64 - sh);
        }
    }
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < r; t += blockDim.x) {
            const int srow = c.perm[R + t];
            if (c.Lint) {
                const uint64_t l = pi->T[t];
                uint64_t *Lr = c.Lint + (int64_t)srow * c.ldl;
                Lr[wq] |= l << sh;
                if (two) Lr[wq + 1] |= l >> (64 - sh);
            }
            if (c.Eint) c.Eint[(int64_t)(R + t) * c.ldw + j] = pi->Erow[t];
        }
    }
}

int g_num_sms = 0;

int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <bool kDecomp>
cudaError_t set_smem_attr()
{
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_update<kDecomp>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

int row_chunks(int ntiles, int est_rows)
{
    const int target = 2 * num_sms();
    int chunks = (target + ntiles - 1) / ntiles;
    const int max_chunks = est_rows / 256 > 1 ? est_rows / 256 : 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    return chunks;
}

}  // namespace

cudaError_t launch_ly(const DecompCtx &c, int j, cudaStream_t s)
{
    int blocks = (c.n + 255) / 256;
    const int cap = 2 * num_sms();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_ly<<<blocks, 256, 0, s>>>(c, j);
    return cudaGetLastError();
}

cudaError_t launch_update(const DecompCtx &c, int j, cudaStream_t s)
{
    const int tile0 = (j + 1) / kTileWords;
    const int ntiles = (c.mu + kTileWords - 1) / kTileWords - tile0;
    if (ntiles <= 0) return cudaSuccess;
    cudaError_t e = set_smem_attr<true>();
    if (e != cudaSuccess) return e;
    int est = c.n - 64 * j;
    if (est < 256) est = 256;
    dim3 grid(ntiles, row_chunks(ntiles, est));
    MmmCtx none{};
    k_update<true><<<grid, kUpdateThreads, kSmemBytes, s>>>(c, none, j, tile0, 0);
    return cudaGetLastError();
}

cudaError_t launch_mmm_pass(const MmmCtx &c, int kb, int m_words, cudaStream_t s)
{
    const int ntiles = (m_words + kTileWords - 1) / kTileWords;
    if (ntiles <= 0 || c.n <= 0) return cudaSuccess;
    cudaError_t e = set_smem_attr<false>();
    if (e != cudaSuccess) return e;
    dim3 grid(ntiles, row_chunks(ntiles, c.n));
    DecompCtx none{};
    k_update<false><<<grid, kUpdateThreads, kSmemBytes, s>>>(none, c, kb, 0, m_words);
    return cudaGetLastError();
}

}  // namespace gf2
