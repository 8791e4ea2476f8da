// Reduced row echelon form of the echelon factor E (the Gauss-Jordan
// option that the paper names among the decomposition's uses, Section 1;
// it does not spell it out, so this is the textbook definition): with U = E
// restricted to the pivot columns -- unit upper triangular; a zero row past
// the rank counts as a unit row -- R = U^-1 E, whose pivot columns are unit
// columns.  The result is unique (it depends on the row space only).
//
// Three kernels; the host recursion in gf2_api.cu (gf2_rref) combines them
// with the Four Russians product:
//   k_rref_inverse, k_rref_diag  every 64-row block by itself, all blocks in
//                 two launches: V_i = U_ii^-1 (the block's own pivot
//                 columns), then E_i <- V_i E_i in place (one CTA per block
//                 and group of column tiles);
//   k_gather_cols the bits of a range of rows at a range of pivot columns,
//                 as a matrix in column blocks: the left operand of the
//                 product E_top ^= E_top[:, pivots of the bottom] R_bottom.
// And the null-space basis read off R (k_free_cols, k_nullspace_fill).
#include "m4rm_core.cuh"
#include "panel_core.cuh"

namespace gf2 {
namespace {

constexpr int kRrefThreads = 256;
constexpr int kRrefC = 4;    // 16 tables of 16 entries: 8 KB, static shared memory
constexpr int kRrefPad = 4;  // bank skew of the staged rows (build_tables)

// U_ii^-1 of every 64-row block i, by rows, into V[64 i ..] (one CTA of 64
// threads per block).  A separate launch: k_rref_diag rewrites the pivot
// columns that this reads.
__global__ void __launch_bounds__(64) k_rref_inverse(const uint64_t *E, int64_t ld, const int32_t *pivcols, int64_t k,
                                                     int64_t m, uint64_t *V)
{
    __shared__ uint64_t ucol[64];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t r0 = 64 * (int64_t)blockIdx.x;  // the block's first row
    const int nb = (int)(k - r0 < 64 ? k - r0 : 64);
    // U_ii by columns: bit s of column c is row r0 + s at column pivcols[r0 + c]
    // (entries below the diagonal are zero in an echelon form); a row
    // without a pivot (past the rank) contributes the unit column e_c
    {
        const int c = tid;
        const int p = c < nb ? pivcols[r0 + c] : -1;
        uint64_t v = 1ull << c;
        if (p >= 0 && p < m) {  // (a column outside E counts as no pivot)
            const uint64_t *col = E + (int64_t)(p >> 6) * ld + r0;
            v = 0;
            for (int s = 0; s < nb; ++s) v |= ((col[s] >> (p & 63)) & 1ull) << s;
        }
        ucol[c] = v;
    }
    __syncthreads();
    // U x = e_c by a backward sweep: bit t of x is final once the columns
    // above t are removed, and column t leaves the right-hand side when it
    // is set; x is column c of the inverse, and a transpose gives the rows
    if (tid < 32) {
        uint64_t x[2] = {1ull << lane, 1ull << (lane + 32)};
        for (int t = 63; t > 0; --t) {
            const uint64_t u = ucol[t] & ((1ull << t) - 1);
            if ((x[0] >> t) & 1) x[0] ^= u;
            if ((x[1] >> t) & 1) x[1] ^= u;
        }
        transpose64(x, lane);  // x[h] = row lane + 32h of U_ii^-1
        V[r0 + lane] = x[0];
        V[r0 + lane + 32] = x[1];
    }
}

// E_i <- U_ii^-1 E_i for every 64-row block i (V from k_rref_inverse), in place
__global__ void __launch_bounds__(kRrefThreads) k_rref_diag(uint64_t *E, int64_t ld, const uint64_t *V, int k, int mw)
{
    __shared__ __align__(16) uint64_t tab[Tabs<kRrefC>::Words];
    __shared__ uint64_t crow[crow_words<kRrefC, kRrefPad>()];
    const int tid = threadIdx.x;
    const int64_t r0 = 64 * (int64_t)blockIdx.x;
    const int nb = (int)(k - r0 < 64 ? k - r0 : 64);
    // each tile of the block's rows: tables of the 64 rows, then row s takes
    // the combination V[r0 + s] of them
    const int ntiles = (mw + kTileWords - 1) / kTileWords;
    const int s = tid / kTileWords, w = tid % kTileWords;
    for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
        const int q = tile * kTileWords + w;
        __syncthreads();  // the previous tile's lookups are done
        crow[tid + kRrefPad * (s / kRrefC)] = (s < nb && q < mw) ? E[(int64_t)q * ld + r0 + s] : 0;
        __syncthreads();
        build_tables<kRrefC, kRrefThreads, kRrefPad>(tab, crow);
        __syncthreads();
        if (s < nb && q < mw) {
            const uint64_t y = V[r0 + s];
            uint64_t acc = 0;
#pragma unroll
            for (int g = 0; g < Tabs<kRrefC>::K; ++g)
                acc ^= tab[tab_entry<kRrefC>(g, (int)((y >> (kRrefC * g)) & (Tabs<kRrefC>::X - 1))) * kTileWords + w];
            E[(int64_t)q * ld + r0 + s] = acc;
        }
    }
}

static_assert(kRrefThreads == 64 * kTileWords, "one thread per (row, word) of a block's tile");

// out word (i, q), i < rows: bit t = row a + i of E at column pivcols[c0 + 64q + t]
// (0 past ncols or at a missing pivot; E has m columns)
__global__ void k_gather_cols(const uint64_t *__restrict__ E, int64_t ld, int64_t m, const int32_t *__restrict__ pivcols,
                              int64_t a, int64_t rows, int64_t c0, int64_t ncols, uint64_t *__restrict__ out, int64_t ldo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int64_t words = (ncols + 63) / 64;
    for (int64_t q = blockIdx.y; q < words; q += gridDim.y) {
        uint64_t v = 0;
        const int tmax = (int)(ncols - 64 * q < 64 ? ncols - 64 * q : 64);
        for (int t = 0; t < tmax; ++t) {
            const int p = pivcols[c0 + 64 * q + t];
            if (p >= 0 && p < m) v |= ((E[(int64_t)(p >> 6) * ld + a + i] >> (p & 63)) & 1ull) << t;
        }
        out[q * ldo + i] = v;
    }
}

// the first t < r with pivcols[t] >= c (pivcols increasing)
__device__ __forceinline__ int64_t pivot_lower_bound(const int32_t *pivcols, int64_t r, int64_t c)
{
    int64_t lo = 0, hi = r;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (pivcols[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// free[j] = the j-th column (increasing) that is not a pivot column
__global__ void k_free_cols(const int32_t *__restrict__ pivcols, int64_t r, int64_t m, int32_t *__restrict__ free)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lb = pivot_lower_bound(pivcols, r, c);
        if (lb < r && pivcols[lb] == c) continue;
        if (c - lb < m - r) free[c - lb] = (int32_t)c;  // (in range for any pivot list)
    }
}

// The null-space basis read off the reduced row echelon form R (Section 1
// names it among the uses of the decomposition): N (m x nul, nul = m - r)
// has column j = the solution of R x = 0 with free variable f_j = 1 and the
// other free variables 0, so row f_j of N is the unit word e_j and row
// pivcols[t] is R's row t at the free columns.  Thread per row of N.
__global__ void k_nullspace_fill(const uint64_t *__restrict__ R, int64_t ldr, const int32_t *__restrict__ pivcols,
                                 int64_t r, const int32_t *__restrict__ free, int64_t nul, uint64_t *__restrict__ N,
                                 int64_t ldn, int64_t m)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t lb = pivot_lower_bound(pivcols, r, i);
    const bool pivot = lb < r && pivcols[lb] == i;
    const int64_t words = (nul + 63) / 64;
    for (int64_t q = blockIdx.y; q < words; q += gridDim.y) {
        uint64_t v = 0;
        if (pivot) {
            const int tmax = (int)(nul - 64 * q < 64 ? nul - 64 * q : 64);
            for (int b = 0; b < tmax; ++b) {
                const int f = free[64 * q + b];
                if (f >= 0 && f < m) v |= ((R[(int64_t)(f >> 6) * ldr + lb] >> (f & 63)) & 1ull) << b;
            }
        } else {
            const int64_t j = i - lb;  // this free column's index
            v = (j >> 6) == q ? 1ull << (j & 63) : 0;
        }
        N[q * ldn + i] = v;
    }
}

int rref_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

cudaError_t launch_rref_diag(uint64_t *E, int64_t ld, const int32_t *pivcols, int64_t k, int64_t m, uint64_t *V,
                             cudaStream_t s)
{
    const int64_t mw = (m + 63) / 64;
    if (k <= 0 || mw <= 0) return cudaSuccess;
    const int64_t blocks = (k + 63) / 64, ntiles = (mw + kTileWords - 1) / kTileWords;
    k_rref_inverse<<<(unsigned)blocks, 64, 0, s>>>(E, ld, pivcols, k, m, V);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // about eight CTAs per SM in all, each over every gy-th tile of its block
    int64_t gy = (8 * (int64_t)rref_sms() + blocks - 1) / blocks;
    if (gy > ntiles) gy = ntiles;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    k_rref_diag<<<dim3((unsigned)blocks, (unsigned)gy), kRrefThreads, 0, s>>>(E, ld, V, (int)k, (int)mw);
    return cudaGetLastError();
}

cudaError_t launch_gather_cols(const uint64_t *E, int64_t ld, int64_t m, const int32_t *pivcols, int64_t a, int64_t rows,
                               int64_t c0, int64_t ncols, uint64_t *out, int64_t ldo, cudaStream_t s)
{
    if (rows <= 0 || ncols <= 0) return cudaSuccess;
    const int64_t words = (ncols + 63) / 64;
    const int64_t gx = (rows + 255) / 256, gy = words < 65535 ? words : 65535;
    k_gather_cols<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(E, ld, m, pivcols, a, rows, c0, ncols, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_nullspace(const uint64_t *R, int64_t ldr, const int32_t *pivcols, int64_t r, int64_t m, int32_t *free,
                             uint64_t *N, int64_t ldn, cudaStream_t s)
{
    const int64_t nul = m - r;
    if (m <= 0 || nul <= 0) return cudaSuccess;
    int64_t g = (m + 255) / 256;
    if (g > 16 * (int64_t)rref_sms()) g = 16 * (int64_t)rref_sms();
    k_free_cols<<<(unsigned)g, 256, 0, s>>>(pivcols, r, m, free);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t words = (nul + 63) / 64;
    const int64_t gx = (m + 255) / 256, gy = words < 65535 ? words : 65535;
    k_nullspace_fill<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(R, ldr, pivcols, r, free, nul, N, ldn, m);
    return cudaGetLastError();
}

}  // namespace gf2
