// Decomposition over a prime field F_p (gf2_fp_decompose of include/gf2.h):
// the remark after eq. (cond:nonsing:Bk) of Section 4.2 carries the block
// method over to F_q -- the pivot condition becomes "the reduced entry beta
// is nonzero" instead of "is one", and beta stays on the diagonal of the
// echelon factor.  For a prime p the result is the PLE form with the same
// pivot rule as over F2: column by column, the first row in the current
// order whose reduced entry is nonzero is exchanged into the pivot slot, the
// rows after it are eliminated (multiplier = entry / beta), no column is
// ever exchanged.  P A = L E with L unit lower trapezoidal (n x k) and E in
// row echelon form (k x m) with leading entries beta at the pivot columns.
//
// GB300 design.  Elements are 32-bit residues (p < 2^31); storage rows never
// move (a position -> row map records the exchanges, as in the F2 path).
// Block columns of kFpB = 32 columns:
//   k_fp_load     the block column of every row into a column-major panel
//                 buffer (a column of the block is contiguous over the rows);
//   k_fp_panel    one cooperative launch for the block (at most one CTA per
//                 SM, each keeping its rows' block entries, pivot marks and
//                 positions in shared memory), one grid barrier per column:
//                 every CTA posts its first candidate (min position with a
//                 nonzero entry among its non-pivot rows, one 64-bit
//                 atomicMin of (position, row)) and copies that row's entries
//                 to its slot; after the barrier every CTA reads the winner's
//                 slot (the pivot row), eliminates its non-pivot rows
//                 (multiplier l = entry * beta^-1, stored in place: the L
//                 entry) and applies the exchange to the rows it owns, while
//                 thread 0 of CTA 0 records it in global memory.  Every wait
//                 is bounded and a give-up leaves rank -1;
//   k_fp_store    the block back into the working copy;
//   k_fp_trsm     the block's pivot rows on the trailing columns: forward
//                 substitution with the block's unit lower multipliers;
//   k_fp_gemm     every other non-pivot row: row -= sum_s L[row][s] U_s on the
//                 trailing columns (64 x 64 output tiles, the <= 32 pivot rows
//                 and multipliers staged in shared memory; for p < 2^16 the
//                 products are summed in 64 bits and reduced once);
//   k_fp_outputs  L and E by position from the working copy.
// Residue arithmetic: a product of two residues (< 2^62) is reduced with a
// floating-point estimate of the quotient (exact within one step for every
// p < 2^31) and one correction each way; beta^-1 = beta^(p-2) (Fermat).
#include <climits>

#include "../../include/gf2.h"
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr int kFpB = 32;           // columns per block column
constexpr int kFpThreads = 256;
constexpr int kFpMaxRowsPerCta = 1024;  // rows one panel CTA keeps in shared memory (128 KB of the block)

struct FpCtx {
    uint32_t *W;        // [n][ldw] working copy, row-major by storage row
    int64_t ldw;
    uint32_t *P;        // [kFpB][n] the current block column, column-major
    int32_t *perm;      // [n] position -> storage row
    int32_t *pos;       // [n] storage row -> position
    int32_t *piv;       // [n] storage row -> its pivot index, or -1
    int32_t *pivcols;   // [k] pivot columns (-1 past the rank)
    int32_t *rank;      // [0] pivots so far, [1] pivots before the current block column
    unsigned long long *found;  // [kFpB] per block column: (position << 32 | row) of its pivot, ~0 = none
    uint32_t *cand;     // [2][grid][kFpB] per column parity and panel CTA: the block entries of its candidate
                        // row (two slots: a CTA writes the next column's while others may still read this one's)
    uint32_t *sync;     // [0] barrier count (zeroed before every panel launch), [1] error word
    int32_t n, m, k;
    uint32_t p;
    double pinv;        // 1.0 / p
    uint32_t two64;     // 2^64 mod p
    uint32_t wait_limit;
};

// x mod p for x < 2^62 (a product of two residues, or a sum of at most 32
// residues): the quotient estimate x * (1/p) in doubles is within one of the
// true quotient (relative error about 2^-52 on a quotient below 2^40 when
// p >= 2^22; x itself exact in a double when p < 2^26), fixed by one step
// each way.
__device__ __forceinline__ uint32_t mod_p(uint64_t x, uint32_t p, double pinv)
{
    const uint64_t q = (uint64_t)((double)x * pinv);
    int64_t r = (int64_t)(x - q * (uint64_t)p);
    if (r < 0) r += p;
    if (r >= (int64_t)p) r -= p;
    return (uint32_t)r;
}

__device__ __forceinline__ uint32_t mul_p(uint32_t a, uint32_t b, uint32_t p, double pinv)
{
    return mod_p((uint64_t)a * b, p, pinv);
}

__device__ __forceinline__ uint32_t sub_p(uint32_t a, uint32_t b, uint32_t p) { return a >= b ? a - b : a + (p - b); }

// beta^(p-2) mod p: the inverse of a nonzero residue (Fermat)
__device__ uint32_t inv_p(uint32_t beta, uint32_t p, double pinv)
{
    uint32_t r = 1, b = beta, e = p - 2;
    while (e) {
        if (e & 1) r = mul_p(r, b, p, pinv);
        b = mul_p(b, b, p, pinv);
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *q)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
    return v;
}

// Grid-wide barrier of the cooperative panel launch; false (in every thread)
// once any CTA has given up waiting.
__device__ bool fp_barrier(const FpCtx &c, uint32_t &epoch, int *s_ok)
{
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c.sync, 1u);
        const uint32_t target = epoch * gridDim.x;
        uint32_t it = 0;
        while (ld_acquire_u32(c.sync) < target) {
            if (ld_acquire_u32(c.sync + 1) & 1u) break;
            if (++it > c.wait_limit) {
                atomicOr(c.sync + 1, 1u);
                break;
            }
            __nanosleep(64);
        }
        *s_ok = (ld_acquire_u32(c.sync + 1) & 1u) == 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// A (row-major, lda) -> W; entries >= p flag *bad; positions, pivot marks
__global__ void k_fp_ingest(const uint32_t *__restrict__ A, int64_t lda, FpCtx c, uint32_t *bad)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)c.n * c.m;
    if (e < c.n) {
        c.perm[e] = (int32_t)e;
        c.pos[e] = (int32_t)e;
        c.piv[e] = -1;
    }
    if (e < c.k) c.pivcols[e] = -1;
    if (e >= total) return;
    const int64_t i = e / c.m, j = e % c.m;
    const uint32_t v = A[i * lda + j];
    if (v >= c.p) atomicOr(bad, 1u);
    c.W[i * c.ldw + j] = v;
}

// the block column [j0, j0 + bw) of every row into P (column-major); the
// per-column pivot slots to "none"
__global__ void k_fp_load(FpCtx c, int j0, int bw)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kFpB) c.found[e] = ~0ull;
    if (e >= (int64_t)c.n * bw) return;
    const int cc = (int)(e / c.n), i = (int)(e % c.n);
    c.P[(int64_t)cc * c.n + i] = c.W[(int64_t)i * c.ldw + j0 + cc];
}

__global__ void k_fp_store(FpCtx c, int j0, int bw)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)c.n * bw) return;
    const int cc = (int)(e / c.n), i = (int)(e % c.n);
    c.W[(int64_t)i * c.ldw + j0 + cc] = c.P[(int64_t)cc * c.n + i];
}

// The pivot steps of the block column [j0, j0 + bw) (cooperative launch).
// CTA b owns the rows [b rpc, (b+1) rpc): their block entries, pivot marks
// and positions live in its shared memory for the whole launch.  Per column,
// one grid barrier: before it every CTA posts its first candidate (the
// smallest (position, row) among its non-pivot rows with a nonzero entry:
// one 64-bit atomicMin) and copies that row's block entries to its slot of
// c.cand; after it every CTA reads the winner's slot (the pivot row), takes
// l = entry beta^-1 for each of its non-pivot rows (stored in place: the L
// entry) and subtracts l x the pivot row from the later block columns, and
// applies the exchange to the rows it owns (the row at position R, found by
// its position, moves to the pivot's; the pivot row takes position R).  The
// global positions, pivot marks and perm are written back at the end, each
// CTA for its own rows, so nothing global is read while another CTA writes it.
__global__ void __launch_bounds__(kFpThreads) k_fp_panel(FpCtx c, int j0, int bw, int rpc)
{
    extern __shared__ uint32_t fp_smem[];
    uint32_t *vals = fp_smem;                                   // [kFpB][rpc]
    int32_t *spiv = reinterpret_cast<int32_t *>(vals + kFpB * rpc);  // [rpc]
    int32_t *spos = spiv + rpc;                                 // [rpc]
    __shared__ uint32_t pivrow[kFpB];
    __shared__ unsigned long long s_min;
    __shared__ uint32_t s_inv;
    __shared__ int s_ok;
    uint32_t epoch = 0;
    const int tid = threadIdx.x;
    const int row0 = blockIdx.x * rpc;
    const int nr = max(0, min(rpc, c.n - row0));
    // the same in every CTA: CTA 0 writes it only at the end, after every CTA
    // has passed the barriers (all read it before their first one)
    int R = c.rank[0];
    if (blockIdx.x == 0 && tid == 0) c.rank[1] = R;
    for (int e = tid; e < bw * nr; e += kFpThreads) {
        const int cc = e / nr, r = e % nr;
        vals[cc * rpc + r] = c.P[(int64_t)cc * c.n + row0 + r];
    }
    for (int r = tid; r < nr; r += kFpThreads) {
        spiv[r] = c.piv[row0 + r];
        spos[r] = c.pos[row0 + r];
    }
    __syncthreads();
    for (int col = 0; col < bw && R < c.k; ++col) {
        // this CTA's first candidate, and its row's block entries to its slot
        unsigned long long best = ~0ull;
        for (int r = tid; r < nr; r += kFpThreads)
            if (spiv[r] < 0 && vals[col * rpc + r] != 0) {
                const unsigned long long key = ((unsigned long long)(uint32_t)spos[r] << 32) | (uint32_t)(row0 + r);
                best = key < best ? key : best;
            }
        if (tid == 0) s_min = ~0ull;
        __syncthreads();
        if (best != ~0ull) atomicMin(&s_min, best);
        __syncthreads();
        const unsigned long long mine = s_min;
        if (mine != ~0ull) {
            const int rl = (int)(mine & 0xFFFFFFFFu) - row0;
            if (tid >= col && tid < bw)
                c.cand[((int64_t)(col & 1) * gridDim.x + blockIdx.x) * kFpB + tid] = vals[tid * rpc + rl];
            if (tid == 0) atomicMin(c.found + col, mine);
        }
        if (!fp_barrier(c, epoch, &s_ok)) return;
        const unsigned long long f = *reinterpret_cast<volatile unsigned long long *>(c.found + col);
        if (f == ~0ull) continue;  // no pivot in this column (every CTA sees the same); nothing moved
        const int fpos = (int)(f >> 32), prow = (int)(f & 0xFFFFFFFFu);
        const int owner = prow / rpc;
        if (tid >= col && tid < bw) pivrow[tid] = __ldcg(c.cand + ((int64_t)(col & 1) * gridDim.x + owner) * kFpB + tid);
        __syncthreads();
        if (tid == 0) s_inv = inv_p(pivrow[col], c.p, c.pinv);
        __syncthreads();
        const uint32_t inv = s_inv;
        const int prl = prow - row0;  // the pivot row's local index (if this CTA owns it)
        for (int r = tid; r < nr; r += kFpThreads) {
            if (r == prl || spiv[r] >= 0) continue;
            const uint32_t a = vals[col * rpc + r];
            if (a == 0) continue;  // multiplier 0: nothing to subtract (the entry already holds it)
            const uint32_t l = mul_p(a, inv, c.p, c.pinv);
            for (int cc = col + 1; cc < bw; ++cc)
                vals[cc * rpc + r] = sub_p(vals[cc * rpc + r], mul_p(l, pivrow[cc], c.p, c.pinv), c.p);
            vals[col * rpc + r] = l;  // the L entry, in place of the eliminated one
        }
        // the exchange of positions R and fpos, on the rows this CTA owns: the
        // row at position R moves to fpos, the pivot row becomes pivot R
        __syncthreads();
        for (int r = tid; r < nr; r += kFpThreads)
            if (r != prl && spos[r] == R) spos[r] = fpos;
        if (tid == 0 && prl >= 0 && prl < nr) {
            spiv[prl] = R;
            spos[prl] = R;
        }
        if (blockIdx.x == 0 && tid == 0) c.pivcols[R] = j0 + col;
        __syncthreads();
        ++R;
    }
    // the block entries, pivot marks and positions of this CTA's rows back
    // to global memory (every position is some row's: perm stays a permutation)
    for (int e = tid; e < bw * nr; e += kFpThreads) {
        const int cc = e / nr, r = e % nr;
        c.P[(int64_t)cc * c.n + row0 + r] = vals[cc * rpc + r];
    }
    for (int r = tid; r < nr; r += kFpThreads) {
        c.piv[row0 + r] = spiv[r];
        c.pos[row0 + r] = spos[r];
        c.perm[spos[r]] = row0 + r;
    }
    if (blockIdx.x == 0 && tid == 0) c.rank[0] = R;
}

// The pivot rows of the block (positions R0 .. R1-1: the ranks before and
// after it) on the trailing columns [jt, m): forward substitution with their
// unit lower multipliers, one thread per column.
__global__ void k_fp_trsm(FpCtx c, int jt)
{
    const int col = jt + blockIdx.x * blockDim.x + threadIdx.x;
    const int R0 = c.rank[1], R1 = c.rank[0];
    if (col >= c.m) return;
    for (int t = R0 + 1; t < R1; ++t) {
        const int64_t rt = c.perm[t];
        uint32_t x = c.W[rt * c.ldw + col];
        for (int s = R0; s < t; ++s) {
            const int64_t rs = c.perm[s];
            const uint32_t l = c.W[rt * c.ldw + c.pivcols[s]];
            if (l) x = sub_p(x, mul_p(l, c.W[rs * c.ldw + col], c.p, c.pinv), c.p);
        }
        c.W[rt * c.ldw + col] = x;
    }
}

// Every non-pivot row i: W[i][col] -= sum_s W[i][pivcol_s] W[row_s][col] over
// the block's pivots s (positions R0.. rank-1), col in [jt, m).  64 x 64
// output tiles by storage row; the multipliers and pivot rows in shared memory.
// SMALL (p < 2^16): a product of two residues is below 2^32, so the <= 32
// products of an output add up in 64 bits and are reduced once.  Otherwise
// the products (< 2^62) add up in 64 bits with a count of the wrap-arounds
// (at most 31), and the sum is reduced once as hi 2^64 + lo.
template <bool SMALL>
__global__ void __launch_bounds__(kFpThreads) k_fp_gemm(FpCtx c, int jt)
{
    __shared__ uint32_t sL[64][kFpB + 1];
    __shared__ uint32_t sU[kFpB][64];
    __shared__ int sRow[64];
    const int R0 = c.rank[1], R1 = c.rank[0];
    const int kb = R1 - R0;
    if (kb <= 0) return;
    const int row0 = blockIdx.y * 64, col0 = jt + blockIdx.x * 64;
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int i = row0 + tid;
        sRow[tid] = (i < c.n && c.piv[i] < 0) ? i : -1;
    }
    __syncthreads();
    for (int e = tid; e < 64 * kFpB; e += kFpThreads) {
        const int r = e / kFpB, s = e % kFpB;
        uint32_t v = 0;
        if (s < kb && sRow[r] >= 0) v = c.W[(int64_t)sRow[r] * c.ldw + c.pivcols[R0 + s]];
        sL[r][s] = v;
    }
    for (int e = tid; e < kFpB * 64; e += kFpThreads) {
        const int s = e / 64, cc = e % 64;
        uint32_t v = 0;
        if (s < kb && col0 + cc < c.m) v = c.W[(int64_t)c.perm[R0 + s] * c.ldw + col0 + cc];
        sU[s][cc] = v;
    }
    __syncthreads();
    // thread -> 16 outputs: column tid % 64, rows tid / 64 + 4 u
    const int cc = tid % 64;
    if (col0 + cc >= c.m) return;
    for (int u = 0; u < 16; ++u) {
        const int r = tid / 64 + 4 * u;
        const int i = sRow[r];
        if (i < 0) continue;
        uint64_t acc = 0;  // at most 32 residues < 2^31 (or products < 2^32): no overflow
        uint32_t hi = 0;
        if (SMALL) {
            for (int s = 0; s < kb; ++s) acc += (uint64_t)sL[r][s] * sU[s][cc];
        } else {
            for (int s = 0; s < kb; ++s) {
                const uint64_t prod = (uint64_t)sL[r][s] * sU[s][cc];
                acc += prod;
                hi += acc < prod;
            }
        }
        if (acc | hi) {
            uint32_t v = mod_p(acc, c.p, c.pinv);
            if (!SMALL && hi) v = mod_p((uint64_t)v + (uint64_t)hi * c.two64, c.p, c.pinv);
            uint32_t *w = c.W + (int64_t)i * c.ldw + col0 + cc;
            *w = sub_p(*w, v, c.p);
        }
    }
}

// L (n x k, by position, unit diagonal, row-major with ldl) and E (k x m,
// row-major with lde) from the working copy; pivot columns past the rank -1
// (already), rank to the caller's word.
__global__ void k_fp_outputs(FpCtx c, uint32_t *L, int64_t ldl, uint32_t *E, int64_t lde, int64_t *rank_out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // a panel launch whose barrier gave up leaves rank -1 (the other outputs zero)
    const int r = (c.sync[1] & 1u) ? -1 : c.rank[0];
    if (e == 0 && rank_out) *rank_out = r;
    if (L && e < (int64_t)c.n * c.k) {
        const int pos = (int)(e / c.k), t = (int)(e % c.k);
        uint32_t v = 0;
        if (t < r) v = pos == t ? 1u : (pos > t ? c.W[(int64_t)c.perm[pos] * c.ldw + c.pivcols[t]] : 0u);
        L[(int64_t)pos * ldl + t] = v;
    }
    if (E && e < (int64_t)c.k * c.m) {
        const int t = (int)(e / c.m), col = (int)(e % c.m);
        uint32_t v = 0;
        if (t < r && col >= c.pivcols[t]) v = c.W[(int64_t)c.perm[t] * c.ldw + col];
        E[(int64_t)t * lde + col] = v;
    }
}

unsigned blocks_for(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

}  // namespace

size_t fp_workspace_bytes(int64_t n, int64_t m)
{
    const int64_t k = n < m ? n : m;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al((size_t)n * m * 4) + al((size_t)kFpB * n * 4) + 3 * al((size_t)n * 4) + al((size_t)(k > 0 ? k : 1) * 4) +
           al(8) + al(kFpB * 8) + al(16) + al(4) + al((size_t)2 * 1024 * kFpB * 4);
}

int fp_decompose(const uint32_t *A, int64_t lda, int64_t n, int64_t m, uint32_t p, int32_t *perm, int32_t *pivcols,
                 int64_t *rank, uint32_t *L, int64_t ldl, uint32_t *E, int64_t lde, bool check, void *ws,
                 uint32_t wait_limit, cudaStream_t s)
{
    const int64_t k = n < m ? n : m;
    char *b = static_cast<char *>(ws);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    FpCtx c{};
    c.W = reinterpret_cast<uint32_t *>(b); b += al((size_t)n * m * 4);
    c.P = reinterpret_cast<uint32_t *>(b); b += al((size_t)kFpB * n * 4);
    c.perm = perm;
    c.pos = reinterpret_cast<int32_t *>(b); b += al((size_t)n * 4);
    c.piv = reinterpret_cast<int32_t *>(b); b += al((size_t)n * 4);
    b += al((size_t)n * 4);  // (reserved)
    c.pivcols = pivcols;
    b += al((size_t)(k > 0 ? k : 1) * 4);
    c.rank = reinterpret_cast<int32_t *>(b); b += al(8);
    c.found = reinterpret_cast<unsigned long long *>(b); b += al(kFpB * 8);
    c.sync = reinterpret_cast<uint32_t *>(b); b += al(16);
    uint32_t *bad = reinterpret_cast<uint32_t *>(b); b += al(4);
    c.cand = reinterpret_cast<uint32_t *>(b);  // room for 2 x 1024 CTAs
    c.ldw = m;
    c.n = (int32_t)n;
    c.m = (int32_t)m;
    c.k = (int32_t)k;
    c.p = p;
    c.pinv = 1.0 / (double)p;
    c.two64 = (uint32_t)((((unsigned __int128)1) << 64) % p);
    c.wait_limit = wait_limit;

    // the panel launch: one CTA per SM at most, rpc rows each in shared memory
    int dev = 0, sms = 1, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
        return GF2_ERR_CUDA;
    if (sms > 1024) sms = 1024;
    int grid = (int)((n + kFpThreads - 1) / kFpThreads);  // at least a row per thread
    grid = grid < 1 ? 1 : (grid > sms ? sms : grid);
    const int rpc = (int)((n + grid - 1) / grid);
    if (rpc > kFpMaxRowsPerCta) return GF2_ERR_UNSUPPORTED;
    const size_t smem = (size_t)rpc * (kFpB + 2) * 4;
    if (cudaFuncSetAttribute(k_fp_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp_panel, kFpThreads, smem) != cudaSuccess)
        return GF2_ERR_CUDA;
    if (!coop || per_sm < 1) return GF2_ERR_UNSUPPORTED;

    if (cudaMemsetAsync(c.rank, 0, 8, s) != cudaSuccess || cudaMemsetAsync(c.sync, 0, 16, s) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, 4, s) != cudaSuccess)
        return GF2_ERR_CUDA;
    int64_t init = (int64_t)n * m;
    if (init < n) init = n;
    if (init < 1) init = 1;
    k_fp_ingest<<<blocks_for(init, 256), 256, 0, s>>>(A, lda, c, bad);
    if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
    if (check) {
        uint32_t h = 0;
        if (cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return GF2_ERR_CUDA;
        if (h) return GF2_ERR_ARG;
    }
    for (int64_t j0 = 0; j0 < m; j0 += kFpB) {
        const int bw = (int)(m - j0 < kFpB ? m - j0 : kFpB);
        const int64_t lw = (int64_t)n * bw > kFpB ? (int64_t)n * bw : kFpB;
        k_fp_load<<<blocks_for(lw, 256), 256, 0, s>>>(c, (int)j0, bw);
        // the grid barrier counts from zero in every panel launch (the error word stays)
        if (cudaMemsetAsync(c.sync, 0, sizeof(uint32_t), s) != cudaSuccess) return GF2_ERR_CUDA;
        FpCtx arg = c;
        int j0i = (int)j0, bwi = bw, rpci = rpc;
        void *args[] = {&arg, &j0i, &bwi, &rpci};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_fp_panel), dim3(grid), dim3(kFpThreads), args,
                                        smem, s) != cudaSuccess)
            return GF2_ERR_CUDA;
        k_fp_store<<<blocks_for((int64_t)n * bw, 256), 256, 0, s>>>(c, (int)j0, bw);
        const int jt = (int)(j0 + bw);
        if (jt < m) {
            k_fp_trsm<<<blocks_for(m - jt, 128), 128, 0, s>>>(c, jt);
            const dim3 g((unsigned)((m - jt + 63) / 64), (unsigned)((n + 63) / 64));
            if (p < 65536u)
                k_fp_gemm<true><<<g, kFpThreads, 0, s>>>(c, jt);
            else
                k_fp_gemm<false><<<g, kFpThreads, 0, s>>>(c, jt);
        }
        if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
    }
    k_fp_outputs<<<blocks_for(((int64_t)n * k > k * m ? (int64_t)n * k : k * m) + 1, 256), 256, 0, s>>>(c, L, ldl, E, lde,
                                                                                                        rank);
    if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
    return GF2_OK;
}

}  // namespace gf2
