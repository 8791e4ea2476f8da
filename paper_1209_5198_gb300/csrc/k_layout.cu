// Layout kernels: the boundary's column-block layout (Section 3 of the
// paper: word (i, q) at q*ld + i) to and from the working layouts used
// inside the library (the tiled copy of A of the decomposition, row-major
// operands of the product and the factors), plus the final scalar outputs.
//
// All of them are 32 x 32-word tile transposes through shared memory so that
// both the column-block side (consecutive rows contiguous) and the row-major
// side (consecutive words of a row contiguous) are read and written with
// coalesced accesses.
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr int kT = 32;     // tile edge (words)
constexpr int kTy = 8;     // threads in y; each thread moves kT / kTy words

// A (column blocks, n rows, mu blocks) -> W: row-major with ldw words per
// row, or (TILED) in column tiles of kTileWords words (word q of row i at
// (q/T)*T*n + T*i + q%T, T = kTileWords) with ldw = mu rounded up to T.  Words q >= mu of W are
// written as zero.  Bits beyond the last column of the last block are
// checked against last_mask; any violation sets *err.
template <bool TILED>
__global__ void k_ingest(const uint64_t *__restrict__ A, int64_t lda, int32_t n, int32_t mu,
                         uint64_t last_mask, uint64_t *__restrict__ W, int64_t ldw,
                         int32_t *__restrict__ perm, int32_t *__restrict__ pivpanel,
                         uint32_t *__restrict__ err)
{
    __shared__ uint64_t tile[kT][kT + 1];
    const int i0 = blockIdx.x * kT, q0 = blockIdx.y * kT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int q = q0 + ty + k * kTy, i = i0 + tx;
        uint64_t v = 0;
        if (q < mu && i < n) {
            v = A[(int64_t)q * lda + i];
            if (q == mu - 1) bad |= (v & ~last_mask) != 0;
        }
        tile[ty + k * kTy][tx] = v;
    }
    if (bad && err) atomicOr(err, 1u);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int i = i0 + ty + k * kTy, q = q0 + tx;
        if (i < n && q < ldw) {
            const int64_t o = TILED ? (int64_t)(q / kTileWords) * kTileWords * n + (int64_t)i * kTileWords + (q % kTileWords)
                                    : (int64_t)i * ldw + q;
            W[o] = tile[tx][ty + k * kTy];
        }
    }
    if (blockIdx.y == 0 && ty == 0 && i0 + tx < n) {
        if (perm) perm[i0 + tx] = i0 + tx;
        if (pivpanel) pivpanel[i0 + tx] = 0x7fffffff;
    }
}

// out (column blocks, `rows` rows, `words` blocks) from row-major R, where
// row i of the output is row row_of[i] of R (identity if row_of is null).
__global__ void k_to_colblocks(const uint64_t *__restrict__ R, int64_t ldr,
                               const int32_t *__restrict__ row_of, int32_t rows, int32_t words,
                               uint64_t *__restrict__ out, int64_t ldo)
{
    __shared__ uint64_t tile[kT][kT + 1];
    const int i0 = blockIdx.x * kT, q0 = blockIdx.y * kT;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int i = i0 + ty + k * kTy, q = q0 + tx;
        uint64_t v = 0;
        if (i < rows && q < words) {
            const int64_t src = row_of ? row_of[i] : i;
            v = R[src * ldr + q];
        }
        tile[ty + k * kTy][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int q = q0 + ty + k * kTy, i = i0 + tx;
        if (q < words && i < rows) out[(int64_t)q * ldo + i] = tile[tx][ty + k * kTy];
    }
}

// E (column blocks, kmax rows) from the row-major pivot rows Eint: row t < r
// keeps its words from the block of its pivot on; everything else is zero.
__global__ void k_finish_E(const uint64_t *__restrict__ Eint, int64_t ldw,
                           const int32_t *__restrict__ pivcols, const PanelInfo *__restrict__ last,
                           int32_t kmax, int32_t mu, uint64_t *__restrict__ E, int64_t lde)
{
    __shared__ uint64_t tile[kT][kT + 1];
    const int rank = last->R + last->r;
    const int t0 = blockIdx.x * kT, q0 = blockIdx.y * kT;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int t = t0 + ty + k * kTy, q = q0 + tx;
        uint64_t v = 0;
        if (t < rank && q < mu && q >= (pivcols[t] >> 6)) v = Eint[(int64_t)t * ldw + q];
        tile[ty + k * kTy][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kT / kTy; ++k) {
        const int q = q0 + ty + k * kTy, t = t0 + tx;
        if (q < mu && t < kmax) E[(int64_t)q * lde + t] = tile[tx][ty + k * kTy];
    }
}

__global__ void k_finish_scalars(const PanelInfo *__restrict__ last, int32_t *__restrict__ pivcols,
                                 int32_t kmax, int64_t *__restrict__ rank_out, const int32_t *fail)
{
    const int rank = (fail && *fail) ? -1 : last->R + last->r;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && rank_out) *rank_out = rank;
    if (t < kmax && t >= rank) pivcols[t] = -1;
}

}  // namespace

cudaError_t launch_ingest(const uint64_t *A, int64_t lda, int32_t n, int32_t mu, uint64_t last_mask,
                          uint64_t *W, int64_t ldw, int32_t *perm_identity, int32_t *pivpanel_init,
                          uint32_t *err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    dim3 grid((n + kT - 1) / kT, (unsigned)((ldw + kT - 1) / kT)), block(kT, kTy);
    k_ingest<false><<<grid, block, 0, s>>>(A, lda, n, mu, last_mask, W, ldw, perm_identity, pivpanel_init, err);
    return cudaGetLastError();
}

cudaError_t launch_ingest_tiled(const uint64_t *A, int64_t lda, int32_t n, int32_t mu, uint64_t last_mask,
                                uint64_t *W, int32_t *perm_identity, int32_t *pivpanel_init, uint32_t *err,
                                cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t ldw = ((mu > 0 ? mu : 1) + kTileWords - 1) / kTileWords * kTileWords;
    dim3 grid((n + kT - 1) / kT, (unsigned)((ldw + kT - 1) / kT)), block(kT, kTy);
    k_ingest<true><<<grid, block, 0, s>>>(A, lda, n, mu, last_mask, W, ldw, perm_identity, pivpanel_init, err);
    return cudaGetLastError();
}

cudaError_t launch_colblocks_from_rowmajor(const uint64_t *R, int64_t ldr, const int32_t *row_of,
                                           int32_t rows, int32_t words, uint64_t *out, int64_t ldo,
                                           cudaStream_t s)
{
    if (rows <= 0 || words <= 0) return cudaSuccess;
    dim3 grid((rows + kT - 1) / kT, (words + kT - 1) / kT), block(kT, kTy);
    k_to_colblocks<<<grid, block, 0, s>>>(R, ldr, row_of, rows, words, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_finish_E(const DecompCtx &c, uint64_t *E, int64_t lde, cudaStream_t s)
{
    if (c.kmax <= 0 || c.mu <= 0) return cudaSuccess;
    dim3 grid((c.kmax + kT - 1) / kT, (c.mu + kT - 1) / kT), block(kT, kTy);
    k_finish_E<<<grid, block, 0, s>>>(c.Eint, c.lde, c.pivcols, c.info + (c.mu - 1), c.kmax, c.mu, E, lde);
    return cudaGetLastError();
}

cudaError_t launch_finish_scalars(const DecompCtx &c, int64_t *rank, cudaStream_t s)
{
    const int threads = 256;
    const int blocks = (c.kmax + threads - 1) / threads > 0 ? (c.kmax + threads - 1) / threads : 1;
    k_finish_scalars<<<blocks, threads, 0, s>>>(c.info + (c.mu - 1), c.pivcols, c.kmax, rank, c.fail);
    return cudaGetLastError();
}

}  // namespace gf2
