// Transpose of an n x m matrix over F2 in column blocks: T = A^T (m x n),
// word (j, p) of T at T[p * ldt + j], bit t = A[64p + t][j].  One warp per
// 64 x 64-bit tile: lane l loads rows l and l + 32 of the tile (one word of
// A's column block each, consecutive lanes on consecutive rows), a register
// transpose across the warp turns them into the tile's columns, and lane l
// stores T's rows 64q + l and 64q + l + 32 (again consecutive).  Rows of A
// past n read as zero; rows of T past m (A's padding columns) are not
// written.  Used by gf2_rank for n < m: rank(A) = rank(A^T), and the
// decomposition is cheaper with more rows than columns (Section 7).
#include "panel_core.cuh"

namespace gf2 {
namespace {

__global__ void __launch_bounds__(256) k_transpose_bits(const uint64_t *__restrict__ A, int64_t lda, int64_t n,
                                                        int64_t m, uint64_t *__restrict__ T, int64_t ldt)
{
    const int lane = threadIdx.x & 31;
    const int64_t pw = (n + 63) / 64, qw = (m + 63) / 64, tiles = pw * qw;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; tile < tiles; tile += warps) {
        const int64_t p = tile % pw, q = tile / pw;  // row block of A, column block of A
        const int64_t r0 = 64 * p + lane, r1 = r0 + 32;
        uint64_t a[2];
        a[0] = r0 < n ? A[q * lda + r0] : 0;
        a[1] = r1 < n ? A[q * lda + r1] : 0;
        transpose64(a, lane);  // a[h] = column lane + 32h of the tile
        const int64_t j0 = 64 * q + lane, j1 = j0 + 32;
        if (j0 < m) T[p * ldt + j0] = a[0];
        if (j1 < m) T[p * ldt + j1] = a[1];
    }
}

}  // namespace

cudaError_t launch_transpose_bits(const uint64_t *A, int64_t lda, int64_t n, int64_t m, uint64_t *T, int64_t ldt,
                                  cudaStream_t s)
{
    if (n <= 0 || m <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t tiles = ((n + 63) / 64) * ((m + 63) / 64);
    int64_t grid = (tiles + 7) / 8;
    if (grid > 16 * (int64_t)sms) grid = 16 * (int64_t)sms;
    k_transpose_bits<<<(unsigned)grid, 256, 0, s>>>(A, lda, n, m, T, ldt);
    return cudaGetLastError();
}

}  // namespace gf2
