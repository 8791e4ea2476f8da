// The product C = A B over F2 on the tensor cores (Section 1's product; the
// alternative to the Four Russians kernel for a long inner dimension).
//
// Every entry of A and B becomes an e4m3 byte, 1.0 (0x38) or 0, and an
// mma.sync m16n8k32 e4m3 x e4m3 -> f32 product sums them; entry (i, j) of C
// over F2 is the lowest bit of the integer sum.  The accumulators are folded
// into integer parity bits every kFoldTiles k-tiles (4096 of the inner
// dimension) and restarted from zero, so no partial sum exceeds 4096 = 2^12:
// its lowest bit survives even an accumulation that keeps only about 13
// significant bits, whatever the tensor pipe's internal precision.  Because the
// whole inner dimension is accumulated before anything is read back, the
// unpacking (one bit per output) costs little; for the rank-64/128 updates of
// the decomposition it would cost as much as the Four Russians lookups, so
// the decomposition does not use this path.
//
// Layout: A8 = A expanded to bytes, n_pad x k_pad, row-major (k contiguous);
// B8 = B transposed and expanded, m_pad x k_pad, row-major (k contiguous), so
// both operands are K-major as the mma wants.  CTA tile 128 x 128 with
// k-steps of 128 bytes, three cp.async stages in shared memory with the
// 16-byte chunks XOR-swizzled by row (conflict-free ldmatrix), 8 warps of
// 64 x 32 each.  The epilogue packs the parities of 32 columns into one
// 32-bit half of an output word of C's column blocks.
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 128;  // CTA tile (rows, cols, k bytes)
constexpr int kStages = 3;
constexpr int kMmaThreads = 256;
constexpr int kTileBytes = kBM * kBK;  // one operand tile of one stage (16 KB)
constexpr int kMmaSmem = kStages * 2 * kTileBytes;
constexpr uint32_t kOne = 0x38;  // 1.0 in e4m3
constexpr int kFoldTiles = 32;   // k-tiles between parity folds (32 x 128 = 4096 of the inner dimension)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk c of row r in a swizzled 128 x 128-byte tile
__device__ __forceinline__ int swz(int r, int c) { return r * kBK + ((c ^ (r & 7)) << 4); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_e4m3(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16 bits -> 16 e4m3 bytes (bit b -> byte b)
__device__ __forceinline__ uint4 expand16(uint32_t bits)
{
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t x = bits >> (4 * q);
        w[q] = ((x & 1) ? kOne : 0) | ((x & 2) ? kOne << 8 : 0) | ((x & 4) ? kOne << 16 : 0) | ((x & 8) ? kOne << 24 : 0);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// A (column blocks of bits) -> A8 rows: A8[i][64q + t] = bit t of word (i, q)
__global__ void k_expand_rows(const uint64_t *__restrict__ A, int64_t lda, int n, int kw, int n_pad, int k_pad,
                              uint8_t *__restrict__ A8)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (q, i), i fastest
    const int qn = k_pad / 64;
    if (e >= (int64_t)qn * n_pad) return;
    const int q = (int)(e / n_pad), i = (int)(e % n_pad);
    const uint64_t w = (i < n && q < kw) ? A[(int64_t)q * lda + i] : 0;
    uint4 *dst = reinterpret_cast<uint4 *>(A8 + (int64_t)i * k_pad + 64 * q);
#pragma unroll
    for (int h = 0; h < 4; ++h) dst[h] = expand16((uint32_t)(w >> (16 * h)) & 0xFFFFu);
}

// B (k x m, column blocks of bits) -> B8 = B^T rows: B8[j][r] = entry (r, j)
__global__ void k_expand_cols(const uint64_t *__restrict__ B, int64_t ldb, int k, int m, int m_pad, int k_pad,
                              uint8_t *__restrict__ B8)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (16-row group g, column j), j fastest
    const int ng = k_pad / 16;
    if (e >= (int64_t)ng * m_pad) return;
    const int g = (int)(e / m_pad), j = (int)(e % m_pad);
    uint32_t bits = 0;
    if (j < m) {
        const uint64_t *col = B + (int64_t)(j >> 6) * ldb;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int r = 16 * g + t;
            if (r < k) bits |= (uint32_t)((col[r] >> (j & 63)) & 1) << t;
        }
    }
    *reinterpret_cast<uint4 *>(B8 + (int64_t)j * k_pad + 16 * g) = expand16(bits);
}

__global__ void __launch_bounds__(kMmaThreads, 1) k_mma8(const uint8_t *__restrict__ A8, const uint8_t *__restrict__ B8,
                                                         int k_pad, uint64_t *__restrict__ C, int64_t ldc, int n, int m,
                                                         int accumulate)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;  // warp tile: rows 64 wm.., cols 32 wn..
    const int row0 = blockIdx.y * kBM, col0 = blockIdx.x * kBN;
    const uint8_t *Ag = A8 + (int64_t)row0 * k_pad;
    const uint8_t *Bg = B8 + (int64_t)col0 * k_pad;
    const int ktiles = k_pad / kBK;

    auto stage_a = [&](int s) { return smem + s * 2 * kTileBytes; };
    auto stage_b = [&](int s) { return smem + s * 2 * kTileBytes + kTileBytes; };
    // each thread copies 4 chunks of A and 4 of B per stage (128 rows x 8 chunks)
    auto load_stage = [&](int s, int kt) {
        uint8_t *sa = stage_a(s), *sb = stage_b(s);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = tid + u * kMmaThreads, r = idx >> 3, cidx = idx & 7;
            cp_async16(smem_addr(sa + swz(r, cidx)), Ag + (int64_t)r * k_pad + kt * kBK + 16 * cidx);
            cp_async16(smem_addr(sb + swz(r, cidx)), Bg + (int64_t)r * k_pad + kt * kBK + 16 * cidx);
        }
    };

    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    // parities of this lane's sums so far, in the epilogue's bit positions:
    // par[mt][hr] bit 8 nt + 2 t + c = lowest bit of acc[mt][nt][2 hr + c]
    const int t = lane & 3;
    uint32_t par[4][2] = {};
    auto fold = [&]() {
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        par[mt][hr] ^= (uint32_t)(__float2int_rn(acc[mt][nt][2 * hr + c]) & 1) << (8 * nt + 2 * t + c);
                        acc[mt][nt][2 * hr + c] = 0.f;
                    }
    };

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < ktiles) load_stage(s, s);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // ldmatrix row / chunk of this lane: A (x4: rows 0-7, 8-15 at byte 0, then at byte 16)
    const int a_row = (lane & 7) + ((lane >> 3) & 1) * 8, a_half = lane >> 4;
    // B (x4: two n8 tiles: rows 0-7 then 8-15; bytes 0 and 16 of each)
    const int b_row = (lane & 7) + ((lane >> 4) & 1) * 8, b_half = (lane >> 3) & 1;
    for (int kt = 0; kt < ktiles; ++kt) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 2) : "memory");
        __syncthreads();
        {
            const int nk = kt + kStages - 1;
            if (nk < ktiles) load_stage(nk % kStages, nk);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        const uint8_t *sa = stage_a(kt % kStages), *sb = stage_b(kt % kStages);
#pragma unroll
        for (int kk = 0; kk < kBK / 32; ++kk) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int r = 64 * wm + 16 * mt + a_row;
                ldsm_x4(smem_addr(sa + swz(r, 2 * kk + a_half)), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const int r = 32 * wn + 16 * np + b_row;
                ldsm_x4(smem_addr(sb + swz(r, 2 * kk + b_half)), bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0],
                        bf[2 * np + 1][1]);
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_e4m3(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
        }
        if ((kt + 1) % kFoldTiles == 0 || kt + 1 == ktiles) fold();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");

    // parities -> 32 columns per row in one 32-bit half word of C
    const int g = lane >> 2;
    const int cbase = col0 + 32 * wn;  // multiple of 32: a low or high half of word cbase / 64
    const int q = cbase >> 6, half = (cbase >> 5) & 1;
    // a half past the last column is still written (zero bits) while its
    // word is one of C's column blocks, so C's padding is never left stale
    const bool col_ok = q < (m + 63) / 64;
    uint32_t *C32 = reinterpret_cast<uint32_t *>(C);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {  // rows g and g + 8 of the m16 tile
            uint32_t bits = par[mt][hr];
            bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
            bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
            const int row = row0 + 64 * wm + 16 * mt + 8 * hr + g;
            if (t == 0 && row < n && col_ok) {
                uint32_t *dst = C32 + 2 * ((int64_t)q * ldc + row) + half;
                *dst = accumulate ? (*dst ^ bits) : bits;
            }
        }
    }
}

// bits beyond the last column in the last column block (rows x 1 words)
__global__ void k_check_last_block(const uint64_t *__restrict__ last, int rows, uint64_t mask, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows && (last[i] & ~mask)) atomicOr(err, 1u);
}

}  // namespace

int64_t mma_pad(int64_t x) { return (x + 127) / 128 * 128; }

cudaError_t launch_check_last_block(const uint64_t *last, int rows, uint64_t mask, uint32_t *err, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_check_last_block<<<(rows + 255) / 256, 256, 0, s>>>(last, rows, mask, err);
    return cudaGetLastError();
}

cudaError_t launch_mma_product(const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb, uint64_t *C,
                               int64_t ldc, int n, int k, int m, int accumulate, uint8_t *A8, uint8_t *B8,
                               cudaStream_t s)
{
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        e = cudaFuncSetAttribute(k_mma8, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    const int n_pad = (int)mma_pad(n), m_pad = (int)mma_pad(m), k_pad = (int)mma_pad(k);
    const int kw = (k + 63) / 64;
    {
        const int64_t total = (int64_t)(k_pad / 64) * n_pad;
        k_expand_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(A, lda, n, kw, n_pad, k_pad, A8);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        const int64_t total = (int64_t)(k_pad / 16) * m_pad;
        k_expand_cols<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(B, ldb, k, m, m_pad, k_pad, B8);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    dim3 grid(m_pad / kBN, n_pad / kBM);
    k_mma8<<<grid, kMmaThreads, kMmaSmem, s>>>(A8, B8, k_pad, C, ldc, n, m, accumulate);
    return cudaGetLastError();
}

}  // namespace gf2
