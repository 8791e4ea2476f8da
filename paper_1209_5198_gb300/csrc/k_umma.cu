// The product C = A B over F2 on the fifth-generation tensor cores
// (tcgen05): the alternative to the Four Russians product for a long inner
// dimension (Section 1's product; Section 6 prices the table method it is
// measured against).
//
// Arithmetic.  Every entry of A and B becomes an e2m1 (fp4) value, 1.0 or 0
// (k_expand_rows: A8 = A; k_expand_cols: B8 = B^T), and tcgen05.mma
// kind::f8f6f4 sums their products into fp32 accumulators in tensor memory;
// entry (i, j) of C over F2 is the lowest bit of the integer sum.  Every
// kUFold stages (4096 of the inner dimension) the epilogue warps read the
// accumulators, fold their lowest bits into packed parity words in
// registers, and the next stage restarts the accumulators from zero, so no
// sum exceeds 4096 = 2^12 and its lowest bit is exact whatever the
// precision the tensor pipe keeps while it accumulates.  The lowest bit of
// an integer-valued float s < 2^23 is the lowest bit of the word of
// s + 2^23 (whose unit in the last place is 1).  The order of the entries
// along the inner dimension is the same permutation for A and B, so it
// does not change any sum.
//
// Data movement.  A8 (n_pad rows) and B8 (m_pad rows) are K-major, two
// entries per byte.  A CTA computes a 128 x 256 tile of C: per stage one TMA
// load brings 128 rows of A8 and one brings 256 rows of B8, 128 entries of
// the inner dimension each, into shared memory as 128-byte rows (the 8-bit
// layout kind::f8f6f4 reads: 8 bytes of packed entries, 8 bytes of gap)
// with the 128-byte swizzle of the tensor core's K-major operand layout
// (8-row atoms of 1024 bytes); four stages ring through an mbarrier
// pipeline.  The tensor maps cover this GPU's memory only (no multicast).
// Warp roles:
//   warp 0 (one thread)  waits until a stage is free, posts its byte count
//                        and issues the two TMA loads;
//   warp 1 (one thread)  allocates 512 tensor-memory columns (two 128 x 256
//                        fp32 accumulators, lane = row, used by alternate
//                        folds), waits until a stage has landed, issues the
//                        four 128 x 256 x 32 MMAs of its 128 entries and
//                        commits them to the stage's "free" barrier (and, at
//                        the end of a fold, to the accumulator's "full"
//                        barrier); a fold waits only until the epilogue has
//                        read the accumulator two folds back;
//   warps 2-5            the epilogue: warp w reads tensor-memory lanes
//                        32 (w % 4).. (the lanes its warp rank may access),
//                        32 columns per tcgen05.ld, keeps the parities of its
//                        row's 256 columns in 8 words, and after the last
//                        fold writes (or XORs) the row's 4 words of C.
// Every wait polls a bounded number of times; a CTA that gives up sets the
// launch's error word (GF2_ERR_TIMEOUT for the caller), waits (bounded) for
// the copies it issued, frees its tensor memory and returns, and the CTAs
// that start after it do nothing.
//
// Persistent: one CTA per SM walks the tiles b, b + gridDim.x, ...;
// tiles are numbered down groups of kUGroup row tiles, so the CTAs that run
// together share their rows of A and columns of B in L2.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "gf2_internal.cuh"

namespace gf2 {
namespace {

// Operand format: 1 = e2m1 (fp4) entries packed two per byte in global
// memory and loaded by TMA into the 8-bit-per-entry layout that kind::f8f6f4
// reads (16 packed entries per 16-byte chunk, then 8 bytes of gap), which
// halves the operand traffic; 0 = e4m3 bytes.  Both run at the same MMA rate.
#ifndef GF2_UMMA_FP4
#define GF2_UMMA_FP4 1
#endif
constexpr bool kUFp4 = GF2_UMMA_FP4 != 0;

constexpr int kUM = 128;                       // rows of a CTA tile (tensor-memory lanes)
constexpr int kUN = 256;                       // columns of a CTA tile (fp32 tensor-memory columns)
constexpr int kUK = 128;                       // inner-dimension bytes per stage (one swizzle row)
constexpr int kUStages = 4;
constexpr int kUFold = 32;                     // stages between parity folds: 4096 of the inner dimension
constexpr int kUGroup = 16;                    // row tiles per rasterisation group
constexpr int kUThreads = 192;                 // 6 warps: TMA, MMA, 4 x epilogue
constexpr int kUABytes = kUM * kUK;            // 16 KB
constexpr int kUBBytes = kUN * kUK;            // 32 KB
constexpr int kUStageBytes = kUABytes + kUBBytes;
// bytes a stage's two TMA loads transfer (the mbarrier's transaction count):
// the packed e2m1 entries count once, the gaps of their shared-memory layout not
constexpr int kUTxBytes = kUFp4 ? kUStageBytes / 2 : kUStageBytes;
constexpr int kUBarBytes = 256;
constexpr int kUSmem = 1024 + kUStages * kUStageBytes + kUBarBytes;  // 1024: alignment slack
constexpr uint32_t kUTmemCols = 2 * kUN;           // two 128 x 256 fp32 accumulators
constexpr uint32_t kUSpinLimit = 1u << 20;     // polls of one wait before the CTA gives up

static_assert(kUSmem <= 227 * 1024, "shared memory of one CTA");

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the completion of the phase of parity `parity`; false once the
// poll limit is reached, another role of the CTA has given up (*fail) or
// another CTA of the launch has (*gerr, the launch's error word).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t *fail,
                                          const volatile uint32_t *gerr)
{
    for (uint32_t it = 0; it < kUSpinLimit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 63 && (*fail || *gerr)) {
            *fail = 1;
            return false;
        }
    }
    *fail = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory operand descriptor of a K-major tile in the 128-byte
// swizzle layout: start address / 16 (bits 0-13), leading byte offset
// (unused for this layout, 1), stride byte offset = 1024 / 16 between 8-row
// atoms (bits 32-45), descriptor version 1 (bits 46-47), layout 2 = 128-byte
// swizzle (bits 61-63).  The tile starts on a 1024-byte boundary; a step of
// 32 bytes along K inside the swizzle row moves the start address only.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f8f6f4: D fp32 (bits 4-5 = 1), A and B
// e2m1 = 5 or e4m3 = 0 (bits 7-9, 10-12), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kUFmt = kUFp4 ? 5u : 0u;
constexpr uint32_t kUIdesc =
    (1u << 4) | (kUFmt << 7) | (kUFmt << 10) | ((uint32_t)(kUN >> 3) << 17) | ((uint32_t)(kUM >> 4) << 24);

__device__ __forceinline__ void umma_f8(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kUIdesc), "r"(accumulate));
}

// arrives on the barrier once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// lowest bits of 32 integer-valued fp32 sums (< 2^23), bit c from v[c]
__device__ __forceinline__ uint32_t parities32(const uint32_t (&v)[32])
{
    uint32_t bits = 0;
#pragma unroll
    for (int c = 0; c < 32; ++c) bits |= (__float_as_uint(__uint_as_float(v[c]) + 8388608.0f) & 1u) << c;
    return bits;
}

// tile t of the launch -> (row tile, column tile), in groups of kUGroup row tiles
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int &tm, int &tn)
{
    const int group = t / (kUGroup * tiles_n);
    const int first_m = group * kUGroup;
    const int gm = min(kUGroup, tiles_m - first_m);
    const int within = t - group * kUGroup * tiles_n;
    tm = first_m + within % gm;
    tn = within / gm;
}

// Persistent: CTA b computes tiles b, b + gridDim.x, ...  The stage ring and
// the two accumulator buffers run on counters that continue across tiles,
// so the loads and MMAs of a tile overlap the last fold and the stores of
// the one before.
__global__ void __launch_bounds__(kUThreads, 1)
    k_umma(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int ktiles, int tiles_m,
           int tiles_n, uint64_t *__restrict__ C, int64_t ldc, int n, int mw, int accumulate, uint32_t *err)
{
    // a CTA of a launch in which another CTA has given up does nothing
    if (*reinterpret_cast<volatile uint32_t *>(err)) return;
    extern __shared__ uint8_t usmem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(usmem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kUStages * kUStageBytes);
    // barriers: full[s] (the stage's bytes landed), empty[s] (its MMAs are
    // done), acc_full[b] (a fold's MMAs into accumulator b are done),
    // acc_empty[b] (the epilogue has read accumulator b), drain (every MMA
    // issued is done, after a give-up); then the tensor-memory address and
    // the give-up flag
    const uint32_t full0 = su32(bars), empty0 = su32(bars + kUStages);
    const uint32_t accf0 = su32(bars + 2 * kUStages), acce0 = su32(bars + 2 * kUStages + 2);
    const uint32_t drain = su32(bars + 2 * kUStages + 4);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2 * kUStages + 5);
    volatile uint32_t *fail = s_tmem + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = tiles_m * tiles_n;
    const int nfold = (ktiles + kUFold - 1) / kUFold;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kUStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);
        }
        mbar_init(drain, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                     "r"(kUTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0 && lane == 0) {
        int64_t g = 0;  // stages issued by this CTA
        for (int t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            for (int kt = 0; kt < ktiles; ++kt, ++g) {
                const int s = (int)(g % kUStages);
                const uint32_t use = (uint32_t)(g / kUStages);
                if (use > 0 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1, fail, err)) break;
                const uint32_t sa = su32(base + s * kUStageBytes);
                mbar_expect_tx(full0 + 8 * s, kUTxBytes);
                tma_load_2d(sa, &ta, kt * kUK, tm * kUM, full0 + 8 * s);
                tma_load_2d(sa + kUABytes, &tb, kt * kUK, tn * kUN, full0 + 8 * s);
            }
        }
        if (*fail) {
            // let the copies in flight land before the CTA leaves (bounded)
            for (int64_t h = g > kUStages ? g - kUStages : 0; h < g; ++h) {
                const uint32_t bar = full0 + 8 * (int)(h % kUStages), par = (uint32_t)(h / kUStages) & 1;
                for (uint32_t it = 0; it < kUSpinLimit && !mbar_test(bar, par); ++it) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        int64_t g = 0, F = 0;  // stages consumed, folds started
        for (int t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
            for (int kt = 0; kt < ktiles; ++kt, ++g) {
                const int s = (int)(g % kUStages);
                const int kf = kt % kUFold;
                const uint32_t b = (uint32_t)(F & 1);
                if (kf == 0 && F >= 2) {
                    // accumulator b was last used by fold F - 2: wait until it has been read
                    if (!mbar_wait(acce0 + 8 * b, (uint32_t)((F >> 1) - 1) & 1, fail, err)) break;
                    tc_fence_after();
                }
                if (!mbar_wait(full0 + 8 * s, (uint32_t)(g / kUStages) & 1, fail, err)) break;
                tc_fence_after();
                const uint32_t sa = su32(base + s * kUStageBytes), sb = sa + kUABytes;
                const uint32_t d = tmem + b * (uint32_t)kUN;
#pragma unroll
                for (int kk = 0; kk < kUK / 32; ++kk)
                    umma_f8(d, sw128_desc(sa + 32 * kk), sw128_desc(sb + 32 * kk), (kf | kk) != 0);
                umma_commit(empty0 + 8 * s);
                if (kf == kUFold - 1 || kt == ktiles - 1) {
                    umma_commit(accf0 + 8 * b);
                    ++F;
                }
            }
        }
        if (*fail) {
            // the MMAs in flight finish before the tensor memory is freed (bounded)
            umma_commit(drain);
            for (uint32_t it = 0; it < kUSpinLimit && !mbar_test(drain, 0); ++it) {
            }
        }
    } else if (warp >= 2) {
        const int q = warp & 3;  // tensor-memory lanes 32 q .. 32 q + 31
        int64_t F = 0;           // folds read
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            uint32_t par[kUN / 32] = {};
            for (int f = 0; f < nfold; ++f, ++F) {
                const uint32_t b = (uint32_t)(F & 1);
                if (!mbar_wait(accf0 + 8 * b, (uint32_t)(F >> 1) & 1, fail, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < kUN / 32; ++c) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * (uint32_t)kUN + (uint32_t)(32 * c), v);
                    par[c] ^= parities32(v);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * b);
            }
            const int row = tm * kUM + 32 * q + lane;
            if (ok && row < n) {
#pragma unroll
                for (int w = 0; w < kUN / 64; ++w) {
                    const int qw = tn * (kUN / 64) + w;
                    if (qw < mw) {
                        const uint64_t v = (uint64_t)par[2 * w] | ((uint64_t)par[2 * w + 1] << 32);
                        uint64_t *dst = C + (int64_t)qw * ldc + row;
                        *dst = accumulate ? (*dst ^ v) : v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUTmemCols) : "memory");
    }
    if (threadIdx.x == 0 && *fail) atomicOr(err, 1u);
}

// ---------------------------------------------------------------- operands
constexpr uint32_t kOne = 0x38;  // 1.0 in e4m3
constexpr uint32_t kOne4 = 0x2;  // 1.0 in e2m1

// bytes of a K-contiguous operand row of k_pad entries in global memory
__host__ __device__ constexpr int64_t urow_bytes(int64_t k_pad) { return kUFp4 ? k_pad / 2 : k_pad; }

// 16 bits -> 16 entries (bit b -> entry b): 16 e4m3 bytes, or 16 e2m1
// nibbles (entry 2i in the low nibble of byte i) in the low 8 of 16 bytes
__device__ __forceinline__ uint4 expand16(uint32_t bits)
{
    uint32_t w[4];
    if (kUFp4) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) v |= ((bits >> (8 * h + i)) & 1u) * (kOne4 << (4 * i));
            w[h] = v;
        }
        w[2] = w[3] = 0;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t x = bits >> (4 * q);
            w[q] = ((x & 1) ? kOne : 0) | ((x & 2) ? kOne << 8 : 0) | ((x & 4) ? kOne << 16 : 0) |
                   ((x & 8) ? kOne << 24 : 0);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// stores the 16 entries of expand16 at byte offset 16 g (e4m3) or 8 g (e2m1) of a row
__device__ __forceinline__ void store16(uint8_t *row, int g, uint4 v)
{
    if (kUFp4)
        *reinterpret_cast<uint2 *>(row + 8 * (int64_t)g) = make_uint2(v.x, v.y);
    else
        *reinterpret_cast<uint4 *>(row + 16 * (int64_t)g) = v;
}

// A (column blocks of bits) -> A8 rows: entry (i, 64q + t) = bit t of word (i, q)
__global__ void k_expand_rows(const uint64_t *__restrict__ A, int64_t lda, int n, int kw, int n_pad, int k_pad,
                              uint8_t *__restrict__ A8)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (q, i), i fastest
    const int qn = k_pad / 64;
    if (e >= (int64_t)qn * n_pad) return;
    const int q = (int)(e / n_pad), i = (int)(e % n_pad);
    const uint64_t w = (i < n && q < kw) ? A[(int64_t)q * lda + i] : 0;
    uint8_t *row = A8 + (int64_t)i * urow_bytes(k_pad);
#pragma unroll
    for (int h = 0; h < 4; ++h) store16(row, 4 * q + h, expand16((uint32_t)(w >> (16 * h)) & 0xFFFFu));
}

// B (k x m, column blocks of bits) -> B8 = B^T rows: entry (j, r) = entry (r, j) of B
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
    store16(B8 + (int64_t)j * urow_bytes(k_pad), g, expand16(bits));
}

// bits beyond the last column in the last column block (rows x 1 words)
__global__ void k_check_last_block(const uint64_t *__restrict__ last, int rows, uint64_t mask, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows && (last[i] & ~mask)) atomicOr(err, 1u);
}

// ---------------------------------------------------------------- peak probe
// The tensor pipe's rate for kind::f8f6f4 128 x 256 x 32 MMAs from shared
// memory (zeros; no loads in the loop): one CTA per SM issues `iters`
// groups of 4 MMAs into one accumulator and commits once.
__global__ void __launch_bounds__(64, 1) k_umma_peak(int iters, uint32_t *err)
{
    extern __shared__ uint8_t usmem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(usmem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kUStageBytes);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 1);
    volatile uint32_t *fail = s_tmem + 1;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kUStageBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(base)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        mbar_init(su32(bars), 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, for the tensor core's reads
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                     "r"((uint32_t)kUN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    if (threadIdx.x == 0) {
        const uint32_t sa = su32(base), sb = sa + kUABytes;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int kk = 0; kk < kUK / 32; ++kk)
                umma_f8(tmem, sw128_desc(sa + 32 * kk), sw128_desc(sb + 32 * kk), (i | kk) != 0);
        umma_commit(su32(bars));
        mbar_wait(su32(bars), 0, fail, err);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kUN) : "memory");
    }
    if (threadIdx.x == 0 && *fail) atomicOr(err, 1u);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// a rows x k_pad operand (K contiguous, urow_bytes per row), boxes of
// box_rows x 128 entries landing as 128-byte rows, 128-byte swizzle
bool make_map(CUtensorMap *map, const uint8_t *p, int rows, int k_pad, int box_rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)urow_bytes(k_pad)};
    const cuuint32_t box[2] = {(cuuint32_t)kUK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType type = kUFp4 ? CU_TENSOR_MAP_DATA_TYPE_16U4_ALIGN16B : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    return enc(map, type, 2, const_cast<uint8_t *>(p), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t prepare_umma(int smem)
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_umma_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

constexpr int kUPeakSmem = kUSmem;  // one probe CTA per SM

}  // namespace

int64_t mma_pad(int64_t x) { return (x + 127) / 128 * 128; }

int64_t mma_row_bytes(int64_t k_pad) { return urow_bytes(k_pad); }

cudaError_t launch_check_last_block(const uint64_t *last, int rows, uint64_t mask, uint32_t *err, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_check_last_block<<<(rows + 255) / 256, 256, 0, s>>>(last, rows, mask, err);
    return cudaGetLastError();
}

cudaError_t launch_expand_operands(const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb, int n, int k, int m,
                                   uint8_t *A8, uint8_t *B8, cudaStream_t s)
{
    const int n_pad = (int)mma_pad(n), m_pad = (int)mma_pad(m), k_pad = (int)mma_pad(k);
    const int kw = (k + 63) / 64;
    cudaError_t e;
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
    return cudaSuccess;
}

// C (+)= A B: A8, B8 expanded by launch_expand_operands (A8 n_pad x k_pad,
// B8 m_pad x k_pad, K contiguous, both 16-byte aligned); err: a word the
// kernel ORs 1 into when a wait gave up.  cudaErrorNotSupported when the
// driver does not provide the tensor-map encoder or rejects a map.
cudaError_t launch_umma_product(const uint8_t *A8, const uint8_t *B8, int n_pad, int m_pad, int k_pad, uint64_t *C,
                                int64_t ldc, int n, int m, int accumulate, uint32_t *err, cudaStream_t s)
{
    cudaError_t e = prepare_umma(kUPeakSmem);
    if (e != cudaSuccess) return e;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A8, n_pad, k_pad, kUM) || !make_map(&tb, B8, m_pad, k_pad, kUN)) return cudaErrorNotSupported;
    const int tiles_m = (n_pad + kUM - 1) / kUM, tiles_n = (m_pad + kUN - 1) / kUN;
    const int ktiles = k_pad / kUK;
    const int64_t tiles = (int64_t)tiles_m * tiles_n;
    if (tiles > 0x7FFFFFFF) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(tiles, sms > 0 ? sms : 1);
    k_umma<<<grid, kUThreads, kUSmem, s>>>(ta, tb, ktiles, tiles_m, tiles_n, C, ldc, n, (m + 63) / 64, accumulate,
                                          err);
    return cudaGetLastError();
}

cudaError_t launch_umma_peak(int ctas, int iters, uint32_t *err, cudaStream_t s)
{
    cudaError_t e = prepare_umma(kUPeakSmem);
    if (e != cudaSuccess) return e;
    k_umma_peak<<<ctas, 64, kUPeakSmem, s>>>(iters, err);
    return cudaGetLastError();
}

double umma_peak_flops_per_iter() { return 2.0 * kUM * kUN * kUK; }

}  // namespace gf2
