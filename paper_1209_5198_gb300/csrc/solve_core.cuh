// Device helpers shared by the triangular solves (k_solve.cu: one system
// over the whole GPU; k_serve.cu: many systems, one CTA each): Four Russians
// tables of 64 solved values and the inverses of the 64 x 64 diagonal blocks
// of L and of E at its pivots (the factors of Lemma 4.1 in PLE form).
#pragma once
#include "gf2_internal.cuh"

namespace gf2 {

// 8 tables of 256 entries: entry (g, x) = XOR of vals[8g + b] over the bits b
// of x (T threads of the CTA).
template <int T>
__device__ __forceinline__ void solve_tables(uint64_t *tab, const uint64_t *vals)
{
    for (int e = threadIdx.x; e < 8 * 256; e += T) {
        const int g = e >> 8, x = e & 255;
        uint64_t acc = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if ((x >> b) & 1) acc ^= vals[8 * g + b];
        tab[e] = acc;
    }
}

// XOR of the 64 solved values selected by the bits of w (Four Russians
// lookups, 8 bits at a time)
__device__ __forceinline__ uint64_t solve_lookup(const uint64_t *tab, uint64_t w)
{
    uint64_t a = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) a ^= tab[g * 256 + (int)((w >> (8 * g)) & 255)];
    return a;
}

// Rows of the inverse of diagonal block J of L (one warp).  Row i of L^-1
// solves y L = e_i: from the last column down, once y_t is final, row t of L
// (below the diagonal) leaves the right-hand side when y_t = 1.
inline __device__ void lower_block_inverse(const SolveCtx &c, int J, int r, uint64_t *wrow, int lane)
{
    const int base = 64 * J, cnt = min(64, r - base);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        wrow[t] = t < cnt ? c.L[(int64_t)J * c.ldl + base + t] : 0;
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        uint64_t y = i < cnt ? (1ull << i) : 0;
#pragma unroll 4
        for (int t = 63; t > 0; --t)
            if ((y >> t) & 1) y ^= wrow[t] & ((1ull << t) - 1);
        c.linv[(int64_t)J * 64 + i] = y;
    }
    __syncwarp();
}

// Rows of the inverse of the diagonal block of column block q of E (one
// warp): U[s][s'] = E[t0+s][p_{t0+s'}] for the cnt pivots t0.. whose columns
// lie in block q (unit upper triangular).  Row i of U^-1 solves y U = e_i,
// swept from the first column up.
inline __device__ void upper_block_inverse(const SolveCtx &c, int q, int r, uint64_t *wrow, int lane)
{
    const int t0 = min(max(__ldcg(c.qstart + q), 0), r);
    const int cnt = min(max(__ldcg(c.qstart + q + 1) - t0, 0), min(64, r - t0));
    if (cnt == 0) return;
    int pb[2];
    uint64_t w[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        pb[h] = s < cnt ? ((c.pivcols[t0 + s] - 64 * q) & 63) : 0;
        w[h] = s < cnt ? c.E[(int64_t)q * c.lde + t0 + s] : 0;
    }
    uint64_t u[2] = {0, 0};
    for (int s2 = 0; s2 < cnt; ++s2) {  // compress the rows to the pivot columns
        const int b = __shfl_sync(0xffffffffu, s2 < 32 ? pb[0] : pb[1], s2 & 31);
        u[0] |= ((w[0] >> b) & 1) << s2;
        u[1] |= ((w[1] >> b) & 1) << s2;
    }
    wrow[lane] = u[0];
    wrow[lane + 32] = u[1];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        uint64_t y = i < cnt ? (1ull << i) : 0;
#pragma unroll 4
        for (int t = 0; t < 63; ++t)
            if ((y >> t) & 1) y ^= wrow[t] & ~((2ull << t) - 1);
        c.uinv[(int64_t)q * 64 + i] = y;
    }
    __syncwarp();
}

}  // namespace gf2
