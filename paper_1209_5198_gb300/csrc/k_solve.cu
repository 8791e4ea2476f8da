// Linear systems A X = B over F2 from the factors of P*A = L*E (the use of
// the decomposition named in Section 1 of the paper; triangular solves with
// the factors of Lemma 4.1).  Up to 64 right-hand sides are packed one word
// per row (bit c = right-hand side c), so every step below is word-wide.
//
//   1. v = P B                                   (v[i] = B[perm[i]])
//   2. forward substitution with the r x r unit lower triangle of L:
//        y_i = v_i xor sum_{t<i} L[i][t] y_t,   i < r
//      and the same sums accumulated into the rows i >= r; right-hand side
//      c is consistent iff bit c of every such residual row is zero
//   3. back substitution with E at the pivot columns (free variables 0):
//        x_{p_t} = y_t xor sum_{t'>t} E[t][p_{t'}] x_{p_{t'}}
//      every other entry of X is zero, and so is every column of X that
//      belongs to an inconsistent right-hand side.
//
// GB300 design.  Both substitutions are blocked by 64: a diagonal block is
// solved by multiplying with its inverse (all inverses are computed up front,
// one warp per block, by column sweeps), and the rows that depend on the
// block take its contribution by Four Russians lookups (8 tables of 256
// words built from the 64 solved values).  The blocks are sequential, so the
// whole solve is ONE cooperative launch with a grid-wide barrier between
// blocks; every CTA works on a fixed slice of the rows.  The barrier's wait
// is bounded: a CTA that gives up sets an error word and every CTA returns.
// L is used in its own column blocks (diagonal block J = rows 64J.. of
// column block J); E likewise, the diagonal block of column block q being
// the pivots whose columns fall in q.
#include "solve_core.cuh"

namespace gf2 {
namespace {

constexpr int kSolveThreads = 256;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr uint32_t kSpinLimit = 1u << 24;  // default polls of a grid-wide wait (~1-2 s of 100 ns sleeps)

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier (all CTAs are co-resident: cooperative launch).  Returns
// false, in every thread, once any CTA has given up waiting.
__device__ bool grid_barrier(uint32_t *count, uint32_t *err, uint32_t &epoch, int *s_ok, uint32_t limit)
{
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const uint32_t target = epoch * gridDim.x;
        uint32_t it = 0;
        while (ld_acquire(count) < target) {
            if (ld_acquire(err) & 1u) break;
            if (++it > limit) {
                atomicOr(err, 1u);
                break;
            }
            __nanosleep(100);
        }
        *s_ok = (ld_acquire(err) & 1u) == 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The barrier between the steps of one solve: grid-wide for the cooperative
// launch, the CTA's own for a solve that one CTA runs alone.
struct GridSync {
    uint32_t *count, *err;
    uint32_t epoch;
    int *s_ok;
    uint32_t limit;
    __device__ bool operator()() { return grid_barrier(count, err, epoch, s_ok, limit); }
};
struct CtaSync {
    __device__ bool operator()()
    {
        __syncthreads();
        return true;
    }
};

struct SolveShared {
    uint64_t tab[8 * 256];
    uint64_t vec[64];  // the right-hand side of the current diagonal block
    uint64_t res[64];  // its solution (spread over the block's columns)
    uint64_t wrow[kSolveWarps][64];
    int s_ok;
};

// One solve, run by G CTAs (this is CTA b) that meet at `bar` between steps.
template <class Sync>
__device__ void solve_body(const SolveCtx &c, int b, int G, Sync &bar, SolveShared &sh)
{
    uint64_t *tab = sh.tab, *vec = sh.vec, *res = sh.res;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = c.n, m = c.m, kmax = min(n, m);
    const int r = (int)min(max(*c.rank, (int64_t)0), (int64_t)kmax);
    const int mu = (m + 63) / 64, nbl = (r + 63) / 64;
    uint32_t *err = c.sync + 1;
    const int gthreads = G * kSolveThreads, gtid = b * kSolveThreads + tid;
    const int gw = b * kSolveWarps + warp, GW = G * kSolveWarps;

    // ---- phase 0: v = P B (padding check), X = 0, the first pivot of each
    // column block, the inverses of the diagonal blocks of L
    for (int i = gtid; i < n; i += gthreads) {
        const int p = c.perm[i];
        uint64_t v = (unsigned)p < (unsigned)n ? c.B[p] : 0;
        if (v & ~c.rhs_mask) {
            if (c.check) atomicOr(err, 2u);
            v &= c.rhs_mask;
        }
        c.v[i] = v;
    }
    for (int i = gtid; i < m; i += gthreads) c.X[i] = 0;
    for (int t = gtid; t < r; t += gthreads) {  // qstart[q] = first pivot t with column >= 64q
        const int q = min(max(c.pivcols[t] >> 6, 0), mu - 1);
        const int qp = t == 0 ? -1 : min(max(c.pivcols[t - 1] >> 6, -1), q);
        for (int qq = qp + 1; qq <= q; ++qq) c.qstart[qq] = t;
    }
    {
        const int qlast = r > 0 ? min(max(c.pivcols[r - 1] >> 6, -1), mu - 1) : -1;
        for (int qq = qlast + 1 + gtid; qq <= mu; qq += gthreads) c.qstart[qq] = r;
    }
    for (int J = gw; J < nbl; J += GW) lower_block_inverse(c, J, r, sh.wrow[warp], lane);
    if (!bar()) return;
    // needed only by the back substitution; the barriers below order them
    for (int q = gw; q < mu; q += GW) upper_block_inverse(c, q, r, sh.wrow[warp], lane);

    // ---- forward substitution, 64 rows at a time
    const int rb = (int)((int64_t)n * b / G), re = (int)((int64_t)n * (b + 1) / G);
    for (int J = 0; J < nbl; ++J) {
        const int base = 64 * J, cnt = min(64, r - base);
        if (tid < 64) vec[tid] = tid < cnt ? __ldcg(c.v + base + tid) : 0;
        __syncthreads();
        if (tid < 64) {
            const uint64_t li = __ldcg(c.linv + (int64_t)J * 64 + tid);
            uint64_t acc = 0;
            for (int t = 0; t < 64; ++t)
                if ((li >> t) & 1) acc ^= vec[t];
            res[tid] = acc;
            if (b == 0 && tid < cnt) c.y[base + tid] = acc;
        }
        __syncthreads();
        solve_tables<kSolveThreads>(tab, res);
        __syncthreads();
        // every row below the block (the residual rows i >= r included)
        const uint64_t *LJ = c.L + (int64_t)J * c.ldl;
        for (int i = max(rb, min(base + 64, r)) + tid; i < re; i += kSolveThreads) {
            const uint64_t w = LJ[i];
            if (w) c.v[i] = __ldcg(c.v + i) ^ solve_lookup(tab, w);
        }
        if (!bar()) return;
    }

    // ---- consistency: OR of the residual rows
    {
        uint64_t bad = 0;
        for (int i = max(rb, r) + tid; i < re; i += kSolveThreads) bad |= __ldcg(c.v + i);
#pragma unroll
        for (int off = 16; off; off >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        if (lane == 0 && bad) atomicOr(reinterpret_cast<unsigned long long *>(c.bad), (unsigned long long)bad);
    }
    if (!bar()) return;
    const uint64_t ok = c.rhs_mask & ~__ldcg(c.bad);
    if (b == 0 && tid == 0) *c.consistent = ok;

    // ---- back substitution, one column block of E at a time, last first
    const int tb = (int)((int64_t)r * b / G), te = (int)((int64_t)r * (b + 1) / G);
    for (int q = mu - 1; q >= 0; --q) {
        const int t0 = min(max(__ldcg(c.qstart + q), 0), r);
        const int cnt = min(max(__ldcg(c.qstart + q + 1) - t0, 0), min(64, r - t0));
        if (cnt == 0) continue;  // the same decision in every CTA: no barrier
        if (tid < 64) {
            vec[tid] = tid < cnt ? __ldcg(c.y + t0 + tid) : 0;
            res[tid] = 0;
        }
        __syncthreads();
        if (tid < cnt) {
            const uint64_t ui = __ldcg(c.uinv + (int64_t)q * 64 + tid);
            uint64_t acc = 0;
            for (int t = 0; t < 64; ++t)
                if ((ui >> t) & 1) acc ^= vec[t];
            const int col = c.pivcols[t0 + tid];
            res[(col - 64 * q) & 63] = acc;
            if (b == 0 && (unsigned)col < (unsigned)m) c.X[col] = acc & ok;
        }
        __syncthreads();
        solve_tables<kSolveThreads>(tab, res);
        __syncthreads();
        const uint64_t *Eq = c.E + (int64_t)q * c.lde;
        for (int t = tb + tid; t < min(te, t0); t += kSolveThreads) {
            const uint64_t w = Eq[t];
            if (w) c.y[t] = __ldcg(c.y + t) ^ solve_lookup(tab, w);
        }
        if (!bar()) return;
    }
}

__global__ void __launch_bounds__(kSolveThreads) k_solve(SolveCtx c)
{
    __shared__ SolveShared sh;
    GridSync bar{c.sync, c.sync + 1, 0, &sh.s_ok, c.wait_limit};
    solve_body(c, blockIdx.x, gridDim.x, bar, sh);
}

}  // namespace

cudaError_t launch_solve(const SolveCtx &c, cudaStream_t s)
{
    int dev = 0, sms = 1, per_sm = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve, kSolveThreads, 0);
    if (e != cudaSuccess) return e;
    if (!coop || per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // one CTA per 256 rows, at most one per SM (each barrier costs every CTA)
    const int rows = c.n > c.m ? c.n : c.m;
    int grid = (rows + kSolveThreads - 1) / kSolveThreads;
    grid = grid < 1 ? 1 : (grid > sms ? sms : grid);
    SolveCtx arg = c;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_solve), dim3(grid), dim3(kSolveThreads), args,
                                       0, s);
}

}  // namespace gf2
