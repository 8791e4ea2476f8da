// Many independent solves A X = B in one launch (the serving form): every CTA
// takes the next system from a shared counter (systems in decreasing size)
// and solves it alone, with the same steps and the same results as the
// whole-GPU solve of k_solve.cu (v = P B, forward substitution with the unit
// lower triangle of L by 64-row blocks, consistency from the residual rows,
// back substitution with E at the pivot columns, free variables 0).
//
// One CTA per system means no grid-wide barrier, but then one SM has to
// stream all of L and E: the design keeps that stream deep.
//   * v (and y, which overwrites v[0..r) block by block) lives in shared
//     memory when the launch's largest system fits (n <= about 26000), so
//     the only global traffic of a block is the column block of L (or E)
//     being applied, read once, coalesced;
//   * each thread issues kServeU independent loads of that column block
//     before it consumes them (the dependent load-lookup-store chain of a
//     plain loop left one load in flight per thread);
//   * 512 threads per CTA.
// The outputs (X, the consistency word, the rank) may live in mapped host
// memory: once they are written and fenced at system scope, the system's
// done word is set, so the host hands each result back without waiting for
// the whole launch.
#include "solve_core.cuh"

namespace gf2 {
namespace {

constexpr int kServeThreads = 512;
constexpr int kServeWarps = kServeThreads / 32;
constexpr int kServeU = 8;
// shared words before v: 8 tables of 256, the block's right-hand side and
// solution (64 + 64), 8 words of flags, one 64-word row buffer per warp
constexpr int kServeFixedWords = 8 * 256 + 64 + 64 + 8 + kServeWarps * 64;
constexpr int kServeMaxSmem = 226 * 1024;  // dynamic part: the opt-in limit (227 KB) less the static words
constexpr int64_t kServeClusterMin = 4096;  // systems from this size take a cluster

template <bool VS>
__device__ void solve_cta(const SolveCtx &c, uint64_t *smem)
{
    constexpr int T = kServeThreads, U = kServeU;
    uint64_t *tab = smem, *vec = tab + 8 * 256, *res = vec + 64, *flags = res + 64, *wrows = flags + 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = c.n, m = c.m, kmax = min(n, m);
    const int r = (int)min(max(*c.rank, (int64_t)0), (int64_t)kmax);
    const int mu = (m + 63) / 64, nbl = (r + 63) / 64;
    uint64_t *v = VS ? wrows + kServeWarps * 64 : c.v;  // v[i], then y[t] in v[t] for t < r

    // ---- v = P B, X = 0, the first pivot of each column block, the inverses
    // of the diagonal blocks
    if (tid == 0) flags[0] = 0;
    for (int i0 = tid; i0 < n; i0 += T * U) {
        int p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * T;
            p[u] = i < n ? c.perm[i] : -1;
        }
        uint64_t b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) b[u] = (unsigned)p[u] < (unsigned)n ? c.B[p[u]] : 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * T < n) v[i0 + u * T] = b[u] & c.rhs_mask;
    }
    for (int i = tid; i < m; i += T) c.X[i] = 0;
    for (int t = tid; t < r; t += T) {  // qstart[q] = first pivot t with column >= 64q
        const int q = min(max(c.pivcols[t] >> 6, 0), mu - 1);
        const int qp = t == 0 ? -1 : min(max(c.pivcols[t - 1] >> 6, -1), q);
        for (int qq = qp + 1; qq <= q; ++qq) c.qstart[qq] = t;
    }
    {
        const int qlast = r > 0 ? min(max(c.pivcols[r - 1] >> 6, -1), mu - 1) : -1;
        for (int qq = qlast + 1 + tid; qq <= mu; qq += T) c.qstart[qq] = r;
    }
    __syncthreads();  // qstart is read by the inverses of E's blocks
    for (int J = warp; J < nbl; J += kServeWarps) lower_block_inverse(c, J, r, wrows + warp * 64, lane);
    for (int q = warp; q < mu; q += kServeWarps) upper_block_inverse(c, q, r, wrows + warp * 64, lane);
    __syncthreads();

    // ---- forward substitution, 64 rows at a time; y_J replaces v on its rows
    for (int J = 0; J < nbl; ++J) {
        const int base = 64 * J, cnt = min(64, r - base);
        if (tid < 64) vec[tid] = tid < cnt ? v[base + tid] : 0;
        __syncthreads();
        if (tid < 64) {
            const uint64_t li = c.linv[(int64_t)J * 64 + tid];
            uint64_t acc = 0;
#pragma unroll 16
            for (int t = 0; t < 64; ++t)
                if ((li >> t) & 1) acc ^= vec[t];
            res[tid] = acc;
            if (tid < cnt) v[base + tid] = acc;
        }
        __syncthreads();
        solve_tables<T>(tab, res);
        __syncthreads();
        // every row below the block (the residual rows i >= r included)
        const uint64_t *LJ = c.L + (int64_t)J * c.ldl;
        for (int i0 = min(base + 64, r) + tid; i0 < n; i0 += T * U) {
            uint64_t w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * T;
                w[u] = i < n ? LJ[i] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (w[u]) v[i0 + u * T] ^= solve_lookup(tab, w[u]);
        }
        __syncthreads();
    }

    // ---- consistency: OR of the residual rows
    {
        uint64_t bad = 0;
        for (int i = r + tid; i < n; i += T) bad |= v[i];
#pragma unroll
        for (int off = 16; off; off >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        if (lane == 0 && bad) atomicOr(reinterpret_cast<unsigned long long *>(flags), (unsigned long long)bad);
    }
    __syncthreads();
    const uint64_t ok = c.rhs_mask & ~flags[0];
    if (tid == 0) *c.consistent = ok;

    // ---- back substitution, one column block of E at a time, last first
    for (int q = mu - 1; q >= 0; --q) {
        const int t0 = min(max(c.qstart[q], 0), r);
        const int cnt = min(max(c.qstart[q + 1] - t0, 0), min(64, r - t0));
        if (cnt == 0) continue;  // the same decision in every thread
        if (tid < 64) {
            vec[tid] = tid < cnt ? v[t0 + tid] : 0;
            res[tid] = 0;
        }
        __syncthreads();
        if (tid < cnt) {
            const uint64_t ui = c.uinv[(int64_t)q * 64 + tid];
            uint64_t acc = 0;
#pragma unroll 16
            for (int t = 0; t < 64; ++t)
                if ((ui >> t) & 1) acc ^= vec[t];
            const int col = c.pivcols[t0 + tid];
            res[(col - 64 * q) & 63] = acc;
            if ((unsigned)col < (unsigned)m) c.X[col] = acc & ok;
        }
        __syncthreads();
        solve_tables<T>(tab, res);
        __syncthreads();
        const uint64_t *Eq = c.E + (int64_t)q * c.lde;
        for (int t0i = tid; t0i < t0; t0i += T * U) {
            uint64_t w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0i + u * T;
                w[u] = t < t0 ? Eq[t] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (w[u]) v[t0i + u * T] ^= solve_lookup(tab, w[u]);
        }
        __syncthreads();
    }
}

template <bool VS>
__global__ void __launch_bounds__(kServeThreads, 2) k_serve(const ServeItem *items, int count, int32_t *next)
{
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int k = s_item;
        __syncthreads();
        if (k >= count) return;
        const ServeItem &it = items[k];
        if (it.nrhs > 0) solve_cta<VS>(it.c, smem);
        if (tid == 0) {
            const int64_t kmax = min(it.c.n, it.c.m);
            *it.rank_out = min(max(*it.c.rank, (int64_t)0), kmax);
        }
        __threadfence_system();
        __syncthreads();
        if (tid == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(it.done), "r"(1u) : "memory");
    }
}

// ---------------------------------------------------------------- clusters
// The same solve for one large system by a cluster of kClusterCTAs CTAs
// (co-scheduled by the hardware on one GPC).  CTA c of the cluster keeps rows
// [c S, (c+1) S) of v and of y (S a multiple of 64) in its own shared memory,
// so a 64-row block lives in one CTA.  Per block every CTA reads the block's
// 64 values from the CTA that holds them through distributed shared memory,
// solves the diagonal block itself (the same 64 words in every CTA), and
// updates its own rows; one hardware cluster barrier per block orders the
// steps (no flag is polled).  Eight SMs stream L and E instead of one.
constexpr int kClusterCTAs = kServeClusterCTAs;

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// word p of the shared memory of CTA `rank` of this cluster (p: the same
// variable in this CTA's shared memory)
__device__ __forceinline__ uint64_t ld_peer(const uint64_t *p, uint32_t rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
    return v;
}

__global__ void __launch_bounds__(kServeThreads, 1) k_serve_cluster(const ServeItem *items, int slice)
{
    constexpr int T = kServeThreads, U = kServeU, CL = kClusterCTAs;
    extern __shared__ __align__(16) uint64_t smem[];
    uint64_t *tab = smem, *vec = tab + 8 * 256, *res = vec + 64, *flags = res + 64, *wrows = flags + 8;
    uint64_t *vs = wrows + kServeWarps * 64;  // this CTA's rows of v
    uint64_t *ys = vs + slice;                // and of y
    const int cr = (int)cluster_rank();
    const ServeItem &it = items[blockIdx.x / CL];
    const SolveCtx &c = it.c;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = c.n, m = c.m, kmax = min(n, m);
    const int r = (int)min(max(*c.rank, (int64_t)0), (int64_t)kmax);
    const int mu = (m + 63) / 64, nbl = (r + 63) / 64;
    const int S = slice, lo = cr * S, hi = min(n, lo + S);  // this CTA's rows [lo, hi)
    const int gtid = cr * T + tid, CT = CL * T, gw = cr * kServeWarps + warp, GW = CL * kServeWarps;
    cluster_sync();  // every CTA of the cluster runs (its shared memory exists)
    if (it.nrhs > 0) {
        // ---- v = P B on this CTA's rows, X = 0, qstart, the diagonal inverses
        for (int i0 = lo + tid; i0 < hi; i0 += T * U) {
            int p[U];
#pragma unroll
            for (int u = 0; u < U; ++u) p[u] = i0 + u * T < hi ? c.perm[i0 + u * T] : -1;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + u * T < hi) vs[i0 + u * T - lo] = ((unsigned)p[u] < (unsigned)n ? c.B[p[u]] : 0) & c.rhs_mask;
        }
        for (int i = gtid; i < m; i += CT) c.X[i] = 0;
        for (int t = gtid; t < r; t += CT) {
            const int q = min(max(c.pivcols[t] >> 6, 0), mu - 1);
            const int qp = t == 0 ? -1 : min(max(c.pivcols[t - 1] >> 6, -1), q);
            for (int qq = qp + 1; qq <= q; ++qq) c.qstart[qq] = t;
        }
        {
            const int qlast = r > 0 ? min(max(c.pivcols[r - 1] >> 6, -1), mu - 1) : -1;
            for (int qq = qlast + 1 + gtid; qq <= mu; qq += CT) c.qstart[qq] = r;
        }
        if (cr == 0 && tid == 0) *c.bad = 0;
        for (int J = gw; J < nbl; J += GW) lower_block_inverse(c, J, r, wrows + warp * 64, lane);
        cluster_sync();  // qstart (read by the inverses of E's blocks), linv, bad
        for (int q = gw; q < mu; q += GW) upper_block_inverse(c, q, r, wrows + warp * 64, lane);

        // ---- forward substitution
        for (int J = 0; J < nbl; ++J) {
            const int base = 64 * J, cnt = min(64, r - base), owner = base / S;
            if (tid < 64) vec[tid] = tid < cnt ? ld_peer(vs + (base - owner * S) + tid, owner) : 0;
            __syncthreads();
            if (tid < 64) {
                const uint64_t li = c.linv[(int64_t)J * 64 + tid];
                uint64_t acc = 0;
#pragma unroll 16
                for (int t = 0; t < 64; ++t)
                    if ((li >> t) & 1) acc ^= vec[t];
                res[tid] = acc;
                if (cr == owner && tid < cnt) ys[base - lo + tid] = acc;
            }
            __syncthreads();
            solve_tables<T>(tab, res);
            __syncthreads();
            const uint64_t *LJ = c.L + (int64_t)J * c.ldl;
            for (int i0 = max(lo, min(base + 64, r)) + tid; i0 < hi; i0 += T * U) {
                uint64_t w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) w[u] = i0 + u * T < hi ? LJ[i0 + u * T] : 0;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u]) vs[i0 + u * T - lo] ^= solve_lookup(tab, w[u]);
            }
            cluster_sync();  // block J+1's rows are final before anyone reads them
        }

        // ---- consistency: OR of the residual rows
        {
            uint64_t bad = 0;
            for (int i = max(lo, r) + tid; i < hi; i += T) bad |= vs[i - lo];
#pragma unroll
            for (int off = 16; off; off >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, off);
            if (lane == 0 && bad) atomicOr(reinterpret_cast<unsigned long long *>(c.bad), (unsigned long long)bad);
        }
        cluster_sync();
        const uint64_t ok = c.rhs_mask & ~__ldcg(c.bad);
        if (cr == 0 && tid == 0) *c.consistent = ok;

        // ---- back substitution
        for (int q = mu - 1; q >= 0; --q) {
            const int t0 = min(max(__ldcg(c.qstart + q), 0), r);
            const int cnt = min(max(__ldcg(c.qstart + q + 1) - t0, 0), min(64, r - t0));
            if (cnt == 0) continue;  // the same in every CTA
            if (tid < 64) {
                const int t = t0 + tid;
                vec[tid] = tid < cnt ? ld_peer(ys + (t - (t / S) * S), t / S) : 0;
                res[tid] = 0;
            }
            __syncthreads();
            if (tid < cnt) {
                const uint64_t ui = c.uinv[(int64_t)q * 64 + tid];
                uint64_t acc = 0;
#pragma unroll 16
                for (int t = 0; t < 64; ++t)
                    if ((ui >> t) & 1) acc ^= vec[t];
                const int col = c.pivcols[t0 + tid];
                res[(col - 64 * q) & 63] = acc;
                if (cr == 0 && (unsigned)col < (unsigned)m) c.X[col] = acc & ok;
            }
            __syncthreads();
            solve_tables<T>(tab, res);
            __syncthreads();
            const uint64_t *Eq = c.E + (int64_t)q * c.lde;
            const int te = min(hi, t0);
            for (int i0 = lo + tid; i0 < te; i0 += T * U) {
                uint64_t w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) w[u] = i0 + u * T < te ? Eq[i0 + u * T] : 0;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (w[u]) ys[i0 + u * T - lo] ^= solve_lookup(tab, w[u]);
            }
            cluster_sync();
        }
    }
    if (cr == 0 && tid == 0) *it.rank_out = min(max(*c.rank, (int64_t)0), (int64_t)kmax);
    __threadfence_system();
    cluster_sync();  // every CTA's outputs are written; no peer reads this CTA's shared memory any more
    if (cr == 0 && tid == 0) asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(it.done), "r"(1u) : "memory");
}

}  // namespace

// rows per CTA of a cluster for an n-row system (a multiple of 64), and
// whether a cluster serves it (larger systems only, their slices in shared
// memory)
int64_t serve_cluster_slice(int64_t n) { return ((n + kClusterCTAs - 1) / kClusterCTAs + 63) / 64 * 64; }

bool serve_by_cluster(int64_t n)
{
    return n >= kServeClusterMin && (kServeFixedWords + 2 * serve_cluster_slice(n)) * 8 <= kServeMaxSmem;
}

cudaError_t launch_serve_cluster(const ServeItem *items, int count, int64_t max_n, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int slice = (int)serve_cluster_slice(max_n);
    const size_t bytes = (size_t)(kServeFixedWords + 2 * slice) * 8;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        e = cudaFuncSetAttribute(k_serve_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, kServeMaxSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * kClusterCTAs));
    cfg.blockDim = dim3(kServeThreads);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCTAs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_serve_cluster, items, slice);
}

cudaError_t launch_serve_solve(const ServeItem *items, int count, int32_t *next, int64_t max_n, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    static bool attr_done[64][2] = {};
    int dev = 0, sms = 1, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t vs_bytes = (size_t)(kServeFixedWords + max_n) * 8;
    const bool vs = vs_bytes <= (size_t)kServeMaxSmem;
    const size_t bytes = vs ? vs_bytes : (size_t)kServeFixedWords * 8;
    const void *fn = vs ? reinterpret_cast<const void *>(k_serve<true>) : reinterpret_cast<const void *>(k_serve<false>);
    if (dev >= 0 && dev < 64 && !attr_done[dev][vs]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kServeMaxSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev][vs] = true;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kServeThreads, bytes);
    if (e != cudaSuccess) return e;
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    const int grid = count < cap ? count : cap;
    if (vs) k_serve<true><<<grid, kServeThreads, bytes, s>>>(items, count, next);
    else k_serve<false><<<grid, kServeThreads, bytes, s>>>(items, count, next);
    return cudaGetLastError();
}

}  // namespace gf2
