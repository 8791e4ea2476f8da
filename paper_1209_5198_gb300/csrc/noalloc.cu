// gf2_rank_noalloc: the rank of a matrix of at most 4096 x 4096, computed
// with scratch memory that the library reserves once, statically, instead
// of allocating it per call.
//
// Some callers cannot allocate device memory when they call into this
// library: programs that reserve a fixed device-memory budget at start-up
// and forbid allocations afterwards, or frameworks that own every device
// buffer and hand a library only the inputs and outputs.  For them this
// entry point needs nothing but the input matrix and the output word.
//
// The scratch is one file-scope __device__ array (kNoallocBytes, about
// 2.7 MiB).  Every GPU that loads the library holds it until the process
// exits.  Host code must not use the array's name as a device address:
// the first call on each device, with that device current, asks the runtime
// for the array's device address (cudaGetSymbolAddress) and keeps it.  Do
// that first call before any stream capture.  All calls on a device share
// the array and it keeps the contents of the last call: calls that overlap
// on the GPU (for instance on two streams) race and give wrong results.
#include <mutex>
#include <vector>

#include "../../include/gf2.h"
#include "gf2_internal.cuh"

using namespace gf2;

namespace {

constexpr int64_t kNoallocMaxDim = 4096;
constexpr int64_t kNoallocMu = kNoallocMaxDim / 64;  // column blocks (and ldw, a multiple of 8)
constexpr size_t kAlignNA = 256;
constexpr size_t align_na(size_t x) { return (x + kAlignNA - 1) / kAlignNA * kAlignNA; }

// layout of the static scratch (worst case n = m = 4096)
constexpr size_t kOffW = 0;
constexpr size_t kOffY = kOffW + align_na((size_t)kNoallocMaxDim * kNoallocMu * 8);
constexpr size_t kOffF = kOffY + align_na((size_t)kNoallocMaxDim * kRing * 8);
constexpr size_t kOffAct = kOffF + align_na((size_t)kNoallocMaxDim * 2 * 8);
constexpr size_t kOffNact = kOffAct + align_na((size_t)kNoallocMaxDim * kRing * 4);
constexpr size_t kOffPP = kOffNact + align_na((size_t)kNoallocMu * 4);
constexpr size_t kOffInfo = kOffPP + align_na((size_t)kNoallocMaxDim * 4);
constexpr size_t kOffPerm = kOffInfo + align_na((size_t)kNoallocMu * sizeof(PanelInfo));
constexpr size_t kOffPiv = kOffPerm + align_na((size_t)kNoallocMaxDim * 4);
constexpr size_t kOffFlag = kOffPiv + align_na((size_t)kNoallocMaxDim * 4);
constexpr size_t kNoallocBytes = kOffFlag + kAlignNA;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_na_mutex;
std::vector<unsigned char *> g_na_ptr;  // device address of the scratch, per device

int noalloc_scratch(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if ((int)g_na_ptr.size() <= dev) g_na_ptr.resize(dev + 1, nullptr);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GF2_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return GF2_OK;
}

}  // namespace

extern "C" int gf2_rank_noalloc(const gf2_mat *A, int64_t *rank_dev, void *stream)
{
    if (!A || !rank_dev || A->rows < 0 || A->cols < 0) return GF2_ERR_ARG;
    const int64_t n = A->rows, m = A->cols;
    if (n > kNoallocMaxDim || m > kNoallocMaxDim) return GF2_ERR_UNSUPPORTED;
    if (n > 0 && m > 0 && (!A->w || A->ld < n)) return GF2_ERR_SHAPE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0 || m == 0) return cudaMemsetAsync(rank_dev, 0, sizeof(int64_t), s) == cudaSuccess ? GF2_OK : GF2_ERR_CUDA;
    unsigned char *base = nullptr;
    int st = noalloc_scratch(&base);
    if (st) return st;

    const int64_t mu = (m + 63) / 64;
    DecompCtx c{};
    c.W = reinterpret_cast<uint64_t *>(base + kOffW);
    c.tstride = n * kTileWords;
    c.lde = (mu + 7) / 8 * 8;
    c.perm = reinterpret_cast<int32_t *>(base + kOffPerm);
    c.pivcols = reinterpret_cast<int32_t *>(base + kOffPiv);
    c.info = reinterpret_cast<PanelInfo *>(base + kOffInfo);
    c.Y = reinterpret_cast<uint64_t *>(base + kOffY);
    c.F = reinterpret_cast<uint64_t *>(base + kOffF);
    c.act = reinterpret_cast<int32_t *>(base + kOffAct);
    c.nact = reinterpret_cast<int32_t *>(base + kOffNact);
    c.pivpanel = reinterpret_cast<int32_t *>(base + kOffPP);
    c.Lint = nullptr;
    c.ldl = 1;
    c.Eint = nullptr;
    c.n = (int32_t)n;
    c.m = (int32_t)m;
    c.mu = (int32_t)mu;
    c.kmax = (int32_t)(n < m ? n : m);
    uint32_t *flag = reinterpret_cast<uint32_t *>(base + kOffFlag);

    // the padding flag starts at zero; the scratch keeps the last call's contents
    if (cudaMemsetAsync(flag, 0, sizeof(uint32_t), s) != cudaSuccess) return GF2_ERR_CUDA;
    const uint64_t last = (m % 64) ? ((1ull << (m % 64)) - 1) : ~0ull;
    if (launch_ingest_tiled(A->w, A->ld, (int32_t)n, (int32_t)mu, last, c.W, c.perm, c.pivpanel, flag, s) != cudaSuccess)
        return GF2_ERR_CUDA;
    uint32_t flag_host = 0;  // a stack word: the copy allocates nothing
    if (cudaMemcpyAsync(&flag_host, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GF2_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GF2_ERR_CUDA;
    if (flag_host) return GF2_ERR_PADDING;
    // the same kernels as gf2_rank, one stream, no look-ahead
    if (cudaMemsetAsync(c.nact, 0, (size_t)c.mu * sizeof(int32_t), s) != cudaSuccess) return GF2_ERR_CUDA;
    for (int j = 0; j < c.mu; ++j) {
        if (launch_panel(c, j, s) != cudaSuccess) return GF2_ERR_CUDA;
        if (launch_next(c, j, s) != cudaSuccess) return GF2_ERR_CUDA;
        int tile_first = 0;
        if (rest_tiles(c, j, 1, &tile_first) > 0 && launch_rest(c, j, 1, (int)(n - 64 * (int64_t)(j + 1)), s) != cudaSuccess)
            return GF2_ERR_CUDA;
    }
    if (launch_finish_scalars(c, rank_dev, s) != cudaSuccess) return GF2_ERR_CUDA;
    return GF2_OK;
}
