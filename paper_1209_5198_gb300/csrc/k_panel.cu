// Panel kernel of the decomposition: one CTA runs the panel step of block j
// (panel_core.cuh) on the SM that the persistent trailing update leaves free.
#include <mutex>

#include "panel_core.cuh"

namespace gf2 {
namespace {

#ifdef GF2_TRACE
__device__ unsigned long long g_panel_trace[kTrSlots * kTraceMaxPanels];  // the trace build's panel stamps
#endif

// Dynamic shared memory of the panel kernel (see kPanelReserveBytes): the
// first kPanelListCap entries of the row list of the general path.
constexpr int kPanelReserveBytes = 160 * 1024;
constexpr int kPanelListCap = kPanelReserveBytes / 12 / 8 * 8;

// <= 128 registers: 128 x 128 fits next to a 512 x 96 k_rest CTA on one SM
__global__ void __launch_bounds__(kPanelThreads, 4) k_panel(DecompCtx c, int j)
{
    __shared__ PanelShared sh;
    extern __shared__ __align__(16) uint64_t panel_dyn[];
    GF2_TR(if (threadIdx.x == 0 && j < kTraceMaxPanels) g_panel_trace[kTrPanelEntry * kTraceMaxPanels + j] = trace_clock();)
    // Launched as a programmatic dependent of the previous panel: wait until
    // that launch has completed and its writes are visible, then let the
    // next panel be scheduled (it waits here in turn).  Without the launch
    // attribute both are no-ops.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#ifdef GF2_TRACE
    if (threadIdx.x == 0 && j < kTraceMaxPanels) g_panel_trace[kTrPanelStart * kTraceMaxPanels + j] = trace_clock();
    panel_block(c, j, sh, panel_dyn, kPanelListCap, j < kTraceMaxPanels ? g_panel_trace : nullptr);
#else
    panel_block(c, j, sh, panel_dyn, kPanelListCap);
#endif
}

// The dynamic shared memory also keeps a panel CTA off any SM holding a
// persistent k_rest CTA (about 67 KB; with this reserve the two need more
// than the 228 KB of an SM): the panel runs on the SM k_rest leaves free,
// without other warps competing for its scheduler.  The general path keeps
// its row list there.
static_assert(kPanelListCap * 12 <= kPanelReserveBytes, "row list in the reserve");

}  // namespace

cudaError_t prepare_panel_kernel()
{
    // several host threads may launch panels at once (the serving engine's
    // decomposition lanes, the entry point without allocation)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelReserveBytes);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

#ifdef GF2_TRACE
cudaError_t read_panel_trace(unsigned long long *out, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_panel_trace, sizeof(g_panel_trace));
    if (e == cudaSuccess && reset) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_panel_trace);
        if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(g_panel_trace));
    }
    return e;
}
#endif

cudaError_t launch_panel(const DecompCtx &c, int j, cudaStream_t s)
{
    const cudaError_t e = prepare_panel_kernel();
    if (e != cudaSuccess) return e;
    // programmatic stream serialization: the launch may start as soon as the
    // previous panel triggers (its CTA then waits in griddepcontrol.wait),
    // which hides the launch latency on the panel chain
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kPanelThreads);
    cfg.dynamicSmemBytes = kPanelReserveBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_panel, c, j);
}

}  // namespace gf2
