// adc_scan_fwd_noalloc: the inclusive scan forward pass for callers that
// cannot allocate device memory.
//
// Some callers have no way to obtain scratch memory: code running inside a
// custom allocator or a memory-pool callback (where calling cudaMalloc would
// re-enter the allocator), plugins and embedded runtimes handed only
// fixed input/output buffers by their host, and real-time paths whose memory
// budget is fixed up front.  For them this entry point keeps the scan's
// look-back scratch (tile flags, tile aggregates and inclusive prefixes, the
// tile counter and the error word) in a file-scope device array, so a call
// needs nothing but its input and output.
//
// The array is kNoAllocScratchBytes (4 MiB) on every GPU that loads the
// library, held until the process exits.  Its device address is looked up
// once per device, on the first call made while that device is current; make
// that first call before capturing any stream.  The address belongs to the
// device's current context: when that context changes (cudaDeviceReset and a
// new primary context), the next call sees a different context id and looks
// the address up again instead of writing through the old one.  Every call on a device reuses
// the same array, and it keeps the previous call's contents: the parts that
// must start at zero are cleared (asynchronously, on the caller's stream) by
// each call.  Two calls whose work may overlap on the GPU (different streams
// without ordering between them) race on the array and must not be issued.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace adc {

constexpr size_t kNoAllocScratchBytes = 4u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kMaxDevices] = {0};

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime
// (no link against the driver library).  Signatures as in cuda.h.
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_looked_up = false;

// Id of the calling thread's current context, 0 when there is none or the
// driver entry points are unavailable.
unsigned long long current_ctx_id() {
    if (!g_ctx_fns_looked_up) {
        g_ctx_fns_looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (g_ctx_current == nullptr || g_ctx_id == nullptr) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || ctx == nullptr || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up on the
// first call on a device, and again whenever the device's context has changed.
adc_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = g_noalloc_ptr[dev] != nullptr ? current_ctx_id() : 0;
    if (g_noalloc_ptr[dev] == nullptr || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        // cudaGetSymbolAddress makes the device's primary context current if
        // none is, so the id read after it is the one the address belongs to.
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return ADC_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = current_ctx_id();
    }
    *out = g_noalloc_ptr[dev];
    return ADC_OK;
}

}  // namespace
}  // namespace adc

using namespace adc;

extern "C" adc_status adc_scan_fwd_noalloc(adc_op op, adc_dtype dt, int64_t n, const void *x, void *y, void *stream) {
    if (op < ADC_OP_ADD || op > ADC_OP_MM5 || (dt != ADC_F32 && dt != ADC_F64) || n < 0) return ADC_ERR_INVALID_ARG;
    const auto ok = [](const void *p, int64_t cnt) {
        return cnt == 0 || (p != nullptr && reinterpret_cast<uintptr_t>(p) % 16 == 0);
    };
    if (!ok(x, n) || !ok(y, n)) return ADC_ERR_INVALID_ARG;
    // The scratch a scan of n elements needs grows with its tile count; beyond
    // the fixed array the call is refused before anything is queued.
    if (scan_ws_bytes(op, dt, n) > kNoAllocScratchBytes) return ADC_ERR_WORKSPACE;
    void *scratch = nullptr;
    adc_status st = noalloc_scratch(&scratch);
    if (st != ADC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(scratch, 0, kWsHeader, s) != cudaSuccess) return ADC_ERR_CUDA;
    return scan_fwd(op, dt, n, x, y, scratch, s);
}
