// Allocation-free variant of the source right-hand side (igapw_rhs_source_noalloc).
//
// igapw_rhs_source sums the quadrature samples one axis at a time and keeps the
// two intermediate tensors between the passes in device memory it allocates on
// its first call for a context (after waiting for the context stream).  Some
// callers cannot let a library allocate at that point: hosts that reserve all
// device memory up front and forbid later allocations, schedulers that admit
// work against a fixed device-memory budget, and latency-critical loops that
// cannot afford the wait.  This entry point takes
// its intermediates from one statically sized device array instead and calls no
// allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds IGAPW_NOALLOC_SCRATCH_BYTES for it until the process exits.
// Host code cannot use the symbol as a device address; the device address is
// fetched once per device with cudaGetSymbolAddress (the device current at the
// time of the call), on that device's first call of this entry point.
#include <cstdio>
#include <mutex>

#include "../../include/igapw.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = IGAPW_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the previous call's intermediates.
static __device__ __align__(256) unsigned char g_source_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_source_scratch on the current device (set-up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_source_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int igapw_rhs_source_noalloc(igapw_ctx* ctx, const void* f_dev, void* b_dev) {
    using namespace igapw;
    if (!ctx) return IGAPW_ERR_ARG;
    if (!f_dev || !b_dev) return record_error(ctx, IGAPW_ERR_ARG, "NULL tensor");
    SourceArgs a;
    size_t need = 0;
    cudaStream_t st = nullptr;
    bool f64 = false;
    int rc = source_setup(ctx, f_dev, b_dev, a, need, st, f64);
    if (rc) return rc;
    const size_t half = kScratchBytes / 2;
    if (need > half) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "igapw_rhs_source_noalloc: each intermediate needs %zu bytes but the static scratch "
                      "holds %zu per intermediate (IGAPW_NOALLOC_SCRATCH_BYTES = %zu); use igapw_rhs_source",
                      need, half, kScratchBytes);
        return record_error(ctx, IGAPW_ERR_ARG, msg);
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return record_error(ctx, IGAPW_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // Both intermediates are written in full by the pass that produces them
    // before any pass reads them, so nothing has to be cleared between calls.
    a.work0 = base;
    a.work1 = static_cast<unsigned char*>(base) + half;
    e = launch_source(a, f64 ? 1 : 0, st);
    if (e != cudaSuccess)
        return record_error(ctx, IGAPW_ERR_CUDA, std::string("source: ") + cudaGetErrorString(e));
    return IGAPW_OK;
}
