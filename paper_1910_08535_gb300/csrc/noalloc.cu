// Allocation-free variant of the source right-hand side (igapw_rhs_source_noalloc).
//
// igapw_rhs_source sums the quadrature samples one axis at a time and keeps the
// two intermediate tensors between the passes in device memory it allocates on
// its first call for a context (after waiting for the context stream).  Some
// callers cannot let a library allocate at that point: hosts that reserve all
// device memory up front and forbid later allocations, schedulers that admit
// work against a fixed device-memory budget, and latency-critical loops that
// cannot afford the wait.  This entry point takes its intermediates from one
// statically sized device array instead and calls no allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds IGAPW_NOALLOC_SCRATCH_BYTES for it until the process exits.
// Host code cannot use the symbol as a device address.  Its device address
// comes from cudaGetSymbolAddress with the context's device current.  This
// translation unit has no kernels, so the array sits in a module of its own,
// which lazy module loading would load (and so allocate) on the first address
// query: igapw_create makes that query, so the array is in place before the
// first call of this entry point.  Every call queries the address again (a
// lookup once the module is loaded), so nothing is cached across
// cudaDeviceReset or contexts.
#include <cstdio>

#include "../../include/igapw.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = IGAPW_NOALLOC_SCRATCH_BYTES;

// Shared by every call on a device; holds the previous call's intermediates.
static __device__ __align__(256) unsigned char g_source_scratch[kScratchBytes];

}  // namespace

namespace igapw {

cudaError_t noalloc_scratch_address(void** out) { return cudaGetSymbolAddress(out, g_source_scratch); }

}  // namespace igapw

extern "C" int igapw_rhs_source_noalloc(igapw_ctx* ctx, const void* f_dev, void* b_dev) {
    using namespace igapw;
    if (!ctx) return IGAPW_ERR_ARG;
    DeviceGuard dg(ctx_device(ctx));
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
    cudaError_t e = noalloc_scratch_address(&base);
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
