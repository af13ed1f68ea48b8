// Chunked explicit-step kernels (FP32-pair mode), degree 4.
#include "chunkstep.cuh"

namespace igapw {

namespace {
template <int W>
cudaError_t pick_mode(const AxisStepArgs& a, int mode, cudaStream_t st) {
    switch (mode) {
        case 0: return run_chunk_step<4, W, 0, IGAPW_CHUNK_ROWS>(a, st);
        case 1: return run_chunk_step<4, W, 1, IGAPW_CHUNK_ROWS>(a, st);
        case 2: return run_chunk_step<4, W, 2, IGAPW_CHUNK_ROWS>(a, st);
        case 3: return run_chunk_step<4, W, 3, IGAPW_CHUNK_ROWS>(a, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_chunk_step_p4(const AxisStepArgs& a, int mode, cudaStream_t st) {
    switch (a.W) {
        case 5: return pick_mode<5>(a, mode, st);
        case 7: return pick_mode<7>(a, mode, st);
        case 9: return pick_mode<9>(a, mode, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace igapw
