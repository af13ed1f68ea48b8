// Split-step dispatch over value type and degree; the kernel is in step.cuh,
// instantiated by step_f64_p*.cu and step_df_p*.cu (compiled in parallel).
#include "kernels.h"

namespace igapw {

cudaError_t launch_axis_step_f64_p2(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_axis_step_f64_p3(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_axis_step_f64_p4(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_axis_step_df_p2(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_axis_step_df_p3(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_axis_step_df_p4(const AxisStepArgs& a, int mode, cudaStream_t st);

cudaError_t launch_chunk_step_p2(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_chunk_step_p3(const AxisStepArgs& a, int mode, cudaStream_t st);
cudaError_t launch_chunk_step_p4(const AxisStepArgs& a, int mode, cudaStream_t st);

cudaError_t launch_axis_step(const AxisStepArgs& a, int mode, bool fp64, int p, cudaStream_t st) {
    // cfg 3: the chunked kernel (chunkstep.cuh), FP32-pair mode, lines_per_block = 32 / 16 / 8
    if (a.cfg == 3) {
        if (fp64) return cudaErrorInvalidValue;
        switch (p) {
            case 2: return launch_chunk_step_p2(a, mode, st);
            case 3: return launch_chunk_step_p3(a, mode, st);
            case 4: return launch_chunk_step_p4(a, mode, st);
        }
        return cudaErrorInvalidValue;
    }
    if (fp64) {
        switch (p) {
            case 2: return launch_axis_step_f64_p2(a, mode, st);
            case 3: return launch_axis_step_f64_p3(a, mode, st);
            case 4: return launch_axis_step_f64_p4(a, mode, st);
        }
    } else {
        switch (p) {
            case 2: return launch_axis_step_df_p2(a, mode, st);
            case 3: return launch_axis_step_df_p3(a, mode, st);
            case 4: return launch_axis_step_df_p4(a, mode, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace igapw
