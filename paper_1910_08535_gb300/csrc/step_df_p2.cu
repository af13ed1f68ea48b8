// Split-step axis kernels: double-float pair values, degree 2.
#include "step.cuh"

namespace igapw {

cudaError_t launch_axis_step_df_p2(const AxisStepArgs& a, int mode, cudaStream_t st) {
    return pick_w<DF, 2>(a, mode, st);
}

}  // namespace igapw
