// Split-step axis kernels: double-float pair values, degree 4.
#include "step.cuh"

namespace igapw {

cudaError_t launch_axis_step_df_p4(const AxisStepArgs& a, int mode, cudaStream_t st) {
    return pick_w<DF, 4>(a, mode, st);
}

}  // namespace igapw
