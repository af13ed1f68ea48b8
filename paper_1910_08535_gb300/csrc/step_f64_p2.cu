// Split-step axis kernels: FP64 values, degree 2.
#include "step.cuh"

namespace igapw {

cudaError_t launch_axis_step_f64_p2(const AxisStepArgs& a, int mode, cudaStream_t st) {
    return pick_w<double, 2>(a, mode, st);
}

}  // namespace igapw
