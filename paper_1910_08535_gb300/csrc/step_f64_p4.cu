// Split-step axis kernels: FP64 values, degree 4.
#include "step.cuh"

namespace igapw {

cudaError_t launch_axis_step_f64_p4(const AxisStepArgs& a, int mode, cudaStream_t st) {
    return pick_w<double, 4>(a, mode, st);
}

}  // namespace igapw
