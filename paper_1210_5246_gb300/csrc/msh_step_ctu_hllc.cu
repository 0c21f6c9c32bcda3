// msh_step_ctu_hllc.cu -- launchers of the corner-transport-upwind form of the characteristic
// step with HLLC (the step kernels of msh_step_kernels.cuh with SCH = 4 and CTU,
// compiled apart in parallel).
#include "msh_step_kernels.cuh"

namespace msh {

template cudaError_t launch_step_ctu<float, 4>(const StepArgs<float> &, int, int, bool, cudaStream_t, int *);
template cudaError_t launch_step_ctu<double, 4>(const StepArgs<double> &, int, int, bool, cudaStream_t, int *);

}  // namespace msh
