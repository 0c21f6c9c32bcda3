// msh_step_kt.cu -- launchers of the two Runge-Kutta stages of the Kurganov-Tadmor
// central scheme (Sec. 3.2) on the step kernels of msh_step_kernels.cuh (compiled apart
// from the MUSCL-Hancock instantiations, in parallel).
#include "msh_step_kernels.cuh"

namespace msh {

template <typename T>
cudaError_t launch_step_kt(const StepArgs<T> &a, int ndim, int rows, int stage, cudaStream_t s) {
  if (a.U1 == nullptr) return cudaErrorInvalidValue;
  return stage == 1 ? launch_step_mode<T, 1, false>(a, ndim, rows, s) : launch_step_mode<T, 2, false>(a, ndim, rows, s);
}

template cudaError_t launch_step_kt<float>(const StepArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_step_kt<double>(const StepArgs<double> &, int, int, int, cudaStream_t);

}  // namespace msh
